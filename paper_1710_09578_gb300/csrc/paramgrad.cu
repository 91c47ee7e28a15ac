// Gradients with respect to the parameter vectors of Diag, Circulant and Toeplitz operators.
//
// The operators of Sec. 2.1.1 are built from parameter vectors (a diagonal d, the first
// column c of a circulant, the generator t of a Toeplitz matrix), and Y = A(theta) X is
// bilinear in (theta, X).  For a real loss with upstream gradient G = dloss/dconj(Y), the
// gradient of parameter entry k is the sum, over the columns and over the matrix entries
// (i, j) that hold theta_k, of G[i] conj(X[j]) -- its real part for a real parameter:
//   Diag       grad_d[i] = sum_c G[i] conj(X[i]);
//   Circulant  grad_c[k] = sum_c sum_i G[i] conj(X[(i - k) mod n]), the circular correlation,
//              evaluated as (1/n) F^H sum_c (F G) conj(F X) (Eq. (5) read backwards);
//   Toeplitz   the same correlation of G and X zero-padded to the embedding length L, read
//              at the embedding's positions (entry m < rows at m, entry rows - 1 + d at L - d).
// For a leaf inside a Product nothing of the forward pass is stored: the leaf's input is
// recomputed from X by the terms applied before it, and the gradient at its output by the
// adjoints of the terms applied after it.
#include <algorithm>
#include <vector>

#include "exec.h"
#include "fm_device.cuh"
#include "pointwise.h"

namespace fm {
namespace {

// out[i] = scale * sum_c a[c * lda + i] * conj(b[c * ldb + i]), i < n (complex, FP32 or FP64)
template <typename T>
__global__ void colsum_conj_kernel(const typename Cx<T>::t* a, int64_t lda, const typename Cx<T>::t* b,
                                   int64_t ldb, typename Cx<T>::t* out, int64_t n, int64_t ncols, T scale) {
  typedef typename Cx<T>::t C;
  pdl_launch_dependents();
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    C acc = cmake((T)0, (T)0);
    for (int64_t c = 0; c < ncols; ++c) acc = cadd(acc, cmul(gld(a + c * lda + i), cconj(gld(b + c * ldb + i))));
    gst(out + i, cscale(acc, scale));
  }
}

// grad[m] = r[m] for m < rows and r[L - (m - rows + 1)] after (the Toeplitz embedding; the
// identity for a circulant with rows = n = L); real_out keeps the real part only
template <typename T>
__global__ void embed_gather_kernel(const typename Cx<T>::t* r, int64_t rows, int64_t plen, int64_t L, void* out,
                                    int real_out) {
  pdl_launch_dependents();
  pdl_wait();
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < plen; m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = m < rows ? m : L - (m - rows + 1);
    const typename Cx<T>::t v = gld(r + src);
    if (real_out) gst(reinterpret_cast<T*>(out) + m, v.x);
    else gst(reinterpret_cast<typename Cx<T>::t*>(out) + m, v);
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

struct Item {
  const fm_op_s* op;
  bool adj;
};

void flatten(const fm_op_s* A, bool adj, std::vector<Item>& seq) {
  if (A->kind == K_PRODUCT) {
    const int k = (int)A->kids.size();
    if (!adj) for (int i = k - 1; i >= 0; --i) flatten(A->kids[i], adj, seq);
    else for (int i = 0; i < k; ++i) flatten(A->kids[i], adj, seq);
  } else if (A->kind == K_HERMITIAN) {
    flatten(A->kids[0], !adj, seq);
  } else {
    seq.push_back({A, adj});
  }
}

View packed(void* p, fm_dtype dt, int64_t n) {
  View v;
  v.p = p;
  v.dt = dt;
  v.n = n;
  v.ostride = n;
  v.ld = n;
  return v;
}

// Apply items [0, k) of seq in order (forward chain), or the adjoints of items (k, end) from
// the last one down (the gradient chain), from `in` into a packed complex temporary.
fm_status run_chain(const std::vector<Item>& seq, int lo, int hi, bool backwards, const View& in, fm_dtype cdt,
                    int64_t ncols, View* out, Ctx& ctx) {
  View cur = in;
  const int n = hi - lo;
  for (int s = 0; s < n; ++s) {
    const Item& it = backwards ? seq[hi - 1 - s] : seq[lo + s];
    const bool adj = backwards ? !it.adj : it.adj;
    const int64_t nout = adj ? it.op->cols : it.op->rows;
    fm_dtype od;
    FM_TRY(natural_out_dtype(it.op, cur.dt, &od));
    View nx = packed(ctx.alloc((size_t)nout * ncols * dtype_size(od)), od, nout);
    FM_TRY(exec(it.op, adj, cur, nx, ncols, 0, ctx));
    cur = nx;
  }
  if (cur.dt != cdt) {
    // the leaf's gradient takes complex columns
    View nx = packed(ctx.alloc((size_t)cur.n * ncols * dtype_size(cdt)), cdt, cur.n);
    PwArgs a;
    a.ncols = ncols;
    a.n_out = cur.n;
    a.in = cur.p;
    a.in_ld = cur.ld;
    a.in_ostride = cur.ostride;
    a.in_cplx = is_complex(cur.dt);
    a.out = nx.p;
    a.out_ld = nx.ld;
    a.out_ostride = nx.ostride;
    a.out_cplx = 1;
    if (!ctx.dry) FM_TRY(pointwise_launch(a, is_double(cdt), ctx.st));
    cur = nx;
  }
  *out = cur;
  return FM_OK;
}

// Correlation sum of one leaf from its complex input Z and output gradient Gt into racc:
// Diag: sum_c Gt conj(Z) (length n); circulant / Toeplitz: (1/L) F^H sum_c F(Gt) conj(F(Z))
// (length L, columns zero-padded to L).
template <typename T>
fm_status leaf_grad(const fm_op_s* leaf, const View& Z, const View& Gt, int64_t ncols, typename Cx<T>::t* racc,
                    Ctx& ctx) {
  typedef typename Cx<T>::t C;
  const cudaStream_t st = ctx.st;
  if (leaf->kind == K_DIAG) {
    if (ctx.dry) return FM_OK;
    return pdl_go("colsum_conj_kernel", colsum_conj_kernel<T>, dim3(grid_for(leaf->rows)), dim3(256), 0, st,
                  (const C*)Gt.p, Gt.ld, (const C*)Z.p, Z.ld, racc, leaf->rows, ncols, (T)1);
  }
  const int64_t L = leaf->L;
  const BigPlan* big = leaf->big.L == L ? &leaf->big : nullptr;
  const fm_dtype cdt = sizeof(T) == 4 ? FM_C64 : FM_C128;
  View Zh = packed(ctx.alloc((size_t)L * ncols * sizeof(C)), cdt, L);
  View Gh = packed(ctx.alloc((size_t)L * ncols * sizeof(C)), cdt, L);
  FM_TRY(exec_dft(L, big, -1, Z, leaf->cols, Zh, ncols, 1.0, ctx));
  FM_TRY(exec_dft(L, big, -1, Gt, leaf->rows, Gh, ncols, 1.0, ctx));
  View R = packed(ctx.alloc((size_t)L * sizeof(C)), cdt, L);
  if (!ctx.dry)
    FM_TRY(pdl_go("colsum_conj_kernel", colsum_conj_kernel<T>, dim3(grid_for(L)), dim3(256), 0, st,
                  (const C*)Gh.p, Gh.ld, (const C*)Zh.p, Zh.ld, (C*)R.p, L, ncols, (T)(1.0 / (double)L)));
  View r = packed(racc, cdt, L);
  return exec_dft(L, big, +1, R, L, r, 1, 1.0, ctx);
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" fm_status fm_param_grad(fm_op A, fm_op leaf, const void* X, int64_t ldx, fm_dtype xdt, const void* G,
                                   int64_t ldg, fm_dtype gdt, int64_t ncols, void* grad, fm_dtype grad_dt,
                                   void* stream) {
  clear_error();
  if (!A || !leaf || !grad) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (leaf->kind != K_DIAG && leaf->kind != K_CIRCULANT && leaf->kind != K_TOEPLITZ) {
    set_error("parameter gradients exist for Diag, Circulant and Toeplitz operators");
    return FM_ERR_INVALID_ARG;
  }
  if (leaf->L == 1 && leaf->kind != K_DIAG) { set_error("parameter gradient of a 1 x 1 operator"); return FM_ERR_UNSUPPORTED; }
  if (ncols < 1 || !X || !G) { set_error("need at least one column of X and G"); return FM_ERR_INVALID_ARG; }
  if (xdt != FM_F32 && xdt != FM_F64 && xdt != FM_C64 && xdt != FM_C128) { set_error("X dtype"); return FM_ERR_DTYPE; }
  fm_dtype nd;
  FM_TRY(natural_out_dtype(A, xdt, &nd));
  if (gdt != nd) { set_error("G must have the dtype of A X (%d)", (int)nd); return FM_ERR_DTYPE; }
  const bool dbl = is_double(xdt);
  const fm_dtype cdt = dbl ? FM_C128 : FM_C64;
  const fm_dtype want = leaf->real ? (dbl ? FM_F64 : FM_F32) : cdt;
  if (grad_dt != want) { set_error("grad dtype must be %d for this leaf and X", (int)want); return FM_ERR_DTYPE; }
  if (ldx < A->cols || ldg < A->rows) { set_error("leading dimension smaller than the column length"); return FM_ERR_SHAPE; }
  std::vector<Item> seq;
  flatten(A, false, seq);
  int pos = -1;
  for (int i = 0; i < (int)seq.size(); ++i) {
    if (seq[i].op != leaf) continue;
    if (seq[i].adj) { set_error("the leaf appears as an adjoint; only A(theta), not A(theta)^H, is supported"); return FM_ERR_UNSUPPORTED; }
    if (pos >= 0) { set_error("the leaf appears more than once in the product"); return FM_ERR_UNSUPPORTED; }
    pos = i;
  }
  if (pos < 0) { set_error("the leaf is not a term of the operator's product"); return FM_ERR_INVALID_ARG; }
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  if (dev != A->device) { set_error("operator lives on device %d, current is %d", A->device, dev); return FM_ERR_INVALID_ARG; }
  Ctx ctx;
  ctx.st = (cudaStream_t)stream;
  FM_TRY(device_tables(dev, &ctx.tabs));
  View xin;
  xin.p = (void*)X;
  xin.dt = xdt;
  xin.ld = ldx;
  xin.n = xin.ostride = A->cols;
  View gin;
  gin.p = (void*)G;
  gin.dt = gdt;
  gin.ld = ldg;
  gin.n = gin.ostride = A->rows;
  const int64_t plen = leaf->kind == K_TOEPLITZ ? leaf->rows + leaf->cols - 1 : leaf->rows;
  auto run = [&]() -> fm_status {
    View Z, Gt;
    FM_TRY(run_chain(seq, 0, pos, false, xin, cdt, ncols, &Z, ctx));
    FM_TRY(run_chain(seq, pos + 1, (int)seq.size(), true, gin, cdt, ncols, &Gt, ctx));
    const int64_t rlen = leaf->kind == K_DIAG ? leaf->rows : leaf->L;
    void* racc = ctx.alloc((size_t)rlen * dtype_size(cdt));
    if (dbl) FM_TRY(leaf_grad<double>(leaf, Z, Gt, ncols, (double2*)racc, ctx));
    else FM_TRY(leaf_grad<float>(leaf, Z, Gt, ncols, (float2*)racc, ctx));
    if (ctx.dry) return FM_OK;
    const int64_t rows = leaf->kind == K_DIAG ? plen : leaf->rows;
    const int64_t L = leaf->kind == K_DIAG ? plen : leaf->L;
    const int real_out = leaf->real ? 1 : 0;
    if (dbl)
      return pdl_go("embed_gather_kernel", embed_gather_kernel<double>, dim3(grid_for(plen)), dim3(256), 0, ctx.st,
                    (const double2*)racc, rows, plen, L, grad, real_out);
    return pdl_go("embed_gather_kernel", embed_gather_kernel<float>, dim3(grid_for(plen)), dim3(256), 0, ctx.st,
                  (const float2*)racc, rows, plen, L, grad, real_out);
  };
  std::lock_guard<std::mutex> lk(A->ws.mu);
  ctx.dry = true;
  FM_TRY(run());
  if (ctx.peak > A->ws.bytes) {
    if (A->ws.ptr) {
      FM_CUDA(cudaStreamSynchronize(ctx.st));
      cudaFree(A->ws.ptr);
      A->ws.ptr = nullptr;
      A->ws.bytes = 0;
    }
    FM_CUDA(cudaMalloc(&A->ws.ptr, ctx.peak));
    A->ws.bytes = ctx.peak;
  }
  ctx.dry = false;
  ctx.base = (char*)A->ws.ptr;
  ctx.used = 0;
  ctx.peak = 0;
  return run();
}
