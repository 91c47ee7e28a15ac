// Block matrices of operators and two-level Toeplitz operators: the building blocks of the
// ultrasound model of Sec. 3, a block matrix H = [H_ij] whose blocks are two-level Toeplitz
// matrices (2-D non-cyclic convolutions), each of which Eq. (7) writes as a zero-padded
// two-level circulant (F (x) F) Diag(h) (F (x) F)^H.
#include <algorithm>
#include <new>
#include <vector>

#include "exec.h"
#include "fm_device.cuh"
#include "pointwise.h"

namespace fm {
namespace {

// Per level, the position in the embedding of length L of generator index k (k < r: k;
// k = r - 1 + d for d in [1, c): L - d) -- the 1-D Toeplitz embedding rule on each axis.
// e[m1 * L2 + m2] = t[k1 * (r2 + c2 - 1) + k2] at the embedded positions, 0 elsewhere.
__global__ void toeplitz2_embed_kernel(const double2* t, int64_t r1, int64_t c1, int64_t r2, int64_t c2, int64_t L1,
                                       int64_t L2, double2* e) {
  const int64_t total = L1 * L2, w = r2 + c2 - 1;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m1 = q / L2, m2 = q % L2;
    const int64_t k1 = m1 < r1 ? m1 : (m1 > L1 - c1 ? r1 - 1 + (L1 - m1) : -1);
    const int64_t k2 = m2 < r2 ? m2 : (m2 > L2 - c2 ? r2 - 1 + (L2 - m2) : -1);
    e[q] = (k1 >= 0 && k2 >= 0) ? t[k1 * w + k2] : make_double2(0.0, 0.0);
  }
}

// index maps of the zero-padding P_in^H (c1 x c2 block of the L1 x L2 grid) and the
// truncation P_out (r1 x r2 block)
std::vector<int32_t> block_index(int64_t a, int64_t b, int64_t L2) {
  std::vector<int32_t> idx((size_t)(a * b));
  for (int64_t i = 0; i < a; ++i)
    for (int64_t j = 0; j < b; ++j) idx[(size_t)(i * b + j)] = (int32_t)(i * L2 + j);
  return idx;
}

int64_t pow2_at_least(int64_t n) {
  int64_t L = 1;
  while (L < n) L <<= 1;
  return L;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" fm_status fm_blocks(const fm_op* blocks, int nrows, int ncols, fm_op* out) {
  clear_error();
  if (!out || !blocks || nrows < 1 || ncols < 1) { set_error("need a grid of at least one block"); return FM_ERR_INVALID_ARG; }
  const int k = nrows * ncols;
  for (int i = 0; i < k; ++i)
    if (!blocks[i]) { set_error("block %d is null", i); return FM_ERR_INVALID_ARG; }
  int64_t rows = 0, cols = 0;
  for (int i = 0; i < nrows; ++i) {
    for (int j = 1; j < ncols; ++j)
      if (blocks[i * ncols + j]->rows != blocks[i * ncols]->rows) {
        set_error("blocks: block (%d, %d) has %lld rows, block (%d, 0) %lld", i, j,
                  (long long)blocks[i * ncols + j]->rows, i, (long long)blocks[i * ncols]->rows);
        return FM_ERR_SHAPE;
      }
    rows += blocks[i * ncols]->rows;
  }
  for (int j = 0; j < ncols; ++j) {
    for (int i = 1; i < nrows; ++i)
      if (blocks[i * ncols + j]->cols != blocks[j]->cols) {
        set_error("blocks: block (%d, %d) has %lld columns, block (0, %d) %lld", i, j,
                  (long long)blocks[i * ncols + j]->cols, j, (long long)blocks[j]->cols);
        return FM_ERR_SHAPE;
      }
    cols += blocks[j]->cols;
  }
  fm_op_s* A = new (std::nothrow) fm_op_s();
  if (!A) return FM_ERR_OOM;
  A->kind = K_BLOCKS;
  cudaGetDevice(&A->device);
  A->real = true;
  for (int i = 0; i < k; ++i) {
    op_retain(blocks[i]);
    A->kids.push_back(blocks[i]);
    A->real = A->real && blocks[i]->real;
  }
  A->blk_r = nrows;
  A->blk_c = ncols;
  A->rows = rows;
  A->cols = cols;
  *out = A;
  return FM_OK;
}

extern "C" fm_status fm_toeplitz2(const void* t, int64_t r1, int64_t c1, int64_t r2, int64_t c2, fm_dtype dt,
                                  void* stream, fm_op* out) {
  clear_error();
  if (!out || !t) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (dt != FM_F32 && dt != FM_F64 && dt != FM_C64 && dt != FM_C128) { set_error("toeplitz2 parameter dtype"); return FM_ERR_DTYPE; }
  if (r1 < 1 || c1 < 1 || r2 < 1 || c2 < 1) { set_error("toeplitz2 shape"); return FM_ERR_SHAPE; }
  const int64_t L1 = pow2_at_least(r1 + c1 - 1), L2 = pow2_at_least(r2 + c2 - 1);
  if (L1 * L2 > (1LL << 24) || r1 * r2 > (1LL << 31) || c1 * c2 > (1LL << 31)) {
    set_error("toeplitz2 embedding %lld x %lld exceeds 2^24 entries", (long long)L1, (long long)L2);
    return FM_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nt = (r1 + c1 - 1) * (r2 + c2 - 1), N = L1 * L2;
  fm_op F1 = nullptr, F2 = nullptr, K = nullptr, KH = nullptr, D = nullptr, Pin = nullptr, PinH = nullptr,
        Pout = nullptr;
  double2* t64 = nullptr;
  double2* e = nullptr;
  double2* spec = nullptr;
  void* ws = nullptr;
  fm_status s = FM_OK;
  // the generator in FP64 (a Diag of the parameter vector does the dtype conversion)
  fm_op Tg = nullptr;
  s = fm_diag(t, nt, dt, stream, &Tg);
  if (s == FM_OK) {
    t64 = Tg->d64;
    cudaError_t err = cudaMalloc(&e, sizeof(double2) * N);
    if (err == cudaSuccess) err = cudaMalloc(&spec, sizeof(double2) * N);
    if (err != cudaSuccess) { set_error("toeplitz2: %s", cudaGetErrorString(err)); s = FM_ERR_OOM; }
  }
  if (s == FM_OK) {
    const int64_t blocks = std::min<int64_t>((N + 255) / 256, 4096);
    toeplitz2_embed_kernel<<<(unsigned)blocks, 256, 0, st>>>(t64, r1, c1, r2, c2, L1, L2, e);
    s = after_launch("toeplitz2_embed_kernel");
  }
  // spectrum of the two-level circulant: (F_L1 (x) F_L2) e, FP64, divided by L1 L2
  if (s == FM_OK) s = fm_fourier(L1, 0, &F1);
  if (s == FM_OK) s = fm_fourier(L2, 0, &F2);
  if (s == FM_OK) {
    const fm_op fs[2] = {F1, F2};
    s = fm_kron(fs, 2, &K);
  }
  if (s == FM_OK) {
    Ctx ctx;
    ctx.st = st;
    int dev = 0;
    cudaGetDevice(&dev);
    s = device_tables(dev, &ctx.tabs);
    View vi, vo;
    vi.p = e;
    vi.dt = FM_C128;
    vi.n = vi.ld = vi.ostride = N;
    vo = vi;
    vo.p = spec;
    if (s == FM_OK) {
      ctx.dry = true;
      s = exec(K, false, vi, vo, 1, 0, ctx);
    }
    if (s == FM_OK && ctx.peak) {
      cudaError_t err = cudaMalloc(&ws, ctx.peak);
      if (err != cudaSuccess) { set_error("toeplitz2: %s", cudaGetErrorString(err)); s = FM_ERR_OOM; }
    }
    if (s == FM_OK) {
      ctx.dry = false;
      ctx.base = (char*)ws;
      ctx.used = ctx.peak = 0;
      s = exec(K, false, vi, vo, 1, 0, ctx);
    }
    if (s == FM_OK) {
      PwArgs a;
      a.ncols = 1;
      a.n_out = N;
      a.in = spec;
      a.in_ld = a.in_ostride = N;
      a.in_cplx = 1;
      a.out = e;          // reuse: e <- spec / (L1 L2)
      a.out_ld = a.out_ostride = N;
      a.out_cplx = 1;
      a.scale = 1.0 / (double)N;
      s = pointwise_launch(a, true, st);
    }
  }
  if (s == FM_OK) {
    // Diag of the scaled spectrum in the parameter's precision family (complex)
    s = fm_diag(e, N, FM_C128, stream, &D);
  }
  if (s == FM_OK) s = fm_hermitian(K, &KH);
  if (s == FM_OK) {
    const std::vector<int32_t> iin = block_index(c1, c2, L2), iout = block_index(r1, r2, L2);
    s = fm_partial(iin.data(), c1 * c2, N, stream, &Pin);
    if (s == FM_OK) s = fm_partial(iout.data(), r1 * r2, N, stream, &Pout);
  }
  if (s == FM_OK) s = fm_hermitian(Pin, &PinH);
  if (s == FM_OK) {
    // T2 = P_out (F (x) F)^H Diag(F2 e / (L1 L2)) (F (x) F) P_in^H
    const fm_op terms[5] = {Pout, KH, D, K, PinH};
    s = fm_product(terms, 5, out);
  }
  if (ws || e || spec) cudaStreamSynchronize(st);
  if (ws) cudaFree(ws);
  if (e) cudaFree(e);
  if (spec) cudaFree(spec);
  for (fm_op h : {Tg, F1, F2, K, KH, D, Pin, PinH, Pout})
    if (h) fm_release(h);
  return s;
}
