// C ABI of the structured-operator library: constructors, validation, workspaces and the
// forward / backward transforms (Eq. (3), Eq. (4)).  Argument checks run on the host
// before anything is launched; nothing throws across the ABI.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "exec.h"
#include "fft.h"
#include "pointwise.h"

namespace fm {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
}
void clear_error() { t_err.clear(); }

static std::mutex g_tab_mu;
static DeviceTables g_tabs[64];
static bool g_tab_ready[64] = {false};

fm_status device_tables(int device, DeviceTables** out) {
  if (device < 0 || device >= 64) { set_error("device %d out of range", device); return FM_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (!g_tab_ready[device]) {
    DeviceTables& t = g_tabs[device];
    FM_CUDA(cudaMalloc(&t.tw32, sizeof(float2) * kTwMax));
    FM_CUDA(cudaMalloc(&t.tw64, sizeof(double2) * kTwMax));
    FM_TRY(twiddle_launch(kTwMax, t.tw32, t.tw64, nullptr));
    FM_CUDA(cudaMalloc(&t.twp32, sizeof(float2) * kPassTwEntries));
    FM_CUDA(cudaMalloc(&t.twp64, sizeof(double2) * kPassTwEntries));
    FM_TRY(pass_twiddle_launch(t.twp32, t.twp64, nullptr));
    FM_CUDA(cudaStreamSynchronize(nullptr));
    g_tab_ready[device] = true;
  }
  *out = &g_tabs[device];
  return FM_OK;
}

DeviceTables* device_tables_if_ready(int device) {
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_tab_mu);
  return g_tab_ready[device] ? &g_tabs[device] : nullptr;
}

void op_retain(fm_op_s* A) { A->refs.fetch_add(1); }

static void free_op(fm_op_s* A) {
  void* bufs[] = {A->spec64, A->spec32, A->spec64_perm, A->spec32_perm, A->d64, A->d32, A->dr64,
                  A->dr32,   A->idx,    A->inv,         A->ws.ptr,      A->m32, A->m64};
  for (void* p : bufs)
    if (p) cudaFree(p);
  free_big_plan(&A->big);
  for (auto* k : A->kids) op_release(k);
  delete A;
}

void op_release(fm_op_s* A) {
  if (A && A->refs.fetch_sub(1) == 1) free_op(A);
}

static fm_op_s* new_op(OpKind k) {
  fm_op_s* A = new (std::nothrow) fm_op_s();
  if (!A) return nullptr;
  A->kind = k;
  cudaGetDevice(&A->device);
  return A;
}

static bool pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }
static bool param_dtype_ok(fm_dtype d) { return d == FM_F32 || d == FM_F64 || d == FM_C64 || d == FM_C128; }

// Copy a parameter array (host or device memory) of n elements to a device c128 buffer of
// length dst_len (zero-padded).
static fm_status param_to_c128(const void* src, fm_dtype dt, int64_t n, int64_t dst_len, double2** out,
                               cudaStream_t st) {
  void* staging = nullptr;
  const size_t bytes = (size_t)n * dtype_size(dt);
  FM_CUDA(cudaMalloc(&staging, bytes > 0 ? bytes : 1));
  cudaError_t e = cudaMemcpyAsync(staging, src, bytes, cudaMemcpyDefault, st);
  if (e != cudaSuccess) {
    cudaFree(staging);
    set_error("copying the parameter array: %s", cudaGetErrorString(e));
    return FM_ERR_CUDA;
  }
  double2* d = nullptr;
  e = cudaMalloc(&d, sizeof(double2) * (size_t)std::max<int64_t>(dst_len, 1));
  if (e != cudaSuccess) {
    cudaFree(staging);
    set_error("cudaMalloc: %s", cudaGetErrorString(e));
    return FM_ERR_OOM;
  }
  fm_status s = to_c128_launch(staging, dt, n, dst_len, d, st);
  cudaStreamSynchronize(st);
  cudaFree(staging);
  if (s != FM_OK) {
    cudaFree(d);
    return s;
  }
  *out = d;
  return FM_OK;
}

// Spectrum of the (embedding) circulant with first column c64 (length L), divided by L.
static fm_status build_spectrum(fm_op_s* A, const double2* c64, int64_t L, cudaStream_t st) {
  A->L = L;
  // Toeplitz operators (many small ones in a FISTA batch) keep the plan for long embeddings
  // only; Circulant and Fourier get it from 2^11 for small FP64 problems
  if (L > fft_max_tile<double>() || (A->kind == K_CIRCULANT && L >= kBigPlanMin))
    FM_TRY(make_big_plan(L, &A->big, st));
  FM_CUDA(cudaMalloc(&A->spec64, sizeof(double2) * L));
  FM_CUDA(cudaMalloc(&A->spec32, sizeof(float2) * L));
  if (A->big.L) {
    FM_CUDA(cudaMalloc(&A->spec64_perm, sizeof(double2) * L));
    FM_CUDA(cudaMalloc(&A->spec32_perm, sizeof(float2) * L));
  }
  FM_TRY(construction_fft64(c64, A->spec64, L, A->big.L ? &A->big : nullptr, st));
  double* dcap = nullptr;
  FM_CUDA(cudaMalloc(&dcap, sizeof(double)));
  fm_status s = spec_cap_launch(A->spec64, L, 1.0, dcap, st);
  if (s == FM_OK)
    s = spectrum_finish_launch(A->spec64, A->spec32, A->spec64_perm, A->spec32_perm, L, A->big.N1, A->big.N2,
                               1.0 / (double)L, st);
  if (s == FM_OK) {
    cudaError_t e = cudaMemcpyAsync(&A->cap, dcap, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("spectrum: %s", cudaGetErrorString(e));
      s = FM_ERR_CUDA;
    }
  }
  cudaFree(dcap);
  return s;
}

// Scalar operators of size 1 keep their single entry as a diagonal.
static fm_status scalar_as_diag(fm_op_s* A, double2* c64, cudaStream_t st) {
  A->d64 = c64;
  FM_CUDA(cudaMalloc(&A->d32, sizeof(float2)));
  if (A->real) {
    FM_CUDA(cudaMalloc(&A->dr64, sizeof(double)));
    FM_CUDA(cudaMalloc(&A->dr32, sizeof(float)));
  }
  FM_TRY(diag_finish_launch(A->d64, 1, A->d32, A->dr64, A->dr32, st));
  FM_CUDA(cudaStreamSynchronize(st));
  double2 h;
  FM_CUDA(cudaMemcpy(&h, A->d64, sizeof(h), cudaMemcpyDeviceToHost));
  A->cap = h.x * h.x + h.y * h.y;
  return FM_OK;
}

static fm_status finish(fm_op_s* A, fm_status s, fm_op* out) {
  if (s != FM_OK) {
    free_op(A);
    return s;
  }
  *out = A;
  return FM_OK;
}

static fm_status check_kids(const fm_op* t, int k) {
  if (!t || k < 1) { set_error("need at least one operator"); return FM_ERR_INVALID_ARG; }
  for (int i = 0; i < k; ++i)
    if (!t[i]) { set_error("operator %d is null", i); return FM_ERR_INVALID_ARG; }
  return FM_OK;
}

static fm_op_s* composite(OpKind kind, const fm_op* t, int k) {
  fm_op_s* A = new_op(kind);
  if (!A) return nullptr;
  for (int i = 0; i < k; ++i) {
    op_retain(t[i]);
    A->kids.push_back(t[i]);
  }
  A->real = true;
  for (auto* c : A->kids) A->real = A->real && c->real;
  return A;
}

// ------------------------------------------------------------------ transforms
static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

static bool dtype_valid(int d) { return d >= FM_I8 && d <= FM_C128; }

static fm_status apply(fm_op A, bool adj, const void* X, int64_t ldx, fm_dtype xdt, void* Y, int64_t ldy,
                       fm_dtype ydt, int64_t ncols, void* stream) {
  clear_error();
  if (!A) { set_error("null operator"); return FM_ERR_INVALID_ARG; }
  if (ncols < 0) { set_error("ncols < 0"); return FM_ERR_INVALID_ARG; }
  if (!dtype_valid(xdt) || !dtype_valid(ydt)) { set_error("bad dtype"); return FM_ERR_INVALID_ARG; }
  const int64_t nin = adj ? A->rows : A->cols, nout = adj ? A->cols : A->rows;
  fm_dtype nd;
  FM_TRY(natural_out_dtype(A, xdt, &nd));
  const bool real_part = is_complex(nd) && ydt == real_of(nd);
  if (nd != ydt && !real_part) {
    set_error("output dtype must be %d (or its real type) for this operator and input", (int)nd);
    return FM_ERR_DTYPE;
  }
  if (ncols == 0) return FM_OK;
  if (!X || !Y) { set_error("null data pointer"); return FM_ERR_INVALID_ARG; }
  if (ldx < nin || ldy < nout) { set_error("leading dimension smaller than the column length"); return FM_ERR_SHAPE; }
  const size_t xb = (size_t)((ncols - 1) * ldx + nin) * dtype_size(xdt);
  const size_t yb = (size_t)((ncols - 1) * ldy + nout) * dtype_size(ydt);
  if (overlap(X, xb, Y, yb)) { set_error("output overlaps input"); return FM_ERR_ALIAS; }
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  if (dev != A->device) { set_error("operator lives on device %d, current is %d", A->device, dev); return FM_ERR_INVALID_ARG; }
  Ctx ctx;
  ctx.st = (cudaStream_t)stream;
  FM_TRY(device_tables(dev, &ctx.tabs));
  View in, out;
  in.p = (void*)X;
  in.dt = xdt;
  in.ld = ldx;
  in.n = nin;
  in.ostride = nin;
  out.p = Y;
  out.dt = ydt;
  out.ld = ldy;
  out.n = nout;
  out.ostride = nout;
  std::lock_guard<std::mutex> lk(A->ws.mu);
  ctx.dry = true;
  FM_TRY(exec(A, adj, in, out, ncols, 0, ctx));
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
  return exec(A, adj, in, out, ncols, 0, ctx);
}

}  // namespace fm

using namespace fm;

extern "C" {

fm_status fm_fourier(int64_t n, int ortho, fm_op* out) {
  clear_error();
  if (!out) { set_error("null output"); return FM_ERR_INVALID_ARG; }
  if (!pow2(n) || n > (1LL << 24)) { set_error("Fourier size %lld: power of two up to 2^24", (long long)n); return FM_ERR_UNSUPPORTED; }
  fm_op_s* A = new_op(K_FOURIER);
  if (!A) return FM_ERR_OOM;
  A->rows = A->cols = A->L = n;
  A->ortho = ortho ? 1 : 0;
  A->real = n == 1;
  fm_status s = FM_OK;
  if (n >= kBigPlanMin) s = make_big_plan(n, &A->big, nullptr);
  if (s == FM_OK) {
    DeviceTables* t;
    s = device_tables(A->device, &t);
  }
  if (s == FM_OK && A->big.L) {
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
  }
  return finish(A, s, out);
}

fm_status fm_circulant(const void* c, int64_t n, fm_dtype dt, void* stream, fm_op* out) {
  clear_error();
  if (!out || !c) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (!param_dtype_ok(dt)) { set_error("circulant parameter dtype"); return FM_ERR_DTYPE; }
  if (!pow2(n) || n > (1LL << 24)) { set_error("circulant size %lld: power of two up to 2^24", (long long)n); return FM_ERR_UNSUPPORTED; }
  fm_op_s* A = new_op(K_CIRCULANT);
  if (!A) return FM_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  A->rows = A->cols = n;
  A->real = !is_complex(dt);
  double2* c64 = nullptr;
  fm_status s = param_to_c128(c, dt, n, n, &c64, st);
  if (s != FM_OK) return finish(A, s, out);
  DeviceTables* t;
  s = device_tables(A->device, &t);
  if (s == FM_OK) s = noalloc_prepare(A->device);
  if (s == FM_OK) {
    if (n == 1) {
      A->L = 1;
      return finish(A, scalar_as_diag(A, c64, st), out);
    }
    s = build_spectrum(A, c64, n, st);
  }
  cudaFree(c64);
  return finish(A, s, out);
}

fm_status fm_toeplitz(const void* tvec, int64_t rows, int64_t cols, fm_dtype dt, void* stream, fm_op* out) {
  clear_error();
  if (!out || !tvec) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (!param_dtype_ok(dt)) { set_error("toeplitz parameter dtype"); return FM_ERR_DTYPE; }
  if (rows < 1 || cols < 1) { set_error("toeplitz shape"); return FM_ERR_SHAPE; }
  int64_t L = 1;
  while (L < rows + cols - 1) L <<= 1;
  if (L > (1LL << 24)) { set_error("toeplitz embedding length %lld > 2^24", (long long)L); return FM_ERR_UNSUPPORTED; }
  fm_op_s* A = new_op(K_TOEPLITZ);
  if (!A) return FM_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  A->rows = rows;
  A->cols = cols;
  A->real = !is_complex(dt);
  double2* t64 = nullptr;
  fm_status s = param_to_c128(tvec, dt, rows + cols - 1, rows + cols - 1, &t64, st);
  if (s != FM_OK) return finish(A, s, out);
  DeviceTables* tb;
  s = device_tables(A->device, &tb);
  if (s == FM_OK && L == 1) {
    A->L = 1;
    return finish(A, scalar_as_diag(A, t64, st), out);
  }
  double2* emb = nullptr;
  if (s == FM_OK) {
    cudaError_t e = cudaMalloc(&emb, sizeof(double2) * L);
    if (e != cudaSuccess) { set_error("cudaMalloc"); s = FM_ERR_OOM; }
  }
  if (s == FM_OK) s = toeplitz_embed_launch(t64, rows, cols, L, emb, st);
  if (s == FM_OK) s = build_spectrum(A, emb, L, st);
  cudaStreamSynchronize(st);
  if (emb) cudaFree(emb);
  cudaFree(t64);
  return finish(A, s, out);
}

fm_status fm_hadamard(int log2n, fm_had_mode mode, fm_op* out) {
  clear_error();
  if (!out) { set_error("null output"); return FM_ERR_INVALID_ARG; }
  if (mode < FM_HAD_FP32 || mode > FM_HAD_INT8) { set_error("bad Hadamard mode"); return FM_ERR_INVALID_ARG; }
  if (log2n < 0 || log2n > 24) { set_error("Hadamard log2n in [0, 24]"); return FM_ERR_UNSUPPORTED; }
  if ((mode == FM_HAD_BF16 || mode == FM_HAD_BF16X2) && (log2n < 4 || log2n > 16)) {
    set_error("BF16 Hadamard needs 4 <= log2n <= 16");
    return FM_ERR_UNSUPPORTED;
  }
  fm_op_s* A = new_op(K_HADAMARD);
  if (!A) return FM_ERR_OOM;
  A->rows = A->cols = A->L = 1LL << log2n;
  A->log2n = log2n;
  A->had_mode = mode;
  A->real = true;
  *out = A;
  return FM_OK;
}

fm_status fm_diag(const void* d, int64_t n, fm_dtype dt, void* stream, fm_op* out) {
  clear_error();
  if (!out || !d) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (!param_dtype_ok(dt)) { set_error("diag parameter dtype"); return FM_ERR_DTYPE; }
  if (n < 1) { set_error("diag size"); return FM_ERR_SHAPE; }
  fm_op_s* A = new_op(K_DIAG);
  if (!A) return FM_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  A->rows = A->cols = n;
  A->real = !is_complex(dt);
  fm_status s = param_to_c128(d, dt, n, n, &A->d64, st);
  if (s == FM_OK) {
    cudaError_t e = cudaMalloc(&A->d32, sizeof(float2) * n);
    if (e == cudaSuccess && A->real) e = cudaMalloc(&A->dr64, sizeof(double) * n);
    if (e == cudaSuccess && A->real) e = cudaMalloc(&A->dr32, sizeof(float) * n);
    if (e != cudaSuccess) { set_error("cudaMalloc"); s = FM_ERR_OOM; }
  }
  if (s == FM_OK) s = diag_finish_launch(A->d64, n, A->d32, A->dr64, A->dr32, st);
  if (s == FM_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
  }
  return finish(A, s, out);
}

fm_status fm_partial(const int32_t* idx, int64_t m, int64_t n, void* stream, fm_op* out) {
  clear_error();
  if (!out || !idx) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (m < 1 || n < 1 || m > n) { set_error("partial shape m=%lld n=%lld", (long long)m, (long long)n); return FM_ERR_SHAPE; }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> h(m);
  cudaError_t e = cudaMemcpyAsync(h.data(), idx, sizeof(int32_t) * m, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { set_error("reading indices: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
  std::vector<int32_t> inv(n, -1);
  for (int64_t r = 0; r < m; ++r) {
    if (h[r] < 0 || h[r] >= n) { set_error("index %d at %lld out of range", h[r], (long long)r); return FM_ERR_INVALID_ARG; }
    if (inv[h[r]] >= 0) { set_error("index %d repeated", h[r]); return FM_ERR_INVALID_ARG; }
    inv[h[r]] = (int32_t)r;
  }
  fm_op_s* A = new_op(K_PARTIAL);
  if (!A) return FM_ERR_OOM;
  A->rows = m;
  A->cols = n;
  A->real = true;
  A->idx_host = h;
  fm_status s = FM_OK;
  e = cudaMalloc(&A->idx, sizeof(int32_t) * m);
  if (e == cudaSuccess) e = cudaMalloc(&A->inv, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = cudaMemcpy(A->idx, h.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(A->inv, inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { set_error("partial upload: %s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
  return finish(A, s, out);
}

fm_status fm_product(const fm_op* terms, int k, fm_op* out) {
  clear_error();
  if (!out) return FM_ERR_INVALID_ARG;
  FM_TRY(check_kids(terms, k));
  for (int i = 0; i + 1 < k; ++i)
    if (terms[i]->cols != terms[i + 1]->rows) {
      set_error("product: term %d has %lld columns, term %d has %lld rows", i, (long long)terms[i]->cols, i + 1,
                (long long)terms[i + 1]->rows);
      return FM_ERR_SHAPE;
    }
  fm_op_s* A = composite(K_PRODUCT, terms, k);
  if (!A) return FM_ERR_OOM;
  A->rows = terms[0]->rows;
  A->cols = terms[k - 1]->cols;
  *out = A;
  return FM_OK;
}

fm_status fm_sum(const fm_op* terms, int k, fm_op* out) {
  clear_error();
  if (!out) return FM_ERR_INVALID_ARG;
  FM_TRY(check_kids(terms, k));
  for (int i = 1; i < k; ++i)
    if (terms[i]->rows != terms[0]->rows || terms[i]->cols != terms[0]->cols) {
      set_error("sum: terms differ in shape");
      return FM_ERR_SHAPE;
    }
  fm_op_s* A = composite(K_SUM, terms, k);
  if (!A) return FM_ERR_OOM;
  A->rows = terms[0]->rows;
  A->cols = terms[0]->cols;
  *out = A;
  return FM_OK;
}

fm_status fm_blkdiag(const fm_op* blocks, int k, fm_op* out) {
  clear_error();
  if (!out) return FM_ERR_INVALID_ARG;
  FM_TRY(check_kids(blocks, k));
  fm_op_s* A = composite(K_BLKDIAG, blocks, k);
  if (!A) return FM_ERR_OOM;
  for (int i = 0; i < k; ++i) {
    A->rows += blocks[i]->rows;
    A->cols += blocks[i]->cols;
  }
  *out = A;
  return FM_OK;
}

fm_status fm_kron(const fm_op* factors, int k, fm_op* out) {
  clear_error();
  if (!out) return FM_ERR_INVALID_ARG;
  FM_TRY(check_kids(factors, k));
  int64_t r = 1, c = 1;
  for (int i = 0; i < k; ++i) {
    if (factors[i]->rows > (1LL << 40) / r || factors[i]->cols > (1LL << 40) / c) {
      set_error("kron: too large");
      return FM_ERR_SHAPE;
    }
    r *= factors[i]->rows;
    c *= factors[i]->cols;
  }
  fm_op_s* A = composite(K_KRON, factors, k);
  if (!A) return FM_ERR_OOM;
  A->rows = r;
  A->cols = c;
  *out = A;
  return FM_OK;
}

fm_status fm_hermitian(fm_op X, fm_op* out) {
  clear_error();
  if (!out || !X) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  fm_op_s* A = composite(K_HERMITIAN, &X, 1);
  if (!A) return FM_ERR_OOM;
  A->rows = X->cols;
  A->cols = X->rows;
  *out = A;
  return FM_OK;
}

fm_status fm_shape(fm_op A, int64_t* rows, int64_t* cols) {
  if (!A || !rows || !cols) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  *rows = A->rows;
  *cols = A->cols;
  return FM_OK;
}

fm_status fm_is_real(fm_op A, int* r) {
  if (!A || !r) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  *r = A->real ? 1 : 0;
  return FM_OK;
}

fm_status fm_out_dtype(fm_op A, fm_dtype in, fm_dtype* out) {
  clear_error();
  if (!A || !out || !dtype_valid(in)) { set_error("bad argument"); return FM_ERR_INVALID_ARG; }
  return natural_out_dtype(A, in, out);
}

fm_status fm_forward(fm_op A, const void* X, int64_t ldx, fm_dtype xdt, void* Y, int64_t ldy, fm_dtype ydt,
                     int64_t ncols, void* stream) {
  return apply(A, false, X, ldx, xdt, Y, ldy, ydt, ncols, stream);
}

fm_status fm_backward(fm_op A, const void* Y, int64_t ldy, fm_dtype ydt, void* X, int64_t ldx, fm_dtype xdt,
                      int64_t ncols, void* stream) {
  return apply(A, true, Y, ldy, ydt, X, ldx, xdt, ncols, stream);
}

fm_status fm_reserve(fm_op A, int64_t ncols, fm_dtype xdt, void* stream) {
  clear_error();
  if (!A || ncols < 0 || !dtype_valid(xdt)) { set_error("bad argument"); return FM_ERR_INVALID_ARG; }
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  size_t need = 0;
  for (int adj = 0; adj < 2; ++adj) {
    fm_dtype od;
    FM_TRY(natural_out_dtype(A, xdt, &od));
    Ctx ctx;
    ctx.st = (cudaStream_t)stream;
    ctx.dry = true;
    FM_TRY(device_tables(dev, &ctx.tabs));
    View in, out;
    in.dt = xdt;
    in.n = adj ? A->rows : A->cols;
    in.ld = in.ostride = in.n;
    out.dt = od;
    out.n = adj ? A->cols : A->rows;
    out.ld = out.ostride = out.n;
    FM_TRY(exec(A, adj != 0, in, out, ncols, 0, ctx));
    need = std::max(need, ctx.peak);
  }
  std::lock_guard<std::mutex> lk(A->ws.mu);
  if (need > A->ws.bytes) {
    if (A->ws.ptr) {
      FM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
      cudaFree(A->ws.ptr);
      A->ws.ptr = nullptr;
      A->ws.bytes = 0;
    }
    FM_CUDA(cudaMalloc(&A->ws.ptr, need));
    A->ws.bytes = need;
  }
  return FM_OK;
}

void fm_release(fm_op A) { op_release(A); }

const char* fm_status_string(fm_status s) {
  switch (s) {
    case FM_OK: return "ok";
    case FM_ERR_INVALID_ARG: return "invalid argument";
    case FM_ERR_SHAPE: return "shape mismatch";
    case FM_ERR_DTYPE: return "dtype not supported";
    case FM_ERR_UNSUPPORTED: return "unsupported";
    case FM_ERR_ALIAS: return "output aliases input";
    case FM_ERR_OOM: return "out of device memory";
    case FM_ERR_CUDA: return "CUDA error";
    case FM_ERR_TIMEOUT: return "device wait timed out";
    case FM_ERR_NUMERIC: return "non-finite value";
  }
  return "unknown status";
}

const char* fm_last_error(void) { return t_err.c_str(); }
uint64_t fm_launch_count(void) { return g_launches.load(); }
const char* fm_version(void) { return "fastmat-gb300 0.1"; }

}  // extern "C"
