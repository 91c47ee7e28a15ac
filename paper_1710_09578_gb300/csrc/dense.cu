// Dense execution of small operators and the calibration that chooses it, plus the circulant
// of an LFSR sequence.
//
// Sec. 2.1.3: below some problem size a plain matrix-vector product beats the fast transform,
// and fastmat's calibration times both to find where.  Here a leaf (Fourier, Circulant,
// Toeplitz, Hadamard) with at most 4096 matrix entries can be switched to a dense product:
// its matrix is materialised once, column by column, as the forward transform of the unit
// vectors, and y = M x (M^H y for the adjoint) runs from shared memory.  fm_calibrate_dense
// times forward + adjoint both ways on probe columns and keeps the faster.
#include <algorithm>
#include <vector>

#include "exec.h"
#include "fm_device.cuh"

namespace fm {
namespace {

constexpr int64_t kDenseMaxEntries = 4096;

// y[c][i] = sum_j M[j * rows + i] x[c][j]   (adj: y[c][j] = sum_i conj(M[j * rows + i]) x[c][i])
// for a tile of columns per CTA: M and the tile's input columns in shared memory.
template <typename T>
__global__ void dense_kernel(const typename Cx<T>::t* M, int64_t rows, int64_t cols, int adj,
                             const typename Cx<T>::t* x, int64_t ldx, typename Cx<T>::t* y, int64_t ldy,
                             int64_t ncols, int cpb, int beta) {
  typedef typename Cx<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sM = reinterpret_cast<C*>(smem_raw);
  const int nin = (int)(adj ? rows : cols), nout = (int)(adj ? cols : rows);
  C* sx = sM + rows * cols;
  pdl_launch_dependents();
  pdl_wait();
  for (int q = threadIdx.x; q < rows * cols; q += blockDim.x) sM[q] = gld(M + q);
  const int64_t c0 = (int64_t)blockIdx.x * cpb;
  for (int q = threadIdx.x; q < cpb * nin; q += blockDim.x) {
    const int64_t c = c0 + q / nin;
    sx[q] = c < ncols ? gld(x + c * ldx + q % nin) : cmake((T)0, (T)0);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < cpb * nout; q += blockDim.x) {
    const int64_t c = c0 + q / nout;
    if (c >= ncols) continue;
    const int o = q % nout;
    const C* xin = sx + (q / nout) * nin;
    C acc = cmake((T)0, (T)0);
    if (!adj) {
      for (int j = 0; j < nin; ++j) acc = cadd(acc, cmul(sM[j * rows + o], xin[j]));
    } else {
      for (int i = 0; i < nin; ++i) acc = cadd(acc, cmul(cconj(sM[o * rows + i]), xin[i]));
    }
    C* p = y + c * ldy + o;
    gst(p, beta ? cadd(gld(p), acc) : acc);
  }
}

__global__ void identity_kernel(double2* e, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x)
    e[q] = make_double2(q / n == q % n ? 1.0 : 0.0, 0.0);
}

__global__ void narrow_kernel(const double2* a, float2* b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = make_float2((float)a[q].x, (float)a[q].y);
}

__global__ void widen_kernel(const float2* a, double2* b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = make_double2(a[q].x, a[q].y);
}

bool dense_capable(const fm_op_s* A) {
  return (A->kind == K_FOURIER || A->kind == K_CIRCULANT || A->kind == K_TOEPLITZ || A->kind == K_HADAMARD) &&
         A->rows * A->cols <= kDenseMaxEntries;
}

// M (column-major) as the forward transform of the unit vectors, FP64 where the operator takes
// complex128 (Hadamard: complex64, its entries are exactly +-1), plus the other precision.
fm_status materialise(fm_op_s* A, cudaStream_t st) {
  const int64_t n = A->cols, m = A->rows, N = n * m;
  double2* I64 = nullptr;
  float2* I32 = nullptr;
  FM_CUDA(cudaMalloc(&A->m64, N * sizeof(double2)));
  FM_CUDA(cudaMalloc(&A->m32, N * sizeof(float2)));
  FM_CUDA(cudaMalloc(&I64, n * n * sizeof(double2)));
  fm_status s = FM_OK;
  identity_kernel<<<(unsigned)std::min<int64_t>((n * n + 255) / 256, 1024), 256, 0, st>>>(I64, n);
  s = after_launch("identity_kernel");
  const bool had = A->kind == K_HADAMARD;
  if (s == FM_OK && had) {
    cudaError_t e = cudaMalloc(&I32, n * n * sizeof(float2));
    if (e != cudaSuccess) { set_error("dense: %s", cudaGetErrorString(e)); s = FM_ERR_OOM; }
    if (s == FM_OK) {
      narrow_kernel<<<(unsigned)std::min<int64_t>((n * n + 255) / 256, 1024), 256, 0, st>>>(I64, I32, n * n);
      s = after_launch("narrow_kernel");
    }
  }
  if (s == FM_OK) {
    s = had ? fm_forward(A, I32, n, FM_C64, A->m32, m, FM_C64, n, st)
            : fm_forward(A, I64, n, FM_C128, A->m64, m, FM_C128, n, st);
  }
  if (s == FM_OK) {
    const unsigned g = (unsigned)std::min<int64_t>((N + 255) / 256, 1024);
    if (had) widen_kernel<<<g, 256, 0, st>>>(A->m32, A->m64, N);
    else narrow_kernel<<<g, 256, 0, st>>>(A->m64, A->m32, N);
    s = after_launch("dense_convert_kernel");
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (s == FM_OK && e != cudaSuccess) { set_error("dense: %s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
  cudaFree(I64);
  if (I32) cudaFree(I32);
  return s;
}

}  // namespace

fm_status dense_apply(const fm_op_s* A, bool adj, const void* in, int64_t ldi, void* out, int64_t ldo, int64_t ncols,
                      bool dbl, int beta, cudaStream_t st) {
  const int64_t nout = adj ? A->cols : A->rows;
  const int64_t nin = adj ? A->rows : A->cols;
  // columns per CTA: a thread per output, at most 4096 staged input entries
  const int cpb = (int)std::max<int64_t>(1, std::min<int64_t>(256 / nout, kDenseMaxEntries / nin));
  const size_t esz = dbl ? sizeof(double2) : sizeof(float2);
  const size_t smem = (size_t)(A->rows * A->cols + cpb * nin) * esz;
  const unsigned grid = (unsigned)((ncols + cpb - 1) / cpb);
  if (grid == 0) return FM_OK;
  if (dbl) {
    auto k = dense_kernel<double>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return pdl_go("dense_kernel<f64>", k, dim3(grid), dim3(256), smem, st, (const double2*)A->m64, A->rows,
                  A->cols, adj ? 1 : 0, (const double2*)in, ldi, (double2*)out, ldo, ncols, cpb, beta);
  }
  auto k = dense_kernel<float>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return pdl_go("dense_kernel<f32>", k, dim3(grid), dim3(256), smem, st, (const float2*)A->m32, A->rows, A->cols,
                adj ? 1 : 0, (const float2*)in, ldi, (float2*)out, ldo, ncols, cpb, beta);
}

}  // namespace fm

using namespace fm;

extern "C" fm_status fm_set_dense(fm_op A, int dense, void* stream) {
  clear_error();
  if (!A) { set_error("null operator"); return FM_ERR_INVALID_ARG; }
  if (!dense_capable(A)) {
    set_error("dense execution takes a Fourier, Circulant, Toeplitz or Hadamard operator of at most %lld entries",
              (long long)kDenseMaxEntries);
    return FM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(A->ws.mu);
  if (dense && !A->m32) {
    A->dense = 0;
    // fm_forward takes the workspace lock itself
    A->ws.mu.unlock();
    fm_status s = materialise(A, (cudaStream_t)stream);
    A->ws.mu.lock();
    if (s != FM_OK) {
      if (A->m32) cudaFree(A->m32);
      if (A->m64) cudaFree(A->m64);
      A->m32 = nullptr;
      A->m64 = nullptr;
      return s;
    }
  }
  A->dense = dense ? 1 : 0;
  return FM_OK;
}

extern "C" fm_status fm_calibrate_dense(fm_op A, int64_t ncols, fm_dtype dt, void* stream, float* ms_fast,
                                        float* ms_dense, int32_t* chosen) {
  clear_error();
  if (!A || ncols < 1) { set_error("bad argument"); return FM_ERR_INVALID_ARG; }
  if (dt != FM_C64 && dt != FM_C128) { set_error("calibrate on complex64 or complex128 probe columns"); return FM_ERR_DTYPE; }
  FM_TRY(fm_set_dense(A, 1, stream));
  FM_TRY(fm_set_dense(A, 0, stream));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t esz = dtype_size(dt);
  const int64_t n = std::max(A->rows, A->cols);
  void *x = nullptr, *y = nullptr, *z = nullptr;
  FM_CUDA(cudaMalloc(&x, ncols * n * esz));
  fm_status s = FM_OK;
  cudaError_t e = cudaMalloc(&y, ncols * n * esz);
  if (e == cudaSuccess) e = cudaMalloc(&z, ncols * n * esz);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, ncols * n * esz, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { set_error("calibrate_dense: %s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
  float t[2] = {0.f, 0.f};
  const int reps = 20;
  for (int mode = 0; mode < 2 && s == FM_OK; ++mode) {
    A->dense = mode;
    for (int r = 0; r < reps + 3 && s == FM_OK; ++r) {
      if (r == 3) cudaEventRecord(e0, st);
      s = fm_forward(A, x, A->cols, dt, y, A->rows, dt, ncols, st);
      if (s == FM_OK) s = fm_backward(A, y, A->rows, dt, z, A->cols, dt, ncols, st);
    }
    if (s == FM_OK) {
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t[mode], e0, e1);
      if (e != cudaSuccess) { set_error("calibrate_dense: %s", cudaGetErrorString(e)); s = FM_ERR_CUDA; }
      t[mode] /= reps;
    }
  }
  A->dense = (s == FM_OK && t[1] < t[0]) ? 1 : 0;
  if (ms_fast) *ms_fast = t[0];
  if (ms_dense) *ms_dense = t[1];
  if (chosen) *chosen = A->dense;
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  if (y) cudaFree(y);
  if (z) cudaFree(z);
  return s;
}

extern "C" fm_status fm_lfsr_circulant(int32_t nbits, uint64_t taps, uint64_t state, int64_t n, void* stream,
                                       fm_op* out) {
  clear_error();
  if (!out) { set_error("null output"); return FM_ERR_INVALID_ARG; }
  if (nbits < 1 || nbits > 63 || state == 0 || (state >> nbits) != 0 || (taps >> nbits) != 0) {
    set_error("lfsr: state must be a nonzero nbits-bit value and taps an nbits-bit mask (1 <= nbits <= 63)");
    return FM_ERR_INVALID_ARG;
  }
  if (n < 1 || n > (1LL << 24) || (n & (n - 1))) { set_error("lfsr circulant size: power of two up to 2^24"); return FM_ERR_UNSUPPORTED; }
  // the first n outputs of the register, +1 for bit 0 and -1 for bit 1
  std::vector<double> c((size_t)n);
  uint64_t s = state;
  for (int64_t k = 0; k < n; ++k) {
    c[(size_t)k] = (s & 1) ? -1.0 : 1.0;
    const uint64_t f = (uint64_t)__builtin_parityll(s & taps);
    s = (s >> 1) | (f << (nbits - 1));
  }
  return fm_circulant(c.data(), n, FM_F64, stream, out);
}
