// Pointwise and gather/scatter kernels: Diag (Eq. (7)), the row selection P and its
// adjoint (zero-fill + scatter), and dtype promotion / accumulation between stages.
// They run only when no neighbouring transform can absorb them into its loads/stores.
#include "fm_device.cuh"
#include "fm_internal.h"
#include "pointwise.h"

namespace fm {

template <typename T>
__global__ void pointwise_kernel(const __grid_constant__ PwArgs a) {
  typedef typename Cx<T>::t C;
  const int64_t total = a.ncols * a.outer * a.n_out * a.inner;
  pdl_launch_dependents();
  pdl_wait();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % a.inner;
    const int64_t r = e / a.inner;
    const int64_t t = r % a.n_out;
    const int64_t r2 = r / a.n_out;
    const int64_t o = r2 % a.outer;
    const int64_t c = r2 / a.outer;
    const int64_t src = a.map ? (int64_t)a.map[t] : t;
    C x = cmake((T)0, (T)0);
    if (src >= 0) {
      const int64_t off = c * a.in_ld + o * a.in_ostride + src * a.inner + i;
      if (a.in_cplx) x = reinterpret_cast<const C*>(a.in)[off];
      else x = cmake(reinterpret_cast<const T*>(a.in)[off], (T)0);
      if (a.dc) {
        C d = reinterpret_cast<const C*>(a.dc)[src];
        x = cmul(x, a.d_conj ? cconj(d) : d);
      } else if (a.dr) {
        x = cscale(x, reinterpret_cast<const T*>(a.dr)[src]);
      }
      x = cscale(x, (T)a.scale);
    }
    const int64_t off = c * a.out_ld + o * a.out_ostride + t * a.inner + i;
    if (a.out_cplx) {
      C* p = reinterpret_cast<C*>(a.out) + off;
      *p = a.beta ? cadd(*p, x) : x;
    } else {
      T* p = reinterpret_cast<T*>(a.out) + off;
      *p = a.beta ? *p + x.x : x.x;
    }
  }
}

template <typename T>
static fm_status pw_go(const PwArgs& a, cudaStream_t st) {
  const int64_t total = a.ncols * a.outer * a.n_out * a.inner;
  if (total == 0) return FM_OK;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  return pdl_go("pointwise_kernel", pointwise_kernel<T>, dim3((unsigned)blocks), dim3(256), 0, st, a);
}

fm_status pointwise_launch(const PwArgs& a, bool dbl, cudaStream_t st) {
  return dbl ? pw_go<double>(a, st) : pw_go<float>(a, st);
}

// int32 accumulation / copy for the exact Hadamard path.
__global__ void i32_copy_kernel(const int* in, int64_t in_ld, int* out, int64_t out_ld, int64_t n,
                                int64_t ncols, int beta) {
  const int64_t total = n * ncols;
  pdl_launch_dependents();
  pdl_wait();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, t = e % n;
    const int v = in[c * in_ld + t];
    int* p = out + c * out_ld + t;
    *p = beta ? *p + v : v;
  }
}

fm_status i32_copy_launch(const int* in, int64_t in_ld, int* out, int64_t out_ld, int64_t n, int64_t ncols,
                          int beta, cudaStream_t st) {
  const int64_t total = n * ncols;
  if (total == 0) return FM_OK;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  return pdl_go("i32_copy_kernel", i32_copy_kernel, dim3((unsigned)blocks), dim3(256), 0, st, in, in_ld, out, out_ld,
                n, ncols, beta);
}

// W_N^m = exp(-2 pi i m / N) for m in [0, N), computed in FP64 with sincospi.
__global__ void twiddle_kernel(int64_t N, float2* t32, double2* t64) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < N; m += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    if (t64) t64[m] = make_double2(c, s);
    if (t32) t32[m] = make_float2((float)c, (float)s);
  }
}

// Entry q of the pass-twiddle tables (layout in fm_device.cuh), from sincospi in FP64.
__global__ void pass_twiddle_kernel(float2* t32, double2* t64) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kPassTwEntries;
       q += (int64_t)gridDim.x * blockDim.x) {
    int s = 1, lr = 1;
    while (q >= pass_tw_offset(s, lr) + ((int64_t)1 << s)) {
      if (lr < (s < 4 ? s : 4)) ++lr;
      else { ++s; lr = 1; }
    }
    const int64_t r = q - pass_tw_offset(s, lr);
    const int64_t i = r >> lr, k = r & ((1 << lr) - 1);
    const int64_t e = (i * k) & (((int64_t)1 << s) - 1);
    double sn, cs;
    sincospi(-2.0 * (double)e / (double)((int64_t)1 << s), &sn, &cs);
    t64[q] = make_double2(cs, sn);
    t32[q] = make_float2((float)cs, (float)sn);
  }
}

fm_status pass_twiddle_launch(float2* t32, double2* t64, cudaStream_t st) {
  pass_twiddle_kernel<<<256, 256, 0, st>>>(t32, t64);
  return after_launch("pass_twiddle_kernel");
}

fm_status twiddle_launch(int64_t N, float2* t32, double2* t64, cudaStream_t st) {
  int64_t blocks = (N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  twiddle_kernel<<<(unsigned)blocks, 256, 0, st>>>(N, t32, t64);
  return after_launch("twiddle_kernel");
}

// Spectrum post-processing at construction: s64 <- s64 * scale, s32 <- (float)s64, and
// the row-permuted copies perm[k1*N2 + k2] = s[k1 + N1*k2] for the two-pass plan.
__global__ void spectrum_finish_kernel(double2* s64, float2* s32, double2* p64, float2* p32, int64_t L, int64_t N1,
                                       int64_t N2, double scale) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = s64[k];
    v.x *= scale;
    v.y *= scale;
    s64[k] = v;
    s32[k] = make_float2((float)v.x, (float)v.y);
    if (p64) {
      const int64_t k1 = k % N1, k2 = k / N1;
      p64[k1 * N2 + k2] = v;
      p32[k1 * N2 + k2] = make_float2((float)v.x, (float)v.y);
    }
  }
}

fm_status spectrum_finish_launch(double2* s64, float2* s32, double2* p64, float2* p32, int64_t L, int64_t N1,
                                 int64_t N2, double scale, cudaStream_t st) {
  int64_t blocks = (L + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  spectrum_finish_kernel<<<(unsigned)blocks, 256, 0, st>>>(s64, s32, p64, p32, L, N1, N2, scale);
  return after_launch("spectrum_finish_kernel");
}

// Parameter conversion at construction: any of f32/f64/c64/c128 -> c128 (and f64 if real).
__global__ void to_c128_kernel(const void* src, int dt, int64_t n, int64_t dst_len, double2* dst) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dst_len; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (k < n) {
      switch (dt) {
        case FM_F32: v.x = reinterpret_cast<const float*>(src)[k]; break;
        case FM_F64: v.x = reinterpret_cast<const double*>(src)[k]; break;
        case FM_C64: {
          float2 f = reinterpret_cast<const float2*>(src)[k];
          v = make_double2(f.x, f.y);
        } break;
        default: v = reinterpret_cast<const double2*>(src)[k]; break;
      }
    }
    dst[k] = v;
  }
}

fm_status to_c128_launch(const void* src, fm_dtype dt, int64_t n, int64_t dst_len, double2* dst, cudaStream_t st) {
  int64_t blocks = (dst_len + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  to_c128_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, (int)dt, n, dst_len, dst);
  return after_launch("to_c128_kernel");
}

// Circulant embedding column of a Toeplitz operator (Sec. 2.1.1):
// c[k] = t[k] for k < rows, c[L - j] = t[rows - 1 + j] for j in [1, cols), 0 elsewhere.
__global__ void toeplitz_embed_kernel(const double2* t, int64_t rows, int64_t cols, int64_t L, double2* c) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (k < rows) v = t[k];
    else if (k > L - cols) v = t[rows - 1 + (L - k)];
    c[k] = v;
  }
}

fm_status toeplitz_embed_launch(const double2* t, int64_t rows, int64_t cols, int64_t L, double2* c,
                                cudaStream_t st) {
  int64_t blocks = (L + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  toeplitz_embed_kernel<<<(unsigned)blocks, 256, 0, st>>>(t, rows, cols, L, c);
  return after_launch("toeplitz_embed_kernel");
}

// Complex diagonal in both precisions from the c128 copy (plus real parts when real).
__global__ void diag_finish_kernel(const double2* d, int64_t n, float2* d32, double* dr64, float* dr32) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = d[k];
    d32[k] = make_float2((float)v.x, (float)v.y);
    if (dr64) dr64[k] = v.x;
    if (dr32) dr32[k] = (float)v.x;
  }
}

fm_status diag_finish_launch(const double2* d, int64_t n, float2* d32, double* dr64, float* dr32, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  diag_finish_kernel<<<(unsigned)blocks, 256, 0, st>>>(d, n, d32, dr64, dr32);
  return after_launch("diag_finish_kernel");
}

// max_k |s_k|^2 of a spectrum (one CTA, FP64): the FISTA step cap.
__global__ void spec_cap_kernel(const double2* s, int64_t L, double scale, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < L; k += blockDim.x) {
    double2 v = s[k];
    m = fmax(m, (v.x * v.x + v.y * v.y) * scale);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

fm_status spec_cap_launch(const double2* s, int64_t L, double scale, double* out, cudaStream_t st) {
  spec_cap_kernel<<<1, 256, 0, st>>>(s, L, scale, out);
  return after_launch("spec_cap_kernel");
}

}  // namespace fm
