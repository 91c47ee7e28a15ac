// Orthogonal matching pursuit on any operator of the library.
//
// OMP is the greedy sparse-recovery loop Sec. 3 cites beside (F)ISTA, and Sec. 4 names the
// rank-1 update form.  Like FISTA it touches the operator only through phi (A x) and
// beta (A^H y): each step takes the correlations c = A^H r (fm_backward), picks
// j = argmax |c_i| (lowest index on ties), fetches the column a_j = A e_j (fm_forward), and
// extends a thin QR factorisation A_S = Q R by one column (classical Gram-Schmidt applied
// twice, which keeps Q orthonormal in floating point); the residual is then
// r <- r - q_k (q_k^H r).  After K steps x_S solves R x_S = Q^H b.  All reductions are
// per-block partial sums added in a fixed order, so a solve is reproducible bit for bit.
#include <algorithm>
#include <cmath>

#include "exec.h"
#include "fm_device.cuh"

namespace fm {
namespace {

constexpr int kOmpThreads = 256;

template <typename T>
__device__ __forceinline__ T cabs2(typename Cx<T>::t z) {
  return z.x * z.x + z.y * z.y;
}

// dst = complex(src): real or complex source of the same precision
template <typename T>
__global__ void omp_to_complex(const void* src, int cplx, typename Cx<T>::t* a, typename Cx<T>::t* b, int64_t m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const typename Cx<T>::t v = cplx ? reinterpret_cast<const typename Cx<T>::t*>(src)[t]
                                     : cmake(reinterpret_cast<const T*>(src)[t], (T)0);
    a[t] = v;
    b[t] = v;
  }
}

// per block: the largest |c_i|^2 of its chunk and its lowest index
template <typename T>
__global__ void omp_argmax_partial(const typename Cx<T>::t* c, int64_t n, int64_t chunk, T* pv, int64_t* pi) {
  __shared__ T sv[kOmpThreads];
  __shared__ int64_t si[kOmpThreads];
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = std::min<int64_t>(n, lo + chunk);
  T bv = (T)-1;
  int64_t bi = -1;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const T v = cabs2<T>(c[i]);
    if (v > bv) { bv = v; bi = i; }    // increasing i per thread: ties keep the lower index
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const T v = sv[threadIdx.x + s];
      const int64_t i = si[threadIdx.x + s];
      if (i >= 0 && (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && (si[threadIdx.x] < 0 || i < si[threadIdx.x])))) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

// the pick j from the partials, in block order; records it and moves the unit vector to e_j
template <typename T>
__global__ void omp_argmax_final(const T* pv, const int64_t* pi, int nblk, int k, int32_t* S,
                                 typename Cx<T>::t* e) {
  if (threadIdx.x != 0) return;
  T bv = (T)-1;
  int64_t bi = 0;
  for (int b = 0; b < nblk; ++b)
    if (pi[b] >= 0 && pv[b] > bv) { bv = pv[b]; bi = pi[b]; }
  if (k > 0) e[S[k - 1]] = cmake((T)0, (T)0);
  S[k] = (int32_t)bi;
  e[bi] = cmake((T)1, (T)0);
}

// part[i * nblk + blk] = sum over the block's chunk of conj(V_i[t]) w[t], i < nv (V rows of
// stride ldv); with V == nullptr the sum of |w[t]|^2
template <typename T>
__global__ void omp_dots_partial(const typename Cx<T>::t* V, int64_t ldv, const typename Cx<T>::t* w, int64_t m,
                                 int64_t chunk, typename Cx<T>::t* part, int nblk) {
  typedef typename Cx<T>::t C;
  __shared__ C red[kOmpThreads];
  const int i = blockIdx.y;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = std::min<int64_t>(m, lo + chunk);
  C acc = cmake((T)0, (T)0);
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    const C wv = w[t];
    if (V) acc = cadd(acc, cmul(cconj(V[i * ldv + t]), wv));
    else acc.x += cabs2<T>(wv);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)i * nblk + blockIdx.x] = red[0];
}

enum { FIN_PROJ = 0, FIN_NORM = 1, FIN_STEP = 2, FIN_RHS = 3 };

// sums of the partials in block order, one thread per vector i:
//   FIN_PROJ  h[i] = sum; R[i, k] += sum        FIN_NORM  R[k, k] = sqrt(sum)
//   FIN_STEP  h[0] = sum (q_k^H r)              FIN_RHS   h[i] = sum (z = Q^H b)
template <typename T>
__global__ void omp_dots_final(const typename Cx<T>::t* part, int nblk, int nv, int mode, int k, int K,
                               typename Cx<T>::t* h, typename Cx<T>::t* R) {
  typedef typename Cx<T>::t C;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    C s = cmake((T)0, (T)0);
    for (int b = 0; b < nblk; ++b) s = cadd(s, part[(int64_t)i * nblk + b]);
    if (mode == FIN_PROJ) {
      h[i] = s;
      R[(int64_t)i * K + k] = cadd(R[(int64_t)i * K + k], s);
    } else if (mode == FIN_NORM) {
      R[(int64_t)k * K + k] = cmake(sqrt(s.x), (T)0);
    } else {
      h[i] = s;
    }
  }
}

// w[t] -= sum_{i < nv} Q_i[t] h[i]
template <typename T>
__global__ void omp_subtract(const typename Cx<T>::t* Q, int64_t ldq, int nv, const typename Cx<T>::t* h,
                             typename Cx<T>::t* w, int64_t m) {
  typedef typename Cx<T>::t C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    C v = w[t];
    for (int i = 0; i < nv; ++i) v = csub(v, cmul(Q[i * ldq + t], h[i]));
    w[t] = v;
  }
}

// q_k = w / R[k, k]
template <typename T>
__global__ void omp_normalize(const typename Cx<T>::t* w, const typename Cx<T>::t* R, int k, int K,
                              typename Cx<T>::t* q, int64_t m) {
  const T inv = (T)1 / R[(int64_t)k * K + k].x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    q[t] = cscale(w[t], inv);
}

// back substitution R x_S = z (one thread) and the scatter x[S[i]] = x_S[i] into the zeroed x
template <typename T>
__global__ void omp_solve(const typename Cx<T>::t* R, const typename Cx<T>::t* z, const int32_t* S, int K,
                          typename Cx<T>::t* xs, void* x, int cplx) {
  typedef typename Cx<T>::t C;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = K - 1; i >= 0; --i) {
    C s = z[i];
    for (int j = i + 1; j < K; ++j) s = csub(s, cmul(R[(int64_t)i * K + j], xs[j]));
    const T d = R[(int64_t)i * K + i].x;
    xs[i] = d != (T)0 ? cscale(s, (T)1 / d) : cmake((T)0, (T)0);
  }
  for (int i = 0; i < K; ++i) {
    if (cplx) reinterpret_cast<C*>(x)[S[i]] = xs[i];
    else reinterpret_cast<T*>(x)[S[i]] = xs[i].x;
  }
}

unsigned blocks_for(int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 1024)); }

template <typename T>
fm_status omp_run(fm_op A, const void* b, fm_dtype dt, int K, void* x, int32_t* support, cudaStream_t st) {
  typedef typename Cx<T>::t C;
  const int64_t m = A->rows, n = A->cols;
  const fm_dtype cdt = sizeof(T) == 4 ? FM_C64 : FM_C128;
  const int cplx = is_complex(dt) ? 1 : 0;
  const int64_t chunk_m = std::max<int64_t>(1024, (m + 255) / 256), chunk_n = std::max<int64_t>(1024, (n + 255) / 256);
  const int nb_m = (int)((m + chunk_m - 1) / chunk_m), nb_n = (int)((n + chunk_n - 1) / chunk_n);
  // workspace: r, bc, w (m each), c, e (n each), Q (K m), R (K K), h (K), z (K), xs (K),
  // partials (K nb_m), argmax partials (nb_n values + indices), support (K)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_r = take(m * sizeof(C)), o_b = take(m * sizeof(C)), o_w = take(m * sizeof(C));
  const size_t o_c = take(n * sizeof(C)), o_e = take(n * sizeof(C));
  const size_t o_Q = take((size_t)K * m * sizeof(C)), o_R = take((size_t)K * K * sizeof(C));
  const size_t o_h = take(K * sizeof(C)), o_z = take(K * sizeof(C)), o_xs = take(K * sizeof(C));
  const size_t o_p = take((size_t)K * std::max(nb_m, 1) * sizeof(C));
  const size_t o_pv = take(nb_n * sizeof(T)), o_pi = take(nb_n * sizeof(int64_t)), o_S = take(K * sizeof(int32_t));
  char* ws = nullptr;
  FM_CUDA(cudaMalloc(&ws, off));
  C* r = (C*)(ws + o_r);
  C* bc = (C*)(ws + o_b);
  C* w = (C*)(ws + o_w);
  C* c = (C*)(ws + o_c);
  C* e = (C*)(ws + o_e);
  C* Q = (C*)(ws + o_Q);
  C* R = (C*)(ws + o_R);
  C* h = (C*)(ws + o_h);
  C* z = (C*)(ws + o_z);
  C* xs = (C*)(ws + o_xs);
  C* part = (C*)(ws + o_p);
  T* pv = (T*)(ws + o_pv);
  int64_t* pi = (int64_t*)(ws + o_pi);
  int32_t* S = (int32_t*)(ws + o_S);
  fm_status s = FM_OK;
  auto go = [&](const char* what) {
    if (s == FM_OK) s = after_launch(what);
  };
  cudaError_t err = cudaMemsetAsync(e, 0, n * sizeof(C), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(R, 0, (size_t)K * K * sizeof(C), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(x, 0, n * (cplx ? sizeof(C) : sizeof(T)), st);
  if (err != cudaSuccess) {
    set_error("fm_omp: %s", cudaGetErrorString(err));
    s = FM_ERR_CUDA;
  }
  if (s == FM_OK) {
    omp_to_complex<T><<<blocks_for(m), 256, 0, st>>>(b, cplx, r, bc, m);
    go("omp_to_complex");
  }
  for (int k = 0; k < K && s == FM_OK; ++k) {
    // correlations and the pick
    s = fm_backward(A, r, m, cdt, c, n, cdt, 1, st);
    if (s != FM_OK) break;
    omp_argmax_partial<T><<<nb_n, kOmpThreads, 0, st>>>(c, n, chunk_n, pv, pi);
    go("omp_argmax_partial");
    if (s == FM_OK) {
      omp_argmax_final<T><<<1, 32, 0, st>>>(pv, pi, nb_n, k, S, e);
      go("omp_argmax_final");
    }
    // the new column and its orthogonalisation against q_0 .. q_{k-1} (twice)
    if (s == FM_OK) s = fm_forward(A, e, n, cdt, w, m, cdt, 1, st);
    for (int pass = 0; pass < 2 && k > 0 && s == FM_OK; ++pass) {
      omp_dots_partial<T><<<dim3(nb_m, k), kOmpThreads, 0, st>>>(Q, m, w, m, chunk_m, part, nb_m);
      go("omp_dots_partial");
      if (s == FM_OK) {
        omp_dots_final<T><<<1, 256, 0, st>>>(part, nb_m, k, FIN_PROJ, k, K, h, R);
        go("omp_dots_final");
      }
      if (s == FM_OK) {
        omp_subtract<T><<<blocks_for(m), 256, 0, st>>>(Q, m, k, h, w, m);
        go("omp_subtract");
      }
    }
    if (s != FM_OK) break;
    omp_dots_partial<T><<<dim3(nb_m, 1), kOmpThreads, 0, st>>>(nullptr, 0, w, m, chunk_m, part, nb_m);
    go("omp_dots_partial");
    if (s == FM_OK) {
      omp_dots_final<T><<<1, 32, 0, st>>>(part, nb_m, 1, FIN_NORM, k, K, h, R);
      go("omp_dots_final");
    }
    if (s == FM_OK) {
      omp_normalize<T><<<blocks_for(m), 256, 0, st>>>(w, R, k, K, Q + (int64_t)k * m, m);
      go("omp_normalize");
    }
    // r <- r - q_k (q_k^H r)
    if (s == FM_OK) {
      omp_dots_partial<T><<<dim3(nb_m, 1), kOmpThreads, 0, st>>>(Q + (int64_t)k * m, m, r, m, chunk_m, part, nb_m);
      go("omp_dots_partial");
    }
    if (s == FM_OK) {
      omp_dots_final<T><<<1, 32, 0, st>>>(part, nb_m, 1, FIN_STEP, k, K, h, R);
      go("omp_dots_final");
    }
    if (s == FM_OK) {
      omp_subtract<T><<<blocks_for(m), 256, 0, st>>>(Q + (int64_t)k * m, m, 1, h, r, m);
      go("omp_subtract");
    }
  }
  // x_S from R x_S = Q^H b
  if (s == FM_OK) {
    omp_dots_partial<T><<<dim3(nb_m, K), kOmpThreads, 0, st>>>(Q, m, bc, m, chunk_m, part, nb_m);
    go("omp_dots_partial");
  }
  if (s == FM_OK) {
    omp_dots_final<T><<<1, 256, 0, st>>>(part, nb_m, K, FIN_RHS, 0, K, z, R);
    go("omp_dots_final");
  }
  if (s == FM_OK) {
    omp_solve<T><<<1, 32, 0, st>>>(R, z, S, K, xs, x, cplx);
    go("omp_solve");
  }
  if (s == FM_OK && support) {
    err = cudaMemcpyAsync(support, S, K * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (err != cudaSuccess) {
      set_error("fm_omp: %s", cudaGetErrorString(err));
      s = FM_ERR_CUDA;
    }
  }
  err = cudaStreamSynchronize(st);
  if (s == FM_OK && err != cudaSuccess) {
    set_error("fm_omp: %s", cudaGetErrorString(err));
    s = FM_ERR_CUDA;
  }
  cudaFree(ws);
  return s;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" fm_status fm_omp(fm_op A, const void* b, fm_dtype dt, int32_t K, void* x, int32_t* support, void* stream) {
  clear_error();
  if (!A || !b || !x) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if (K < 1 || K > A->cols || K > A->rows || K > 4096) {
    set_error("fm_omp: K must be in [1, min(rows, cols, 4096)]");
    return FM_ERR_INVALID_ARG;
  }
  if (dt != FM_C64 && dt != FM_C128 && dt != FM_F32 && dt != FM_F64) { set_error("fm_omp dtype"); return FM_ERR_DTYPE; }
  if (!is_complex(dt) && !A->real) { set_error("fm_omp: a complex operator needs complex b and x"); return FM_ERR_DTYPE; }
  fm_dtype od;
  FM_TRY(natural_out_dtype(A, complex_of(dt), &od));
  if (od != complex_of(dt)) { set_error("fm_omp: the operator does not map complex columns to complex columns"); return FM_ERR_DTYPE; }
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  if (dev != A->device) { set_error("operator lives on device %d, current is %d", A->device, dev); return FM_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  return is_double(dt) ? omp_run<double>(A, b, dt, K, x, support, st) : omp_run<float>(A, b, dt, K, x, support, st);
}
