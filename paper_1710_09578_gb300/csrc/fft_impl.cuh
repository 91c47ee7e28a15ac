// Batched Stockham FFT engine for the Fourier, Circulant and Toeplitz operators.
//
// One CTA owns a tile of V vectors of length L (L * V = THREADS * EPT elements) in
// shared memory and runs radix-8/4/2 Stockham passes over it: each thread keeps EPT
// elements in registers, multiplies by the twiddles of the pass, does the small DFT in
// registers and writes the results to their auto-sorted place, so no bit reversal is
// ever needed (the DFT of Eq. (1), evaluated by the butterfly factorisation the paper
// mentions in Sec. 1).  For a circulant or Toeplitz operator the forward transform, the
// multiplication by the precomputed spectrum (Eq. (5); Sec. 2.1.1) and the inverse
// transform all run in the same CTA: the last forward pass and the first inverse pass
// touch the same elements, so the spectrum product happens in registers.
//
// Vectors are read through a general strided view so that one kernel serves plain
// column blocks, mode products of Kron (the transform runs along one axis of the column
// seen as [outer][L][inner]) and the two-pass plan for long transforms.  Diag and row
// selection (P, P^H) neighbours of a Product, zero-padding and truncation for the
// Toeplitz embedding, twiddles of the two-pass plan, scaling and accumulation (for Sum)
// are fused into the loads and stores.
#pragma once
#include "fft.h"
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {

// Per-vector addressing, computed once per tile into shared memory.
struct VecInfo {
  int64_t in_off;   // element offset of t = 0 (column 2c in IO_RP mode); -1: vector absent
  int64_t out_off;
  int32_t in_n2;    // ((o*inner + i) / in_fdiv) % in_fmod
  int32_t out_n2;
  int32_t tw_n2;    // ((o*inner + i) / tw_div) % tw_mod
  int32_t flags;    // bit 0: second real column of a pair exists
  int64_t soff;     // spectrum row offset
};

template <typename C>
__host__ __device__ constexpr size_t fft_vinfo_offset(int E) {
  return (((size_t)(E + E / 16 + 1) * sizeof(C)) + 15) & ~(size_t)15;
}

template <typename T>
__device__ __forceinline__ typename Cx<T>::t fft_load(const FftArgs<T>& a, const VecInfo& vi, int t) {
  typedef typename Cx<T>::t C;
  if (vi.in_off < 0) return cmake((T)0, (T)0);
  const int64_t n = (int64_t)t * a.in_fmul + vi.in_n2;
  if (n >= a.Lin) return cmake((T)0, (T)0);
  int64_t src = n;
  if (a.pre_map) {
    src = a.pre_map[n];
    if (src < 0) return cmake((T)0, (T)0);
  }
  const int64_t off = vi.in_off + src * a.in_tstride;
  C x;
  if (a.in_mode == IO_C) {
    x = reinterpret_cast<const C*>(a.in)[off];
  } else {
    const T* p = reinterpret_cast<const T*>(a.in);
    T re = p[off];
    T im = (a.in_mode == IO_RP && (vi.flags & 1)) ? p[off + a.in_ld] : (T)0;
    x = cmake(re, im);
  }
  if (a.pre_dc) {
    C d = a.pre_dc[n];
    x = cmul(x, a.pre_conj ? cconj(d) : d);
  } else if (a.pre_dr) {
    x = cscale(x, a.pre_dr[n]);
  }
  return x;
}

template <typename T>
__device__ __forceinline__ void fft_store(const FftArgs<T>& a, const VecInfo& vi, int t, typename Cx<T>::t x) {
  typedef typename Cx<T>::t C;
  if (vi.out_off < 0) return;
  const int64_t n = (int64_t)t * a.out_fmul + vi.out_n2;
  if (n >= a.Lout) return;
  if (a.post_dc) {
    C d = a.post_dc[n];
    x = cmul(x, a.post_conj ? cconj(d) : d);
  } else if (a.post_dr) {
    x = cscale(x, a.post_dr[n]);
  }
  x = cscale(x, a.scale);
  int64_t dst = n;
  if (a.post_map) {
    dst = a.post_map[n];
    if (dst < 0) return;
  }
  const int64_t off = vi.out_off + dst * a.out_tstride;
  if (a.out_mode == IO_C) {
    C* p = reinterpret_cast<C*>(a.out) + off;
    if (a.beta) x = cadd(x, *p);
    *p = x;
  } else {
    T* p = reinterpret_cast<T*>(a.out) + off;
    *p = a.beta ? x.x + *p : x.x;
    if (a.out_mode == IO_RP && (vi.flags & 1)) {
      p += a.out_ld;
      *p = a.beta ? x.y + *p : x.y;
    }
  }
}

template <int R> struct LogR { static constexpr int v = R == 8 ? 3 : (R == 4 ? 2 : 1); };

// Butterfly b = tid + q*THREADS of a radix-R pass covers vector v and index j in [0, L/R);
// its R inputs are t = j + k L/R.
__device__ __forceinline__ void bfly_coords(int b, int logV, int logLR, int vfast, int& j, int& v) {
  if (vfast) {
    v = b & ((1 << logV) - 1);
    j = b >> logV;
  } else {
    j = b & ((1 << logLR) - 1);
    v = b >> logLR;
  }
}

__device__ __forceinline__ int lin_index(int t, int v, int logL, int logV, int vfast) {
  return vfast ? ((t << logV) + v) : ((v << logL) + t);
}

// Load the R inputs t = j + k L/R of each of this thread's butterflies.
template <int R, int THREADS, int EPT, typename C>
__device__ __forceinline__ void regs_from_smem(C (&r)[EPT], const C* s, int logL, int logV, int vfast) {
  const int logLR = logL - LogR<R>::v;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly_coords(threadIdx.x + q * THREADS, logV, logLR, vfast, j, v);
#pragma unroll
    for (int k = 0; k < R; ++k) r[q * R + k] = s[spad(lin_index(j + (k << logLR), v, logL, logV, vfast))];
  }
}

// Store the outputs of a radix-R pass to their Stockham positions (j/Ns) Ns R + j%Ns + k Ns.
// For the last pass (Ns R = L) these are the natural positions j + k L/R.
template <int R, int THREADS, int EPT, typename C>
__device__ __forceinline__ void regs_to_smem(const C (&r)[EPT], C* s, int logL, int logV, int vfast, int logNs) {
  const int logR = LogR<R>::v;
  const int logLR = logL - logR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly_coords(threadIdx.x + q * THREADS, logV, logLR, vfast, j, v);
    const int jm = j & ((1 << logNs) - 1);
    const int base = ((j >> logNs) << (logNs + logR)) + jm;
#pragma unroll
    for (int k = 0; k < R; ++k) s[spad(lin_index(base + (k << logNs), v, logL, logV, vfast))] = r[q * R + k];
  }
}

// Twiddle W_{Ns R}^{dir k jm} then DFT_R, for each butterfly of this thread.
template <int R, int THREADS, int EPT, typename C>
__device__ __forceinline__ void pass_compute(C (&r)[EPT], int logL, int logV, int vfast, int logNs, int dir,
                                             const C* __restrict__ tw) {
  const int logR = LogR<R>::v;
  const int logLR = logL - logR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly_coords(threadIdx.x + q * THREADS, logV, logLR, vfast, j, v);
    if (logNs > 0) {
      const int jm = j & ((1 << logNs) - 1);
      C w = tw[jm << (kTwLog - logNs - logR)];
      if (dir > 0) w = cconj(w);
      C wk = w;
#pragma unroll
      for (int k = 1; k < R; ++k) {
        r[q * R + k] = cmul(r[q * R + k], wk);
        if (k + 1 < R) wk = cmul(wk, w);
      }
    }
    if (R == 8) dft8(&r[q * R], dir);
    else if (R == 4) dft4(&r[q * R], dir);
    else dft2(&r[q * R]);
  }
}

// Spectrum product at the natural positions t = j + k L/R of the last forward pass.
template <int R, int THREADS, int EPT, typename C>
__device__ __forceinline__ void spec_mul(C (&r)[EPT], const C* __restrict__ spec, int conj, const VecInfo* vinfo,
                                         int logL, int logV, int vfast) {
  const int logLR = logL - LogR<R>::v;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly_coords(threadIdx.x + q * THREADS, logV, logLR, vfast, j, v);
    const C* sp = spec + vinfo[v].soff + j;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      C w = sp[k << logLR];
      r[q * R + k] = cmul(r[q * R + k], conj ? cconj(w) : w);
    }
  }
}

#define FM_RADIX_SWITCH(R, CALL) \
  switch (R) {                   \
    case 8: { CALL(8); } break;  \
    case 4: { CALL(4); } break;  \
    default: { CALL(2); } break; \
  }

template <typename T>
int fft_max_tile() { return sizeof(T) == 4 ? 16384 : 8192; }

}  // namespace fm
