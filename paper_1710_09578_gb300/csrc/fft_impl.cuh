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
    src = gld(a.pre_map + n);
    if (src < 0) return cmake((T)0, (T)0);
  }
  const int64_t off = vi.in_off + src * a.in_tstride;
  C x;
  if (a.in_mode == IO_C) {
    x = gld(reinterpret_cast<const C*>(a.in) + off);
  } else {
    const T* p = reinterpret_cast<const T*>(a.in);
    T re = gld(p + off);
    T im = (a.in_mode == IO_RP && (vi.flags & 1)) ? gld(p + off + a.in_ld) : (T)0;
    x = cmake(re, im);
  }
  if (a.pre_dc) {
    C d = gld(a.pre_dc + n);
    x = cmul(x, a.pre_conj ? cconj(d) : d);
  } else if (a.pre_dr) {
    x = cscale(x, gld(a.pre_dr + n));
  }
  return x;
}

// Stores run in two phases so that the loads they need (diagonal, row map) are all issued
// before the first store: prep applies the diagonal and the scale to x and returns the
// destination row (-1: nothing to store); commit writes (or accumulates) x there.
template <typename T>
__device__ __forceinline__ int fft_store_prep(const FftArgs<T>& a, const VecInfo& vi, int t,
                                              typename Cx<T>::t& x) {
  typedef typename Cx<T>::t C;
  if (vi.out_off < 0) return -1;
  const int64_t n = (int64_t)t * a.out_fmul + vi.out_n2;
  if (n >= a.Lout) return -1;
  if (a.post_dc) {
    C d = gld(a.post_dc + n);
    x = cmul(x, a.post_conj ? cconj(d) : d);
  } else if (a.post_dr) {
    x = cscale(x, gld(a.post_dr + n));
  }
  x = cscale(x, a.scale);
  return a.post_map ? gld(a.post_map + n) : (int)n;
}

template <typename T>
__device__ __forceinline__ void fft_store_commit(const FftArgs<T>& a, const VecInfo& vi, int dst,
                                                 typename Cx<T>::t x) {
  typedef typename Cx<T>::t C;
  if (dst < 0) return;
  const int64_t off = vi.out_off + (int64_t)dst * a.out_tstride;
  if (a.out_mode == IO_C) {
    C* p = reinterpret_cast<C*>(a.out) + off;
    if (a.beta) x = cadd(x, gld(p));
    gst(p, x);
  } else {
    T* p = reinterpret_cast<T*>(a.out) + off;
    gst(p, a.beta ? x.x + gld(p) : x.x);
    if (a.out_mode == IO_RP && (vi.flags & 1)) {
      p += a.out_ld;
      gst(p, a.beta ? x.y + gld(p) : x.y);
    }
  }
}

template <typename T>
int fft_max_tile() { return sizeof(T) == 4 ? 16384 : 8192; }

}  // namespace fm
