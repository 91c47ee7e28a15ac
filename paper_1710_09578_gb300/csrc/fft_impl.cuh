// Batched Stockham FFT engine for the Fourier, Circulant and Toeplitz operators.
//
// One CTA owns a tile of V vectors of length L (L * V = THREADS * EPT elements) in
// shared memory and runs radix-16/8/4/2 Stockham passes over it: each thread keeps EPT
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

// The R inputs t = j + k M (k < R) of one butterfly of vector vi into x[0..R), with the
// fused pre operations (row map P^H, diagonal, real-pair packing).  The uniform decisions
// are taken once per butterfly, and offsets inside a vector are 32-bit: the launcher only
// accepts vectors that span fewer than 2^31 elements.
template <typename T, int R>
__device__ __forceinline__ void fft_load_bfly(const FftArgs<T>& a, const VecInfo& vi, int j, int M,
                                              typename Cx<T>::t* x) {
  typedef typename Cx<T>::t C;
  const C zero = cmake((T)0, (T)0);
  if (vi.in_off < 0) {
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = zero;
    return;
  }
  const int fmul = (int)a.in_fmul, Lin = (int)a.Lin, ts = (int)a.in_tstride;
  const int n0 = j * fmul + vi.in_n2, dn = M * fmul;
  if (a.in_mode == IO_C && !a.pre_map && n0 + (R - 1) * dn < Lin) {
    // complex input, no row map, the whole butterfly inside the vector: no per-element checks
    const C* p = reinterpret_cast<const C*>(a.in) + vi.in_off;
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = gld(p + (n0 + k * dn) * ts);
  } else {
    int src[R];
    if (a.pre_map) {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int n = n0 + k * dn;
        src[k] = n < Lin ? gld(a.pre_map + n) : -1;
      }
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int n = n0 + k * dn;
        src[k] = n < Lin ? n : -1;
      }
    }
    if (a.in_mode == IO_C) {
      const C* p = reinterpret_cast<const C*>(a.in) + vi.in_off;
#pragma unroll
      for (int k = 0; k < R; ++k) x[k] = src[k] >= 0 ? gld(p + src[k] * ts) : zero;
    } else {
      const T* p = reinterpret_cast<const T*>(a.in) + vi.in_off;
      const bool two = a.in_mode == IO_RP && (vi.flags & 1);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        T re = (T)0, im = (T)0;
        if (src[k] >= 0) {
          re = gld(p + src[k] * ts);
          if (two) im = gld(p + src[k] * ts + a.in_ld);
        }
        x[k] = cmake(re, im);
      }
    }
  }
  if (a.pre_dc) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      if (n < Lin) {
        const C d = gld(a.pre_dc + n);
        x[k] = cmul(x[k], a.pre_conj ? cconj(d) : d);
      }
    }
  } else if (a.pre_dr) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      if (n < Lin) x[k] = cscale(x[k], gld(a.pre_dr + n));
    }
  }
}

// The R outputs t = j + k M of one butterfly of vector vi, with the fused post operations
// (diagonal, scale, row map P, accumulation, real-pair unpacking); every load the stores
// need is issued before the first store.
template <typename T, int R>
__device__ __forceinline__ void fft_store_bfly(const FftArgs<T>& a, const VecInfo& vi, int j, int M,
                                               typename Cx<T>::t* x) {
  typedef typename Cx<T>::t C;
  if (vi.out_off < 0) return;
  const int fmul = (int)a.out_fmul, Lout = (int)a.Lout, ts = (int)a.out_tstride;
  const int n0 = j * fmul + vi.out_n2, dn = M * fmul;
  if (a.post_dc) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      if (n < Lout) {
        const C d = gld(a.post_dc + n);
        x[k] = cmul(x[k], a.post_conj ? cconj(d) : d);
      }
    }
  } else if (a.post_dr) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      if (n < Lout) x[k] = cscale(x[k], gld(a.post_dr + n));
    }
  }
  if (a.scale != (T)1) {
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = cscale(x[k], a.scale);
  }
  if (a.out_mode == IO_C && !a.post_map && !a.beta && n0 + (R - 1) * dn < Lout) {
    // complex output, no row map, no accumulation, the whole butterfly inside the vector
    C* p = reinterpret_cast<C*>(a.out) + vi.out_off;
#pragma unroll
    for (int k = 0; k < R; ++k) gst(p + (n0 + k * dn) * ts, x[k]);
    return;
  }
  int dst[R];
  if (a.post_map) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      dst[k] = n < Lout ? gld(a.post_map + n) : -1;
    }
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int n = n0 + k * dn;
      dst[k] = n < Lout ? n : -1;
    }
  }
  if (a.out_mode == IO_C) {
    C* p = reinterpret_cast<C*>(a.out) + vi.out_off;
    if (a.beta) {
      C old[R];
#pragma unroll
      for (int k = 0; k < R; ++k) old[k] = dst[k] >= 0 ? gld(p + dst[k] * ts) : cmake((T)0, (T)0);
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (dst[k] >= 0) gst(p + dst[k] * ts, cadd(x[k], old[k]));
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (dst[k] >= 0) gst(p + dst[k] * ts, x[k]);
    }
  } else {
    T* p = reinterpret_cast<T*>(a.out) + vi.out_off;
    const bool two = a.out_mode == IO_RP && (vi.flags & 1);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (dst[k] < 0) continue;
      T* q = p + dst[k] * ts;
      gst(q, a.beta ? x[k].x + gld(q) : x[k].x);
      if (two) gst(q + a.out_ld, a.beta ? x[k].y + gld(q + a.out_ld) : x[k].y);
    }
  }
}

template <typename T>
int fft_max_tile() { return sizeof(T) == 4 ? 16384 : 8192; }

}  // namespace fm
