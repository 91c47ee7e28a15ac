// Tile FFT kernel with the transform length fixed at compile time.
//
// V vectors of length L per CTA, radix-16 (then 8/4/2) Stockham passes, or radix-32 passes where
// a thread holds 32 elements, with the elements of each butterfly in registers (the DFT of
// Eq. (1) by the butterfly factorisation of Sec. 1) and
// the spectrum product of a circulant (Eq. (5)) in registers between the last forward and
// the first inverse pass.  With L a template parameter the radix schedule, the
// thread-to-butterfly mapping and every in-tile index are compile-time constants, so the
// passes unroll completely.
//
// The first pass reads its butterfly inputs (elements j + k L/R) straight from HBM and the
// last pass writes its outputs (natural order, j + k L/R) straight to HBM; shared memory
// only carries the exchanges between passes.  The thread-to-butterfly mapping follows the
// layout in HBM: VF (vectors contiguous, a strided axis) gives consecutive threads
// consecutive vectors, otherwise consecutive threads take consecutive elements of a
// vector, so each warp access is a few full 32-byte sectors either way (a second pass whose
// contiguous rows land interleaved in the output transposes them through shared memory
// first: store_staged).  A thread issues all of its loads before the first shared-memory
// store.  Loads and stores go through the
// per-vector table and the fused pre/post operations of FftArgs (Diag, row selection,
// zero-padding and truncation, two-pass twiddles, scale, accumulation).
#pragma once
#include "fft_impl.cuh"

namespace fm {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// Radix schedule (log2 of the radix of each pass, first to last): radix-16 passes where
// they save an exchange through shared memory, radix 8 where a radix-2 pass would be left
// over (measured on GB300: lengths 2^9 and 2^6 run faster as 8 x 8 x 8 and 8 x 8).
__host__ __device__ constexpr int sched_lr(int logl, int p) {
  constexpr int t[15][4] = {{0, 0, 0, 0}, {1, 0, 0, 0}, {2, 0, 0, 0}, {3, 0, 0, 0}, {4, 0, 0, 0},
                            {3, 2, 0, 0}, {3, 3, 0, 0}, {4, 3, 0, 0}, {4, 4, 0, 0}, {3, 3, 3, 0},
                            {4, 4, 2, 0}, {4, 4, 3, 0}, {4, 4, 4, 0}, {4, 4, 3, 2}, {4, 4, 4, 2}};
  return t[logl][p];
}
__host__ __device__ constexpr int sched_nr(int logl) {
  int n = 0;
  while (n < 4 && sched_lr(logl, n) > 0) ++n;
  return n;
}

// Tiles whose threads hold fewer than 16 elements cap the radix at 2^LMAX (the EPT elements
// of a thread must hold whole butterflies): ceil(LOGL / LMAX) passes, larger radices first.
__host__ __device__ constexpr int sched_cap_nr(int logl, int lmax) { return (logl + lmax - 1) / lmax; }
__host__ __device__ constexpr int sched_cap_lr(int logl, int lmax, int p) {
  return p < sched_cap_nr(logl, lmax)
             ? logl / sched_cap_nr(logl, lmax) + (p < logl % sched_cap_nr(logl, lmax) ? 1 : 0)
             : 0;
}
// log2 of the largest radix a thread with EPT elements can hold (at most 32).
template <int EPT>
__host__ __device__ constexpr int ept_lmax() {
  return EPT >= 32 ? 5 : (EPT >= 16 ? 4 : (EPT >= 8 ? 3 : (EPT >= 4 ? 2 : 1)));
}

// Radix 32 (threads of 32 elements): as few passes as radix 32 allows, balanced.
template <int LOGL, int LMAX = 4>
struct Sched {
  static_assert(LOGL >= 1 && LOGL <= 14, "transform length 2^1 .. 2^14 per tile");
  static_assert(LMAX >= 1 && LMAX <= 5, "radix 2 .. 32");
  static constexpr int NR = LMAX == 4 ? sched_nr(LOGL) : sched_cap_nr(LOGL, LMAX);
  __host__ __device__ static constexpr int lr(int p) {
    return LMAX == 4 ? sched_lr(LOGL, p) : sched_cap_lr(LOGL, LMAX, p);
  }
  // log2 Ns before forward pass q (radices in order) and before inverse pass q (reversed)
  __host__ __device__ static constexpr int ns_fwd(int q) {
    int s = 0;
    for (int i = 0; i < q; ++i) s += lr(i);
    return s;
  }
  __host__ __device__ static constexpr int ns_inv(int q) {
    int s = 0;
    for (int i = 0; i < q; ++i) s += lr(NR - 1 - i);
    return s;
  }
};

// Shared-memory word of element t of tile vector v (VF: vectors fastest), one pad slot
// every 16 words.
//
// LAY 1: the layout of radix-32 tiles.  Strided tiles of 2^10 (8 vectors, VF) write the
// elements t = 32 j + k (k < 32) of butterfly j in one exchange and read t = j + 32 k in the
// other; with t = 32 th + tl, word = 264 th + 8 tl + v.  Tiles with contiguous vectors (not VF)
// whose first pass has radix 32 take one pad slot every 32 words: word = v (L + L / 32) + t +
// t / 32.  In both, every exchange pattern of the tile steps a register by a constant, and in
// each half-warp the 8-byte words fall in 16 distinct bank pairs, where the layout with a pad
// every 16 words puts two (contiguous) or four (strided) butterflies on the same pairs.
template <bool VF, int LOGL, int LOGV, int LAY = 0>
__device__ __forceinline__ int sp2(int t, int v) {
  if constexpr (LAY == 1 && VF) {
    static_assert(LOGL == 10 && LOGV == 3, "radix-32 layout of strided tiles: 8 vectors of 2^10");
    return (t >> 5) * 264 + (t & 31) * 8 + v;
  } else if constexpr (LAY == 1) {
    return v * ((1 << LOGL) + (1 << (LOGL - 5))) + t + (t >> 5);
  } else {
    const int lin = VF ? ((t << LOGV) + v) : ((v << LOGL) + t);
    return lin + (lin >> 4);
  }
}
template <int EPT, int LOGL, int LOGV, bool VF>
__host__ __device__ constexpr int layout_of() {
  return EPT < 32 ? 0 : (VF ? ((LOGL == 10 && LOGV == 3) ? 1 : 0) : (Sched<LOGL, 5>::lr(0) == 5 ? 1 : 0));
}

// Butterfly q of this thread in a radix-2^LR pass: vector v, index j in [0, L/R).  THREADS is
// the size of the thread group that owns the tile (the whole CTA, or one of its groups).
template <bool VF, int THREADS, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void bfly2(int q, int& j, int& v) {
  const int b = (threadIdx.x & (THREADS - 1)) + q * THREADS;
  if (VF) {
    v = b & ((1 << LOGV) - 1);
    j = b >> LOGV;
  } else {
    j = b & ((1 << (LOGL - LR)) - 1);
    v = b >> (LOGL - LR);
  }
}

// Elements t0 + k DT (k < R) of vector v: when the word step is a multiple of 16 the pad
// slots between two of them are a constant too, so the addresses are one base plus
// compile-time offsets.  In the radix-32 layouts the steps are constants for DT = 1 (t0 = R j,
// never across a pad) and, strided, DT = 32 or, contiguous, DT a multiple of 32.
template <int DT, bool VF, int LOGV>
__host__ __device__ constexpr int lay1_step() {
  return VF ? (DT == 1 ? (1 << LOGV) : 264) : (DT == 1 ? 1 : DT + DT / 32);
}
template <bool VF, int DT>
__host__ __device__ constexpr bool lay1_const() {
  return VF ? (DT == 1 || DT == 32) : (DT == 1 || DT % 32 == 0);
}
template <bool VF, int LOGL, int LOGV, int DT, int R, int LAY, typename C>
__device__ __forceinline__ void s_gather(C* x, const C* s, int t0, int v) {
  constexpr int S = VF ? (DT << LOGV) : DT;
  if constexpr (LAY == 1) {
    static_assert(!VF || lay1_const<VF, DT>(), "radix-32 strided layout: the two exchanges of a 2^10 tile");
    if constexpr (lay1_const<VF, DT>()) {
      const C* p = s + sp2<VF, LOGL, LOGV, 1>(t0, v);
#pragma unroll
      for (int k = 0; k < R; ++k) x[k] = p[k * lay1_step<DT, VF, LOGV>()];
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k) x[k] = s[sp2<VF, LOGL, LOGV, 1>(t0 + k * DT, v)];
    }
  } else if constexpr (S % 16 == 0) {
    const C* p = s + sp2<VF, LOGL, LOGV>(t0, v);
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = p[k * (S + S / 16)];
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sp2<VF, LOGL, LOGV>(t0 + k * DT, v)];
  }
}
template <bool VF, int LOGL, int LOGV, int DT, int R, int LAY, typename C>
__device__ __forceinline__ void s_scatter(const C* x, C* s, int t0, int v) {
  constexpr int S = VF ? (DT << LOGV) : DT;
  if constexpr (LAY == 1) {
    static_assert(!VF || lay1_const<VF, DT>(), "radix-32 strided layout: the two exchanges of a 2^10 tile");
    if constexpr (lay1_const<VF, DT>()) {
      C* p = s + sp2<VF, LOGL, LOGV, 1>(t0, v);
#pragma unroll
      for (int k = 0; k < R; ++k) p[k * lay1_step<DT, VF, LOGV>()] = x[k];
    } else {
#pragma unroll
      for (int k = 0; k < R; ++k) s[sp2<VF, LOGL, LOGV, 1>(t0 + k * DT, v)] = x[k];
    }
  } else if constexpr (S % 16 == 0) {
    C* p = s + sp2<VF, LOGL, LOGV>(t0, v);
#pragma unroll
    for (int k = 0; k < R; ++k) p[k * (S + S / 16)] = x[k];
  } else {
#pragma unroll
    for (int k = 0; k < R; ++k) s[sp2<VF, LOGL, LOGV>(t0 + k * DT, v)] = x[k];
  }
}

template <typename C, bool VF, int THREADS, int EPT, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void p2_read(C (&r)[EPT], const C* s) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
    s_gather<VF, LOGL, LOGV, (1 << (LOGL - LR)), R, layout_of<EPT, LOGL, LOGV, VF>()>(&r[q * R], s, j, v);
  }
}

// outputs of a radix-2^LR pass to (j / Ns) Ns R + j % Ns + k Ns (natural order when Ns R = L)
template <typename C, bool VF, int THREADS, int EPT, int LOGL, int LOGV, int LR, int LOGNS>
__device__ __forceinline__ void p2_write(const C (&r)[EPT], C* s) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
    const int base = ((j >> LOGNS) << (LOGNS + LR)) + (j & ((1 << LOGNS) - 1));
    s_scatter<VF, LOGL, LOGV, (1 << LOGNS), R, layout_of<EPT, LOGL, LOGV, VF>()>(&r[q * R], s, base, v);
  }
}

// x[k] *= w^k for k = 1 .. R-1; the powers as a tree (w^2, w^4, w^8 by squaring, the rest
// as one product of those), so the dependency chain stays short.
template <typename C, int R>
__device__ __forceinline__ void twiddle_powers(C* x, C w) {
  if constexpr (R == 2) {
    x[1] = cmul(x[1], w);
  } else {
    C p[R < 16 ? R : (R == 16 ? 16 : 8)];
    p[1] = w;
    p[2] = cmul(w, w);
    p[3] = cmul(p[2], w);
    if constexpr (R >= 8) {
      p[4] = cmul(p[2], p[2]);
      p[5] = cmul(p[4], w);
      p[6] = cmul(p[4], p[2]);
      p[7] = cmul(p[4], p[3]);
    }
    if constexpr (R == 16) {
      p[8] = cmul(p[4], p[4]);
#pragma unroll
      for (int k = 9; k < 16; ++k) p[k] = cmul(p[8], p[k - 8]);
    }
    if constexpr (R == 32) {
      // w^(8a + b) = w^(8a) w^b: eight low powers and three high ones live, not 31
      const C w8 = cmul(p[4], p[4]);
#pragma unroll
      for (int k = 1; k < 8; ++k) x[k] = cmul(x[k], p[k]);
      C h = w8;
#pragma unroll
      for (int a = 1; a < 4; ++a) {
        x[8 * a] = cmul(x[8 * a], h);
#pragma unroll
        for (int b = 1; b < 8; ++b) x[8 * a + b] = cmul(x[8 * a + b], cmul(h, p[b]));
        if (a < 3) h = cmul(h, w8);
      }
    } else {
#pragma unroll
      for (int k = 1; k < R; ++k) x[k] = cmul(x[k], p[k]);
    }
  }
}

// The R twiddles W_{Ns R}^((j mod Ns) k), k < R, of butterfly j: one row of the pass-twiddle
// table (fm_device.cuh), read as 16-byte vectors through the read-only path (the table is
// written once per device, long before any transform).
template <int LR>
__device__ __forceinline__ void tw_row(float2 (&w)[1 << LR], const float2* row) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < R / 2; ++q) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row) + q);
    w[2 * q] = make_float2(v.x, v.y);
    w[2 * q + 1] = make_float2(v.z, v.w);
  }
}
template <int LR>
__device__ __forceinline__ void tw_row(double2 (&w)[1 << LR], const double2* row) {
#pragma unroll
  for (int k = 0; k < (1 << LR); ++k) w[k] = __ldg(row + k);
}

// x * conj(w)
template <typename C> __device__ __forceinline__ C cmul_conj(C a, C b) {
  return cmake(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

template <typename C, bool VF, int THREADS, int EPT, int LOGL, int LOGV, int LR, int LOGNS>
__device__ __forceinline__ void p2_compute(C (&r)[EPT], int dir, const C* __restrict__ twp) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    if (LOGNS > 0) {
      int j, v;
      bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
      // (a radix-32 pass reads its base twiddle W_(Ns R)^(j mod Ns) from the radix-16 table of
      // the same span: entry 1 of row j mod Ns there is the same power)
      constexpr int LT = LR < 4 ? LR : 4;
      const C* row = twp + pass_tw_offset(LOGNS + LR, LT) + ((int64_t)(j & ((1 << LOGNS) - 1)) << LT);
      if constexpr (sizeof(C) == 16) {
        static_assert(LR <= 4, "radix-32 passes are compiled for FP32 tiles only");
        // FP64: every power from the table (a product tree of FP64 multiplies costs more)
        C w[R];
        tw_row<LR>(w, row);
        if (dir > 0) {
#pragma unroll
          for (int k = 1; k < R; ++k) r[q * R + k] = cmul_conj(r[q * R + k], w[k]);
        } else {
#pragma unroll
          for (int k = 1; k < R; ++k) r[q * R + k] = cmul(r[q * R + k], w[k]);
        }
      } else {
        // FP32: the base twiddle from the table and its powers by a product tree (measured
        // faster on GB300 than reading all R - 1 powers: fewer loads in flight per butterfly)
        C w = __ldg(row + 1);
        if (dir > 0) w = cconj(w);
        twiddle_powers<C, R>(&r[q * R], w);
      }
    }
    if (R == 32) dft32(&r[q * R], dir);
    else if (R == 16) dft16(&r[q * R], dir);
    else if (R == 8) dft8(&r[q * R], dir);
    else if (R == 4) dft4(&r[q * R], dir);
    else dft2(&r[q * R]);
  }
}

// FRESH: the first pass's inputs came from global memory, so no thread can still be reading the
// exchange buffer when the first pass writes it (the barrier before that write is skipped).
// Barrier of the thread group that owns a tile: the whole CTA, or group threadIdx.x / THREADS
// of BLOCK / THREADS groups with a named barrier of its own (ids 1, 2, ...).
template <int THREADS, int BLOCK>
__device__ __forceinline__ void tile_sync() {
  if constexpr (THREADS == BLOCK) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / THREADS)), "r"(THREADS) : "memory");
  }
}

// LM: cap of log2 of the radix (0: the largest radix a thread's EPT elements hold).
template <int EPT, int LM>
__host__ __device__ constexpr int radix_cap() { return LM > 0 && LM < ept_lmax<EPT>() ? LM : ept_lmax<EPT>(); }

template <typename C, bool VF, int THREADS, int EPT, int LOGL, int LOGV, int P, bool INV, bool FRESH = false,
          int LM = 0, int BLOCK = THREADS>
__device__ __forceinline__ void p2_run(C (&r)[EPT], C* s, int dir, const C* tw) {
  using S = Sched<LOGL, radix_cap<EPT, LM>()>;
  if constexpr (P < S::NR) {
    constexpr int LR = INV ? S::lr(S::NR - 1 - P) : S::lr(P);
    constexpr int LOGNS = INV ? S::ns_inv(P) : S::ns_fwd(P);
    if constexpr (P > 0) p2_read<C, VF, THREADS, EPT, LOGL, LOGV, LR>(r, s);
    p2_compute<C, VF, THREADS, EPT, LOGL, LOGV, LR, LOGNS>(r, dir, tw);
    if constexpr (P + 1 < S::NR) {
      if constexpr (!(FRESH && P == 0)) tile_sync<THREADS, BLOCK>();
      p2_write<C, VF, THREADS, EPT, LOGL, LOGV, LR, LOGNS>(r, s);
      tile_sync<THREADS, BLOCK>();
    }
    p2_run<C, VF, THREADS, EPT, LOGL, LOGV, P + 1, INV, FRESH, LM, BLOCK>(r, s, dir, tw);
  }
}

// Two-pass twiddle W_N^(t n2) on the R elements t = j + k M of a butterfly (n2 = the
// vector's column in the plan): two table reads per butterfly (W^(j n2) and the step
// W^(M n2)), then runs of H elements by recurrence, each run started from the previous one by
// the step's H-th power (formed by squaring), so no product chain is longer than H + R / H.
template <typename T, int R, int H>
__device__ __forceinline__ void tw_butterfly(typename Cx<T>::t* x, const typename Cx<T>::t* tab, int64_t mask,
                                             int conj, int j, int M, int64_t n2) {
  typedef typename Cx<T>::t C;
  C w = gld(tab + (((int64_t)j * n2) & mask));
  C ws = gld(tab + (((int64_t)M * n2) & mask));
  if (conj) {
    w = cconj(w);
    ws = cconj(ws);
  }
  C wh = ws;
#pragma unroll
  for (int e = 1; e < H; e <<= 1) wh = cmul(wh, wh);
#pragma unroll
  for (int h = 0; h < R; h += H) {
    C u = w;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      x[h + k] = cmul(x[h + k], u);
      if (k + 1 < H) u = cmul(u, ws);
    }
    if (h + H < R) w = cmul(w, wh);
  }
}

// Inputs of the first pass straight from HBM: element j + k L/R of vector v into register
// q R + k of butterfly q, every load issued before any is used.
template <typename T, bool VF, bool SIMPLE, int THREADS, int EPT, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void load_first(typename Cx<T>::t (&r)[EPT], const FftArgs<T>& a,
                                           const VecInfo* vinfo) {
  typedef typename Cx<T>::t C;
  constexpr int R = 1 << LR, M = 1 << (LOGL - LR);
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
    const VecInfo& vi = vinfo[v];
    if (SIMPLE) {
      // unit stride: constant offsets from one base; otherwise one base and a step
      const bool unit = a.in_tstride == 1;
      const int64_t step = unit ? M : (int64_t)M * a.in_tstride;
      const C* in = reinterpret_cast<const C*>(a.in) + vi.in_off + (unit ? j : (int64_t)j * a.in_tstride);
      if (vi.in_off >= 0 && j + (R - 1) * M < a.Lin) {
        // the whole butterfly lies inside the vector: no per-element checks
#pragma unroll
        for (int k = 0; k < R; ++k) r[q * R + k] = gld(unit ? in + k * M : in + k * step);
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const bool ok = vi.in_off >= 0 && j + k * M < a.Lin;
          r[q * R + k] = ok ? gld(unit ? in + k * M : in + k * step) : cmake((T)0, (T)0);
        }
      }
    } else {
      // fused loads in runs of at most 8 (registers: each run keeps its row indices live)
      constexpr int H = R > 8 ? 8 : R;
#pragma unroll
      for (int h = 0; h < R; h += H) fft_load_bfly<T, H>(a, vi, j + h * M, M, &r[q * R + h]);
    }
  }
  if (!SIMPLE && a.pre_tw) {
    constexpr int H = R > 8 ? 8 : R;
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int j, v;
      bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
      tw_butterfly<T, R, H>(&r[q * R], a.pre_tw, a.tw_mask, a.pre_tw_conj, j, M, vinfo[v].tw_n2);
    }
  }
}

// Outputs of the last pass (natural order, element j + k L/R in register q R + k) straight
// to HBM; with fused post operations the loads they need for a butterfly come first.
template <typename T, bool VF, bool SIMPLE, int THREADS, int EPT, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void store_last(typename Cx<T>::t (&r)[EPT], const FftArgs<T>& a,
                                           const VecInfo* vinfo) {
  typedef typename Cx<T>::t C;
  constexpr int R = 1 << LR, M = 1 << (LOGL - LR);
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<VF, THREADS, LOGL, LOGV, LR>(q, j, v);
    const VecInfo& vi = vinfo[v];
    if (SIMPLE) {
      const bool unit = a.out_tstride == 1;
      const int64_t step = unit ? M : (int64_t)M * a.out_tstride;
      C* out = reinterpret_cast<C*>(a.out) + vi.out_off + (unit ? j : (int64_t)j * a.out_tstride);
      if (vi.out_off >= 0 && j + (R - 1) * M < a.Lout) {
#pragma unroll
        for (int k = 0; k < R; ++k) gst(unit ? out + k * M : out + k * step, r[q * R + k]);
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (vi.out_off >= 0 && j + k * M < a.Lout) gst(unit ? out + k * M : out + k * step, r[q * R + k]);
        }
      }
    } else {
      constexpr int H = R > 8 ? 8 : R;
      if (a.post_tw) tw_butterfly<T, R, H>(&r[q * R], a.post_tw, a.tw_mask, a.post_tw_conj, j, M, vi.tw_n2);
#pragma unroll
      for (int h = 0; h < R; h += H) fft_store_bfly<T, H>(a, vi, j + h * M, M, &r[q * R + h]);
    }
  }
}

// Outputs of the last pass through shared memory, for tiles whose vectors are contiguous on
// the input side (consecutive threads on consecutive elements of a vector) but interleaved on
// the output side (element t of vector v at t * out_fmul + v: the second pass of a long
// transform).  The registers go to word t (V + 1) + v (both the write and the read below are
// free of bank conflicts), then each thread stores elements of consecutive vectors, so a
// warp's stores cover whole sectors instead of one 8-byte word in each of 32.  Plain complex
// output with scale and accumulation only (the launcher checks).
template <typename T, int THREADS, int EPT, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void store_staged(typename Cx<T>::t (&r)[EPT], typename Cx<T>::t* s, const FftArgs<T>& a,
                                             const VecInfo* vinfo) {
  typedef typename Cx<T>::t C;
  constexpr int R = 1 << LR, M = 1 << (LOGL - LR), V = 1 << LOGV;
  __syncthreads();  // every thread is done with the exchange buffer
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<false, THREADS, LOGL, LOGV, LR>(q, j, v);
#pragma unroll
    for (int k = 0; k < R; ++k) s[(j + k * M) * (V + 1) + v] = r[q * R + k];
  }
  __syncthreads();
  const int fmul = (int)a.out_fmul, Lout = (int)a.Lout, ts = (int)a.out_tstride;
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const int e = (int)threadIdx.x + i * THREADS;
    const int v = e & (V - 1), t = e >> LOGV;
    const VecInfo& vi = vinfo[v];
    const int n = t * fmul + vi.out_n2;
    if (vi.out_off < 0 || n >= Lout) continue;
    C y = s[t * (V + 1) + v];
    if (a.scale != (T)1) y = cscale(y, a.scale);
    C* p = reinterpret_cast<C*>(a.out) + vi.out_off + (int64_t)n * ts;
    if (a.beta) y = cadd(y, gld(p));
    gst(p, y);
  }
}

// Resident CTAs per SM the register allocation is held to, for FP32 tiles: 4 x 256 threads
// (32 warps per SM; at most a few registers spill), 3 x 256 for the convolution tiles of
// 2^5, 2^6 and 2^9 (radix-8 passes with two butterflies per thread, whose spectrum product
// would spill tens of bytes at 64 registers), 2 x 512 x 16 and 2 x 256 x 32 (radix-32
// tiles, 128 registers); the 512 x 32 and FP64 tiles need their registers.
template <typename T, int LOGL, int THREADS, int EPT, bool CONV>
__host__ __device__ constexpr int fft2_min_blocks() {
  return sizeof(T) != 4 || THREADS < 256
             ? 1
             : (THREADS <= 256 ? (EPT >= 32 ? 2 : (CONV && (LOGL == 5 || LOGL == 6 || LOGL == 9) ? 3 : 4))
                               : (EPT <= 16 ? 2 : 1));
}

// The exchange buffer (none when a single radix pass does the whole transform in
// registers), then the per-vector table.
template <typename C, int LOGL, int EPT, int LM = 0>
__host__ __device__ constexpr size_t fft2_vinfo_offset(int E) {
  return Sched<LOGL, radix_cap<EPT, LM>()>::NR > 1 ? fft_vinfo_offset<C>(E) : 0;
}

// SIMPLE: no fused operation on either side (complex in and out, natural index, no map,
// diagonal, twiddle, scale or accumulation): loads and stores are a base plus a stride.
// CONV: transform, spectrum product, inverse transform (circulant and Toeplitz products).
// G > 1: the tile's V vectors are split into G groups of V / G, each transformed by THREADS / G
// threads with barriers of their own (the groups never wait for one another).
template <typename T, int LOGL, int THREADS, int EPT, bool VF, bool SIMPLE, bool CONV, int LM = 0, int G = 1>
__global__ void __launch_bounds__(THREADS, fft2_min_blocks<T, LOGL, THREADS, EPT, CONV>())
    fft2_kernel(const __grid_constant__ FftArgs<T> a) {
  typedef typename Cx<T>::t C;
  constexpr int E = THREADS * EPT, LOGE = ilog2c(E), LOGV = LOGE - LOGL, V = 1 << LOGV;
  using S = Sched<LOGL, radix_cap<EPT, LM>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  VecInfo* vinfo = reinterpret_cast<VecInfo*>(smem_raw + fft2_vinfo_offset<C, LOGL, EPT, LM>(E));
  const int64_t g0 = (int64_t)blockIdx.x * V;
  const int64_t nvec = a.ncu * a.outer * a.inner;
  pdl_launch_dependents();

  for (int v = threadIdx.x; v < V; v += THREADS) {
    VecInfo vi;
    const int64_t g = g0 + v;
    if (g < nvec) {
      const int64_t i = g % a.inner, q = g / a.inner;
      const int64_t o = q % a.outer, c = q / a.outer;
      const int64_t oi = o * a.inner + i;
      const int64_t cin = a.in_mode == IO_RP ? 2 * c : c;
      const int64_t cout = a.out_mode == IO_RP ? 2 * c : c;
      vi.in_off = cin * a.in_ld + o * a.in_ostride + (i % a.in_imod);
      vi.out_off = cout * a.out_ld + o * a.out_ostride + (i % a.out_imod);
      vi.in_n2 = (int32_t)((oi / a.in_fdiv) % a.in_fmod);
      vi.out_n2 = (int32_t)((oi / a.out_fdiv) % a.out_fmod);
      vi.tw_n2 = (int32_t)((oi / a.tw_div) % a.tw_mod);
      vi.flags = (2 * c + 1 < a.ncols) ? 1 : 0;
      vi.soff = a.spec_omod > 1 ? ((o % a.spec_omod) << LOGL) : 0;
    } else {
      vi.in_off = -1;
      vi.out_off = -1;
      vi.in_n2 = vi.out_n2 = vi.tw_n2 = 0;
      vi.flags = 0;
      vi.soff = 0;
    }
    vinfo[v] = vi;
  }
  pdl_wait();
  __syncthreads();

  constexpr int LR0 = S::lr(0);
  constexpr int LRL = S::lr(S::NR - 1);
  // this thread's group: its threads, its vectors and its part of the exchange buffer
  static_assert(G >= 1 && V % G == 0 && THREADS / G >= 32, "groups of whole warps and whole vectors");
  constexpr int TG = THREADS / G, LOGVG = LOGV - ilog2c(G), EG = E / G;
  const int grp = G > 1 ? (int)(threadIdx.x / TG) : 0;
  C* sg = s + grp * (EG + EG / 16);
  const VecInfo* vg = vinfo + grp * (V / G);
  C r[EPT];
  load_first<T, VF, SIMPLE, TG, EPT, LOGL, LOGVG, LR0>(r, a, vg);
  p2_run<C, VF, TG, EPT, LOGL, LOGVG, 0, false, true, LM, THREADS>(r, sg, a.dir0, a.tw);
  if constexpr (CONV) {
    // spectrum product at the natural positions t = j + k L/R of the last forward radix
    constexpr int R = 1 << LRL;
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int j, v;
      bfly2<VF, TG, LOGL, LOGVG, LRL>(q, j, v);
      const C* sp = a.spec + vg[v].soff + j;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        // the spectrum is written once at construction: read-only path
        C w = __ldg(sp + (k << (LOGL - LRL)));
        r[q * R + k] = cmul(r[q * R + k], a.spec_conj ? cconj(w) : w);
      }
    }
    p2_run<C, VF, TG, EPT, LOGL, LOGVG, 0, true, false, LM, THREADS>(r, sg, -a.dir0, a.tw);
    store_last<T, VF, SIMPLE, TG, EPT, LOGL, LOGVG, LR0>(r, a, vg);
  } else {
    if constexpr (!VF && !SIMPLE && G == 1 && LOGV >= 4) {
      if (a.out_stage) {
        store_staged<T, THREADS, EPT, LOGL, LOGV, LRL>(r, s, a, vinfo);
        return;
      }
    }
    store_last<T, VF, SIMPLE, TG, EPT, LOGL, LOGVG, LRL>(r, a, vg);
  }
}

// Tile shapes: 0 the default (2^12 elements, or one vector), 1 wide (16 vectors of a
// strided view, 8 for 2^10 so that two CTAs of 16 elements per thread share an SM), 2 small (2^9 elements, four warps of 4 elements per thread: many CTAs for
// small FP64 problems, with a warp on every SM sub-partition's FP64 unit), 4 radix 32 (FP32
// 2^9 and 2^10: 2^13 elements, 256 threads of 32 elements, two passes per transform instead of
// three).
template <int LOGL, int MODE> struct TileCfg {
  static constexpr int LOGE = MODE == 4 ? 13
                              : MODE == 1 ? (LOGL + 4 > 13 ? 13 : (LOGL + 4 < 12 ? 12 : LOGL + 4))
                              : MODE == 2 ? (LOGL < 9 ? 9 : LOGL)
                                          : (LOGL < 12 ? 12 : LOGL);
  static constexpr int THREADS = MODE == 2 ? 128 : (MODE == 4 || LOGE <= 12 ? 256 : 512);
  static constexpr int EPT = (1 << LOGE) / THREADS;
};

template <typename T, int LOGL, int THREADS, int EPT, bool VF, bool SIMPLE, bool CONV, int LM, int G>
fm_status fft2_start(const FftArgs<T>& a, int64_t tiles, size_t smem, cudaStream_t st) {
  auto kern = fft2_kernel<T, LOGL, THREADS, EPT, VF, SIMPLE, CONV, LM, G>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned long long> attr_bytes[32];
  if (dev < 32 && attr_bytes[dev].load() < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("fft smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_bytes[dev].store(smem);
  }
  // the kernel's label in errors and traces: element type, length, layout, convolution
  static const std::string label = std::string("fft2_kernel<") + (sizeof(T) == 4 ? "f32" : "f64") + ",L=2^" +
                                   std::to_string(LOGL) + (VF ? ",strided" : "") + (SIMPLE ? "" : ",fused") +
                                   (CONV ? ",conv" : "") + (LM ? ",radix<=" + std::to_string(1 << LM) : "") +
                                   (!LM && EPT >= 32 ? ",radix=32" : "") +
                                   (G > 1 ? ",groups=" + std::to_string(G) : "") + ">";
  return pdl_go(label.c_str(), kern, dim3((unsigned)tiles), dim3(THREADS), smem, st, a);
}

template <typename T, int LOGL, int THREADS, int EPT, bool VF, int LM, int G = 1>
fm_status fft2_pick(const FftArgs<T>& a, bool simple, int64_t tiles, size_t smem, cudaStream_t st) {
  if (a.conv) {
    return simple ? fft2_start<T, LOGL, THREADS, EPT, VF, true, true, LM, G>(a, tiles, smem, st)
                  : fft2_start<T, LOGL, THREADS, EPT, VF, false, true, LM, G>(a, tiles, smem, st);
  }
  return simple ? fft2_start<T, LOGL, THREADS, EPT, VF, true, false, LM, G>(a, tiles, smem, st)
                : fft2_start<T, LOGL, THREADS, EPT, VF, false, false, LM, G>(a, tiles, smem, st);
}

// The radix-capped schedules (radix <= 8) are compiled for the FP32 tiles of 2^9 .. 2^12, the
// lengths of the benchmarked passes; elsewhere the cap is ignored.
template <typename T, int LOGL>
constexpr bool has_rcap_variant() { return sizeof(T) == 4 && LOGL >= 9 && LOGL <= 12; }

template <typename T, int LOGL, int MODE>
fm_status fft2_launch_cfg(FftArgs<T> a, cudaStream_t st) {
  typedef typename Cx<T>::t C;
  constexpr int THREADS = TileCfg<LOGL, MODE>::THREADS;
  constexpr int EPT = TileCfg<LOGL, MODE>::EPT;
  constexpr int E = THREADS * EPT;
  constexpr int V = E >> LOGL;
  a.L = 1 << LOGL;
  a.logL = LOGL;
  a.V = V;
  a.logV = ilog2c(V);
  const int64_t nvec = a.ncu * a.outer * a.inner;
  if (nvec == 0) return FM_OK;
  const int64_t tiles = (nvec + V - 1) / V;
  if (tiles > 0x7fffffffLL) { set_error("fft: too many tiles"); return FM_ERR_UNSUPPORTED; }
  // offsets inside a vector are 32-bit in the kernel
  const int64_t lim = (int64_t)1 << 31;
  if ((a.Lin + 1) * a.in_tstride >= lim || (a.Lout + 1) * a.out_tstride >= lim || a.L * a.in_fmul >= lim ||
      a.L * a.out_fmul >= lim || a.Lin >= lim || a.Lout >= lim) {
    set_error("fft: a vector spans 2^31 elements or more");
    return FM_ERR_UNSUPPORTED;
  }
  a.in_vcontig = (a.inner > 1 || a.in_ostride == 1) ? 1 : 0;
  a.out_vcontig = (a.inner > 1 || a.out_ostride == 1) ? 1 : 0;
  const bool capped = MODE != 4 && has_rcap_variant<T, LOGL>() && a.rcap == 3 && ept_lmax<EPT>() > 3;
  const size_t smem = (capped ? fft2_vinfo_offset<C, LOGL, EPT, 3>(E) : fft2_vinfo_offset<C, LOGL, EPT>(E)) +
                      (size_t)V * sizeof(VecInfo);
  // transposed outputs through shared memory (store_staged): contiguous input vectors (not
  // VF), at least 16 of them, whose element t lands at t * out_fmul + (vector index)
  a.out_stage = (V >= 16 && !(a.in_vcontig && V > 1) && !a.conv && a.out_mode == IO_C && !a.post_map && !a.post_dc &&
                 !a.post_dr && !a.post_tw && a.inner == 1 && a.out_fdiv == 1 && a.out_fmul >= V && a.out_fmod >= V)
                    ? 1 : 0;
  const bool simple = a.in_mode == IO_C && a.out_mode == IO_C && !a.pre_map && !a.pre_dc && !a.pre_dr &&
                      !a.pre_tw && !a.post_tw && !a.post_dc && !a.post_dr && !a.post_map && a.scale == (T)1 &&
                      !a.beta && a.in_fmul == 1 && a.in_fmod == 1 && a.out_fmul == 1 && a.out_fmod == 1;
  if constexpr (MODE != 4 && has_rcap_variant<T, LOGL>() && ept_lmax<EPT>() > 3) {
    if (capped) {
      if constexpr (V > 1) {
        if (a.in_vcontig) return fft2_pick<T, LOGL, THREADS, EPT, true, 3>(a, simple, tiles, smem, st);
      }
      return fft2_pick<T, LOGL, THREADS, EPT, false, 3>(a, simple, tiles, smem, st);
    }
  }
  if constexpr (V > 1) {
    // tile shape 3: the wide strided tile in 4 independent groups (FP32 wide tiles only)
    if constexpr (MODE == 1 && sizeof(T) == 4 && V % 4 == 0 && THREADS / 4 >= 32) {
      if (a.tile == 3 && a.in_vcontig) return fft2_pick<T, LOGL, THREADS, EPT, true, 0, 4>(a, simple, tiles, smem, st);
    }
    if (a.in_vcontig) return fft2_pick<T, LOGL, THREADS, EPT, true, 0>(a, simple, tiles, smem, st);
  }
  return fft2_pick<T, LOGL, THREADS, EPT, false, 0>(a, simple, tiles, smem, st);
}

template <typename T, int LOGL>
fm_status fft2_launch(FftArgs<T> a, cudaStream_t st) {
  // a wider tile for strided views of 2^9 .. 2^10 (FP32) or 2^9 (FP64): below 2^9 the
  // default tile already holds 16 vectors, above it E = 16 L exceeds shared memory
  constexpr int maxloge = sizeof(T) == 4 ? 14 : 13;
  if constexpr (sizeof(T) == 8 && LOGL >= 5 && LOGL <= 9) {
    if (a.small) return fft2_launch_cfg<T, LOGL, 2>(a, st);
  }
  if constexpr (sizeof(T) == 4 && (LOGL == 9 || LOGL == 10)) {
    // radix-32 tiles: by default for strided views of 2^10 (measured on GB300: the Kron
    // circulant pass of 2^10 along a stride of 64, 350 -> 310 us), and where a.tile is 4
    if (a.tile == 4 || (a.tile == 0 && LOGL == 10 && a.inner >= 16)) return fft2_launch_cfg<T, LOGL, 4>(a, st);
  }
  if constexpr (LOGL >= 9 && LOGL + 4 <= maxloge) {
    // wide tiles for strided views by default (a.tile 0); a.tile 1 forces the default tile and
    // 2 or 3 the wide one (the calibration's choice)
    const bool wide = (a.tile == 2 || a.tile == 3) ? a.inner > 1 : (a.tile == 1 ? false : a.inner >= 16);
    if (wide) return fft2_launch_cfg<T, LOGL, 1>(a, st);
  }
  return fft2_launch_cfg<T, LOGL, 0>(a, st);
}

}  // namespace fm
