// Tile FFT kernel with the transform length fixed at compile time.
//
// Same algorithm and the same launch descriptor (FftArgs) as the runtime-length engine in
// fft_impl.cuh -- V vectors of length L per CTA in shared memory, radix-8/4/2 Stockham
// passes with the elements of each butterfly in registers, the spectrum product of a
// circulant between the last forward and the first inverse pass -- but with L a template
// parameter the radix schedule, the thread-to-butterfly mapping and every in-tile index
// are compile-time constants, so the passes unroll completely and the shared-memory
// addresses of a butterfly reduce to one base plus constant strides.  Loads and stores
// still go through the per-vector table and the fused pre/post operations of FftArgs.
#pragma once
#include "fft_impl.cuh"

namespace fm {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

template <int LOGL>
struct Sched {
  static constexpr int NR = (LOGL + 2) / 3;  // passes: radix 8, then one radix 4 or 2
  __host__ __device__ static constexpr int lr(int p) { return p < LOGL / 3 ? 3 : LOGL - 3 * (LOGL / 3); }
  __host__ __device__ static constexpr int ns_inv(int q) {
    int s = 0;
    for (int i = 0; i < q; ++i) s += lr(NR - 1 - i);
    return s;
  }
};

template <int LOGL, int LOGV>
__device__ __forceinline__ int sp2(int t, int v) {
  constexpr bool VF = (1 << LOGV) >= 16;
  const int lin = VF ? ((t << LOGV) + v) : ((v << LOGL) + t);
  return lin + (lin >> 4);
}

template <int THREADS, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void bfly2(int q, int& j, int& v) {
  constexpr bool VF = (1 << LOGV) >= 16;
  const int b = threadIdx.x + q * THREADS;
  if (VF) {
    v = b & ((1 << LOGV) - 1);
    j = b >> LOGV;
  } else {
    j = b & ((1 << (LOGL - LR)) - 1);
    v = b >> (LOGL - LR);
  }
}

template <typename C, int THREADS, int EPT, int LOGL, int LOGV, int LR>
__device__ __forceinline__ void p2_read(C (&r)[EPT], const C* s) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<THREADS, LOGL, LOGV, LR>(q, j, v);
#pragma unroll
    for (int k = 0; k < R; ++k) r[q * R + k] = s[sp2<LOGL, LOGV>(j + (k << (LOGL - LR)), v)];
  }
}

// outputs of a radix-2^LR pass to (j / Ns) Ns R + j % Ns + k Ns (natural order when Ns R = L)
template <typename C, int THREADS, int EPT, int LOGL, int LOGV, int LR, int LOGNS>
__device__ __forceinline__ void p2_write(const C (&r)[EPT], C* s) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int j, v;
    bfly2<THREADS, LOGL, LOGV, LR>(q, j, v);
    const int base = ((j >> LOGNS) << (LOGNS + LR)) + (j & ((1 << LOGNS) - 1));
#pragma unroll
    for (int k = 0; k < R; ++k) s[sp2<LOGL, LOGV>(base + (k << LOGNS), v)] = r[q * R + k];
  }
}

template <typename C, int THREADS, int EPT, int LOGL, int LOGV, int LR, int LOGNS>
__device__ __forceinline__ void p2_compute(C (&r)[EPT], int dir, const C* __restrict__ tw) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    if (LOGNS > 0) {
      int j, v;
      bfly2<THREADS, LOGL, LOGV, LR>(q, j, v);
      C w = tw[(j & ((1 << LOGNS) - 1)) << (kTwLog - LOGNS - LR)];
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

// Two-pass twiddle W_N^(t n2) of element t of a vector (n2 = its column in the plan).
template <typename T>
__device__ __forceinline__ typename Cx<T>::t tw_direct(typename Cx<T>::t x, const typename Cx<T>::t* tab,
                                                      int64_t mask, int conj, int t, const VecInfo& vi) {
  if (!tab) return x;
  typename Cx<T>::t w = gld(tab + (((int64_t)t * vi.tw_n2) & mask));
  return cmul(x, conj ? cconj(w) : w);
}

// The same twiddle along a staged loop in which a thread keeps one vector and t advances by
// a constant: w <- w * W^(dt n2) after each element (falls back to table reads otherwise).
template <typename T>
struct TwRec {
  typedef typename Cx<T>::t C;
  const C* tab;
  int64_t mask;
  int conj;
  bool rec;
  C w, ws;
  __device__ __forceinline__ TwRec(const C* tab_, int64_t mask_, int conj_, const VecInfo* vinfo, bool one_vector,
                                   int dt, int logv)
      : tab(tab_), mask(mask_), conj(conj_), rec(tab_ && one_vector) {
    if (rec) {
      const VecInfo& vi = vinfo[threadIdx.x & ((1 << logv) - 1)];
      const int t0 = threadIdx.x >> logv;
      w = gld(tab + (((int64_t)t0 * vi.tw_n2) & mask));
      ws = gld(tab + (((int64_t)dt * vi.tw_n2) & mask));
      if (conj) {
        w = cconj(w);
        ws = cconj(ws);
      }
    }
  }
  __device__ __forceinline__ C apply(C x, int t, const VecInfo& vi) {
    if (!tab) return x;
    if (!rec) return tw_direct<T>(x, tab, mask, conj, t, vi);
    x = cmul(x, w);
    w = cmul(w, ws);
    return x;
  }
};

template <typename C, int THREADS, int EPT, int LOGL, int LOGV, int P, bool INV>
__device__ __forceinline__ void p2_run(C (&r)[EPT], C* s, int dir, const C* tw) {
  using S = Sched<LOGL>;
  if constexpr (P < S::NR) {
    constexpr int LR = INV ? S::lr(S::NR - 1 - P) : S::lr(P);
    constexpr int LOGNS = INV ? S::ns_inv(P) : 3 * P;
    if constexpr (P > 0) p2_read<C, THREADS, EPT, LOGL, LOGV, LR>(r, s);
    p2_compute<C, THREADS, EPT, LOGL, LOGV, LR, LOGNS>(r, dir, tw);
    if constexpr (P + 1 < S::NR) {
      __syncthreads();
      p2_write<C, THREADS, EPT, LOGL, LOGV, LR, LOGNS>(r, s);
      __syncthreads();
    }
    p2_run<C, THREADS, EPT, LOGL, LOGV, P + 1, INV>(r, s, dir, tw);
  }
}

// SIMPLE: no fused operation on either side (complex in and out, natural index, no map,
// diagonal, scale or accumulation): loads and stores are a base plus a stride.
// Resident CTAs per SM the register allocation is held to, for FP32 tiles: 3 x 256 threads
// (24 warps per SM), 2 x 512 x 16; the 512 x 32 and FP64 tiles need their registers.
template <typename T, int THREADS, int EPT>
__host__ __device__ constexpr int fft2_min_blocks() {
  return sizeof(T) != 4 ? 1 : (THREADS <= 256 ? 3 : (EPT <= 16 ? 2 : 1));
}

template <typename T, int LOGL, int THREADS, int EPT, bool SIMPLE>
__global__ void __launch_bounds__(THREADS, fft2_min_blocks<T, THREADS, EPT>()) fft2_kernel(const __grid_constant__ FftArgs<T> a) {
  typedef typename Cx<T>::t C;
  constexpr int E = THREADS * EPT, LOGE = ilog2c(E), LOGV = LOGE - LOGL, V = 1 << LOGV;
  constexpr int L = 1 << LOGL;
  using S = Sched<LOGL>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  VecInfo* vinfo = reinterpret_cast<VecInfo*>(smem_raw + fft_vinfo_offset<C>(E));
  const int64_t g0 = (int64_t)blockIdx.x * V;
  const int64_t nvec = a.ncu * a.outer * a.inner;

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
  __syncthreads();

  // load: every element of this thread first (all loads in flight together), then the
  // shared-memory stores, in the order that is contiguous in HBM
  C r[EPT];
  if (SIMPLE) {
    const C* in = reinterpret_cast<const C*>(a.in);
    const int64_t ts = a.in_tstride;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      int t, v;
      if (a.in_vcontig) { v = e & (V - 1); t = e >> LOGV; }
      else { t = e & (L - 1); v = e >> LOGL; }
      const int64_t off = vinfo[v].in_off;
      r[i] = (off >= 0 && t < a.Lin) ? gld(in + off + t * ts) : cmake((T)0, (T)0);
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      int t, v;
      if (a.in_vcontig) { v = e & (V - 1); t = e >> LOGV; }
      else { t = e & (L - 1); v = e >> LOGL; }
      s[sp2<LOGL, LOGV>(t, v)] = r[i];
    }
  } else if (a.in_vcontig) {
    // vectors fastest: with V <= THREADS each thread keeps one vector and t steps by
    // THREADS / V, so the two-pass twiddle W^(t n2) follows a recurrence
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      const int v = e & (V - 1), t = e >> LOGV;
      r[i] = fft_load<T>(a, vinfo[v], t);
    }
    TwRec<T> tw(a.pre_tw, a.tw_mask, a.pre_tw_conj, vinfo, V <= THREADS, THREADS >> LOGV, LOGV);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      const int v = e & (V - 1), t = e >> LOGV;
      s[sp2<LOGL, LOGV>(t, v)] = tw.apply(r[i], t, vinfo[v]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      const int t = e & (L - 1), v = e >> LOGL;
      r[i] = fft_load<T>(a, vinfo[v], t);
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      const int t = e & (L - 1), v = e >> LOGL;
      s[sp2<LOGL, LOGV>(t, v)] = tw_direct<T>(r[i], a.pre_tw, a.tw_mask, a.pre_tw_conj, t, vinfo[v]);
    }
  }
  __syncthreads();

  constexpr int LR0 = S::lr(0);
  constexpr int LRL = S::lr(S::NR - 1);
  p2_read<C, THREADS, EPT, LOGL, LOGV, LR0>(r, s);
  p2_run<C, THREADS, EPT, LOGL, LOGV, 0, false>(r, s, a.dir0, a.tw);
  if (a.conv) {
    // spectrum product at the natural positions t = j + k L/R of the last forward radix
    constexpr int R = 1 << LRL;
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int j, v;
      bfly2<THREADS, LOGL, LOGV, LRL>(q, j, v);
      const C* sp = a.spec + vinfo[v].soff + j;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        C w = gld(sp + (k << (LOGL - LRL)));
        r[q * R + k] = cmul(r[q * R + k], a.spec_conj ? cconj(w) : w);
      }
    }
    p2_run<C, THREADS, EPT, LOGL, LOGV, 0, true>(r, s, -a.dir0, a.tw);
  }

  // store, staged through shared memory
  __syncthreads();
  if (a.conv) p2_write<C, THREADS, EPT, LOGL, LOGV, LR0, LOGL - LR0>(r, s);
  else p2_write<C, THREADS, EPT, LOGL, LOGV, LRL, LOGL - LRL>(r, s);
  __syncthreads();
  if (SIMPLE) {
    C* out = reinterpret_cast<C*>(a.out);
    const int64_t ts = a.out_tstride;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      int t, v;
      if (a.out_vcontig) { v = e & (V - 1); t = e >> LOGV; }
      else { t = e & (L - 1); v = e >> LOGL; }
      r[i] = s[sp2<LOGL, LOGV>(t, v)];
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = threadIdx.x + i * THREADS;
      int t, v;
      if (a.out_vcontig) { v = e & (V - 1); t = e >> LOGV; }
      else { t = e & (L - 1); v = e >> LOGL; }
      const int64_t off = vinfo[v].out_off;
      if (off >= 0 && t < a.Lout) gst(out + off + t * ts, r[i]);
    }
  } else {
    // two phases in groups of 8 elements: the loads of the fused post operations (diagonal,
    // row map) of a group first, then its stores
    constexpr int G = EPT < 8 ? EPT : 8;
    TwRec<T> tw(a.post_tw, a.tw_mask, a.post_tw_conj, vinfo, a.out_vcontig && V <= THREADS, THREADS >> LOGV, LOGV);
#pragma unroll
    for (int g = 0; g < EPT; g += G) {
      int dst[G];
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const int e = threadIdx.x + (g + k) * THREADS;
        int t, v;
        if (a.out_vcontig) { v = e & (V - 1); t = e >> LOGV; }
        else { t = e & (L - 1); v = e >> LOGL; }
        C x = s[sp2<LOGL, LOGV>(t, v)];
        x = a.out_vcontig ? tw.apply(x, t, vinfo[v])
                          : tw_direct<T>(x, a.post_tw, a.tw_mask, a.post_tw_conj, t, vinfo[v]);
        dst[k] = fft_store_prep<T>(a, vinfo[v], t, x);
        r[g + k] = x;
      }
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const int e = threadIdx.x + (g + k) * THREADS;
        const int v = a.out_vcontig ? (e & (V - 1)) : (e >> LOGL);
        fft_store_commit<T>(a, vinfo[v], dst[k], r[g + k]);
      }
    }
  }
}

template <int LOGL, bool WIDE> struct TileCfg {
  static constexpr int LOGE = WIDE ? (LOGL + 4 > 14 ? 14 : (LOGL + 4 < 12 ? 12 : LOGL + 4))
                                   : (LOGL < 12 ? 12 : LOGL);
  static constexpr int THREADS = LOGE <= 12 ? 256 : 512;
  static constexpr int EPT = (1 << LOGE) / THREADS;
};

template <typename T, int LOGL, bool WIDE>
fm_status fft2_launch_cfg(FftArgs<T> a, cudaStream_t st) {
  typedef typename Cx<T>::t C;
  constexpr int THREADS = TileCfg<LOGL, WIDE>::THREADS;
  constexpr int EPT = TileCfg<LOGL, WIDE>::EPT;
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
  a.in_vcontig = (a.inner > 1 || a.in_ostride == 1) ? 1 : 0;
  a.out_vcontig = (a.inner > 1 || a.out_ostride == 1) ? 1 : 0;
  const size_t smem = fft_vinfo_offset<C>(E) + (size_t)V * sizeof(VecInfo);
  const bool simple = a.in_mode == IO_C && a.out_mode == IO_C && !a.pre_map && !a.pre_dc && !a.pre_dr &&
                      !a.pre_tw && !a.post_tw && !a.post_dc && !a.post_dr && !a.post_map && a.scale == (T)1 &&
                      !a.beta && a.in_fmul == 1 && a.in_fmod == 1 && a.out_fmul == 1 && a.out_fmod == 1;
  auto kern = simple ? fft2_kernel<T, LOGL, THREADS, EPT, true> : fft2_kernel<T, LOGL, THREADS, EPT, false>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned long long> attr_bytes[2][32];
  if (dev < 32 && attr_bytes[simple][dev].load() < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("fft smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_bytes[simple][dev].store(smem);
  }
  kern<<<(unsigned)tiles, THREADS, smem, st>>>(a);
  return after_launch("fft2_kernel");
}

template <typename T, int LOGL>
fm_status fft2_launch(FftArgs<T> a, cudaStream_t st) {
  // a wider tile for strided views of 2^9 .. 2^10 (FP32) or 2^9 (FP64): below 2^9 the
  // default tile already holds 16 vectors, above it E = 16 L exceeds shared memory
  constexpr int maxloge = sizeof(T) == 4 ? 14 : 13;
  if constexpr (LOGL >= 9 && LOGL + 4 <= maxloge) {
    if (a.inner >= 16) return fft2_launch_cfg<T, LOGL, true>(a, st);
  }
  return fft2_launch_cfg<T, LOGL, false>(a, st);
}

}  // namespace fm
