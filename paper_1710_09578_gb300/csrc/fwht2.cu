// Walsh-Hadamard transform along a strided axis (Kron mode products, columns seen as
// [outer][n][inner] with inner >= 16), length fixed at compile time.
//
// H_n = H_2 (x) ... (x) H_2, so the transform is one +- butterfly per index bit, in any
// order.  A CTA holds V = E / n vectors; round p transforms index bits [4p, 4p + 4) of
// every vector with the 16 (or fewer) elements of a group in registers.  The first round
// reads its groups straight from HBM and the last round writes straight to HBM; shared
// memory only carries the exchanges between rounds.  Consecutive threads take
// consecutive vectors (consecutive inner indices), so every warp access is a run of
// contiguous elements.
#include "fm_device.cuh"
#include "fm_internal.h"
#include "fwht.h"
#include "fwht_rounds.cuh"

namespace fm {
namespace {

template <typename W> __device__ __forceinline__ W w_zero();
template <> __device__ __forceinline__ float w_zero<float>() { return 0.f; }
template <> __device__ __forceinline__ int w_zero<int>() { return 0; }
template <> __device__ __forceinline__ float2 w_zero<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ float w_load(const float* p) { return gld(p); }
__device__ __forceinline__ float2 w_load(const float2* p) { return gld(p); }
__device__ __forceinline__ int w_load(const int8_t* p) {
  short v;
  asm volatile("ld.global.s8 %0, [%1];" : "=h"(v) : "l"(p));
  return (int)v;
}
__device__ __forceinline__ int w_load(const int* p) { return gld(p); }
__device__ __forceinline__ float w_old(const float* p) { return gld(p); }
__device__ __forceinline__ float2 w_old(const float2* p) { return gld(p); }
__device__ __forceinline__ int w_old(const int* p) { return gld(p); }
__device__ __forceinline__ void w_store(float* p, float v) { gst(p, v); }
__device__ __forceinline__ void w_store(float2* p, float2 v) { gst(p, v); }
__device__ __forceinline__ void w_store(int* p, int v) {
  asm volatile("st.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct WVec2 {
  int64_t in_off;  // -1 if absent
  int64_t out_off;
};

template <typename W, int THREADS, int EPT, int LOGL, int LOGV, int P>
__device__ __forceinline__ void wround_smem(W (&r)[EPT], W* s) {
  using Rd = WRound<LOGL, P>;
  constexpr int R = 1 << Rd::RB;
  if constexpr (P > 0) {
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int v;
      const int t0 = wgroup<THREADS, LOGV, Rd::SH, Rd::RB>(q, v);
#pragma unroll
      for (int k = 0; k < R; ++k) r[q * R + k] = s[wsp<LOGV>(t0 + (k << Rd::SH), v)];
    }
  }
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) wht_group<W, R>(&r[q * R]);
  if constexpr (P + 1 < Rd::NR) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int v;
      const int t0 = wgroup<THREADS, LOGV, Rd::SH, Rd::RB>(q, v);
#pragma unroll
      for (int k = 0; k < R; ++k) s[wsp<LOGV>(t0 + (k << Rd::SH), v)] = r[q * R + k];
    }
    __syncthreads();
    wround_smem<W, THREADS, EPT, LOGL, LOGV, P + 1>(r, s);
  }
}

template <typename Tin, typename W, typename Tout, int LOGL, int THREADS, int EPT>
__global__ void __launch_bounds__(THREADS, THREADS <= 256 ? 3 : 1) fwht2_kernel(const __grid_constant__ FwhtArgs a) {
  constexpr int E = THREADS * EPT, LOGE = ilog2w(E), LOGV = LOGE - LOGL, V = 1 << LOGV;
  constexpr int NR = WRound<LOGL, 0>::NR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* s = reinterpret_cast<W*>(smem_raw);
  constexpr size_t voff = NR > 1 ? ((((size_t)(E + E / 16 + 1) * sizeof(W)) + 15) & ~(size_t)15) : 0;
  WVec2* vinfo = reinterpret_cast<WVec2*>(smem_raw + voff);
  const int64_t g0 = (int64_t)blockIdx.x * V;
  const int64_t nvec = a.ncols * a.outer * a.inner;
  pdl_launch_dependents();
  for (int v = threadIdx.x; v < V; v += THREADS) {
    WVec2 vi;
    const int64_t g = g0 + v;
    if (g < nvec) {
      const int64_t i = g % a.inner, q = g / a.inner;
      const int64_t o = q % a.outer, c = q / a.outer;
      vi.in_off = c * a.in_ld + o * a.in_ostride + i;
      vi.out_off = c * a.out_ld + o * a.out_ostride + i;
    } else {
      vi.in_off = -1;
      vi.out_off = -1;
    }
    vinfo[v] = vi;
  }
  pdl_wait();
  __syncthreads();

  // round 0 straight from HBM
  using R0 = WRound<LOGL, 0>;
  constexpr int R = 1 << R0::RB;
  const int its = (int)a.in_tstride, ots = (int)a.out_tstride;
  W r[EPT];
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int v;
    const int t0 = wgroup<THREADS, LOGV, 0, R0::RB>(q, v);
    const int64_t off = vinfo[v].in_off;
    const Tin* p = reinterpret_cast<const Tin*>(a.in) + off;
#pragma unroll
    for (int k = 0; k < R; ++k) r[q * R + k] = off >= 0 ? w_load(p + (t0 + k) * its) : w_zero<W>();
  }
  wround_smem<W, THREADS, EPT, LOGL, LOGV, 0>(r, s);

  // last round straight to HBM
  using RL = WRound<LOGL, NR - 1>;
  constexpr int RLn = 1 << RL::RB;
#pragma unroll
  for (int q = 0; q < EPT / RLn; ++q) {
    int v;
    const int t0 = wgroup<THREADS, LOGV, RL::SH, RL::RB>(q, v);
    const int64_t off = vinfo[v].out_off;
    if (off < 0) continue;
    Tout* p = reinterpret_cast<Tout*>(a.out) + off;
    if (a.beta) {
      W old[RLn];
#pragma unroll
      for (int k = 0; k < RLn; ++k) old[k] = w_old(p + (t0 + (k << RL::SH)) * ots);
#pragma unroll
      for (int k = 0; k < RLn; ++k) w_store(p + (t0 + (k << RL::SH)) * ots, w_add(r[q * RLn + k], old[k]));
    } else {
#pragma unroll
      for (int k = 0; k < RLn; ++k) w_store(p + (t0 + (k << RL::SH)) * ots, r[q * RLn + k]);
    }
  }
}

template <typename Tin, typename W, typename Tout, int LOGL>
fm_status fwht2_start(const FwhtArgs& a, cudaStream_t st) {
  constexpr int THREADS = 256, EPT = 16, E = THREADS * EPT, V = E >> LOGL;
  constexpr int NR = WRound<LOGL, 0>::NR;
  const size_t voff = NR > 1 ? ((((size_t)(E + E / 16 + 1) * sizeof(W)) + 15) & ~(size_t)15) : 0;
  const size_t smem = voff + (size_t)V * sizeof(WVec2);
  const int64_t nvec = a.ncols * a.outer * a.inner;
  const int64_t tiles = (nvec + V - 1) / V;
  if (tiles == 0) return FM_OK;
  if (tiles > 0x7fffffffLL) { set_error("fwht: too many tiles"); return FM_ERR_UNSUPPORTED; }
  auto kern = fwht2_kernel<Tin, W, Tout, LOGL, THREADS, EPT>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned long long> attr_bytes[32];
  if (dev < 32 && attr_bytes[dev].load() < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("fwht smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_bytes[dev].store(smem);
  }
  return pdl_go("fwht2_kernel", kern, dim3((unsigned)tiles), dim3(THREADS), smem, st, a);
}

template <typename Tin, typename W, typename Tout>
fm_status fwht2_dispatch(const FwhtArgs& a, cudaStream_t st) {
  switch (a.logL) {
    case 1: return fwht2_start<Tin, W, Tout, 1>(a, st);
    case 2: return fwht2_start<Tin, W, Tout, 2>(a, st);
    case 3: return fwht2_start<Tin, W, Tout, 3>(a, st);
    case 4: return fwht2_start<Tin, W, Tout, 4>(a, st);
    case 5: return fwht2_start<Tin, W, Tout, 5>(a, st);
    case 6: return fwht2_start<Tin, W, Tout, 6>(a, st);
    case 7: return fwht2_start<Tin, W, Tout, 7>(a, st);
    case 8: return fwht2_start<Tin, W, Tout, 8>(a, st);
    default: break;
  }
  set_error("fwht2: no kernel for log2 n = %d", a.logL);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace

// Strided axes with at least 16 vectors side by side (inner >= 16) and n <= 256: the tile
// holds 16 or more vectors, each warp access covers contiguous inner indices.
bool fwht2_ok(const FwhtArgs& a) {
  if (a.logL < 1 || a.logL > 8 || a.inner < 16) return false;
  const int64_t n = (int64_t)1 << a.logL;
  return (n + 1) * a.in_tstride < ((int64_t)1 << 31) && (n + 1) * a.out_tstride < ((int64_t)1 << 31);
}

fm_status fwht2_launch(const FwhtArgs& a, fm_dtype in_dt, cudaStream_t st) {
  switch (in_dt) {
    case FM_F32: return fwht2_dispatch<float, float, float>(a, st);
    case FM_C64: return fwht2_dispatch<float2, float2, float2>(a, st);
    case FM_I8: return fwht2_dispatch<int8_t, int, int>(a, st);
    case FM_I32: return fwht2_dispatch<int, int, int>(a, st);
    default: break;
  }
  set_error("fwht: dtype %d not supported", (int)in_dt);
  return FM_ERR_DTYPE;
}

}  // namespace fm
