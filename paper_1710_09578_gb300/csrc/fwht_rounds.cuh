// In-register Walsh-Hadamard rounds shared by the strided-axis kernel (fwht2.cu) and the
// fused Kron tile (kron_hf.cu): round P transforms index bits [4P, 4P + 4) of every vector
// of a tile held in shared memory with vectors fastest (word (t V + v) + pad), the group of
// up to 16 elements a thread owns in registers.
#pragma once
#include "fm_device.cuh"

namespace fm {

__host__ __device__ constexpr int ilog2w(int x) { return x <= 1 ? 0 : 1 + ilog2w(x >> 1); }

__device__ __forceinline__ float w_add(float a, float b) { return a + b; }
__device__ __forceinline__ float w_sub(float a, float b) { return a - b; }
__device__ __forceinline__ int w_add(int a, int b) { return a + b; }
__device__ __forceinline__ int w_sub(int a, int b) { return a - b; }
__device__ __forceinline__ float2 w_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 w_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename W, int R>
__device__ __forceinline__ void wht_group(W* x) {
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if ((i & h) == 0) {
        const W a = x[i], b = x[i + h];
        x[i] = w_add(a, b);
        x[i + h] = w_sub(a, b);
      }
    }
  }
}

// Round P: bits [4P, 4P + RB) of an n = 2^LOGL vector.
template <int LOGL, int P>
struct WRound {
  static constexpr int SH = 4 * P;
  static constexpr int RB = LOGL - SH < 4 ? LOGL - SH : 4;
  static constexpr int NR = (LOGL + 3) / 4;
};

// Group q of this thread in a round: vector v and first element t0 (elements t0 + k 2^SH).
template <int THREADS, int LOGV, int SH, int RB>
__device__ __forceinline__ int wgroup(int q, int& v) {
  const int b = threadIdx.x + q * THREADS;
  v = b & ((1 << LOGV) - 1);
  const int j = b >> LOGV;
  return ((j >> SH) << (SH + RB)) | (j & ((1 << SH) - 1));
}

template <int LOGV>
__device__ __forceinline__ int wsp(int t, int v) {
  const int lin = (t << LOGV) + v;
  return lin + (lin >> 4);
}

}  // namespace fm
