// Fused mode products for Kron(H, ..., F): the Hadamard factor of the outermost axis and
// the Fourier factor of the innermost (contiguous) axis applied in one pass.
//
// The mode products of a Kron operator commute (each acts on its own axis of the column
// seen as a tensor, Sec. 3, Eq. (7)-style compositions), so the outer and inner factors can
// be applied together.  A CTA takes the tile [2^LA][2^LB] of one column and one index of
// the middle axes: rows are 2^LB contiguous complex64 elements, row a sits a * sa further
// on.  The Fourier transform of the rows runs as the Stockham passes of the FFT tile kernel
// (first pass straight from HBM, rows contiguous in shared memory), the Walsh-Hadamard
// transform of the 2^LB columns as register rounds over the same shared-memory words
// (vectors fastest), the last round straight to HBM.  One pass over HBM instead of two.
#include "fft2.cuh"
#include "fwht_rounds.cuh"
#include "kron_hf.h"

namespace fm {
namespace {

template <int THREADS, int EPT, int LA, int LB, int P>
__device__ __forceinline__ void hrounds(float2 (&r)[EPT], float2* s, const KronHFArgs& a, float2* out) {
  using Rd = WRound<LA, P>;
  constexpr int R = 1 << Rd::RB;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int v;
    const int t0 = wgroup<THREADS, LB, Rd::SH, Rd::RB>(q, v);
#pragma unroll
    for (int k = 0; k < R; ++k) r[q * R + k] = s[wsp<LB>(t0 + (k << Rd::SH), v)];
    wht_group<float2, R>(&r[q * R]);
  }
  if constexpr (P + 1 < Rd::NR) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int v;
      const int t0 = wgroup<THREADS, LB, Rd::SH, Rd::RB>(q, v);
#pragma unroll
      for (int k = 0; k < R; ++k) s[wsp<LB>(t0 + (k << Rd::SH), v)] = r[q * R + k];
    }
    __syncthreads();
    hrounds<THREADS, EPT, LA, LB, P + 1>(r, s, a, out);
  } else {
    // last round: element (row t0 + k 2^SH, column v) straight to HBM
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int v;
      const int t0 = wgroup<THREADS, LB, Rd::SH, Rd::RB>(q, v);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        float2* p = out + (int64_t)(t0 + (k << Rd::SH)) * a.sa + v;
        float2 y = cscale(r[q * R + k], a.scale);
        if (a.beta) y = cadd(y, gld(p));
        gst(p, y);
      }
    }
  }
}

template <int LA, int LB>
__global__ void __launch_bounds__(1 << (LA + LB - 4), 1) kron_hf_kernel(const __grid_constant__ KronHFArgs a) {
  constexpr int THREADS = 1 << (LA + LB - 4), EPT = 16;
  using S = Sched<LB>;
  constexpr int LR0 = S::lr(0), LRL = S::lr(S::NR - 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int64_t col = tile / a.nmid, mid = tile % a.nmid;
  const float2* in = a.in + col * a.in_ld + (mid << LB);
  float2* out = a.out + col * a.out_ld + (mid << LB);
  float2 r[EPT];
  pdl_launch_dependents();
  pdl_wait();
  // Fourier along the rows: first pass straight from HBM (elements j + k M of row v)
  {
    constexpr int R = 1 << LR0, M = 1 << (LB - LR0);
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int j, v;
      bfly2<false, THREADS, LB, LA, LR0>(q, j, v);
      const float2* p = in + (int64_t)v * a.sa + j;
#pragma unroll
      for (int k = 0; k < R; ++k) r[q * R + k] = gld(p + k * M);
    }
  }
  p2_run<float2, false, THREADS, EPT, LB, LA, 0, false, true>(r, s, a.dir, a.tw);
  __syncthreads();
  p2_write<float2, false, THREADS, EPT, LB, LA, LRL, LB - LRL>(r, s);  // natural order, rows contiguous
  __syncthreads();
  // Walsh-Hadamard along the columns (the 2^LB columns are the vectors, fastest)
  hrounds<THREADS, EPT, LA, LB, 0>(r, s, a, out);
}

// ---- the same pass with each tile split over a cluster of CL = 2 or 4 CTAs
// CTA rank r of the cluster holds rows [2^LAL r, 2^LAL (r + 1)) of the [2^LA][2^LB] tile, LAL =
// LA - log2 CL (1/CL of the shared memory, so CL clusters' CTAs share an SM and one tile's loads
// overlap another's arithmetic).  Each CTA runs the row Fourier transforms and H_{2^LAL} over its
// rows; the top log2 CL Hadamard digits (H_CL across the CTAs) combine the parts: rank r writes
// columns [2^LB r / CL, 2^LB (r + 1) / CL) of all rows, reading the other CTAs' parts of those
// columns from their shared memory (distributed shared memory, (CL - 1) / CL^2 of the tile per
// CTA).  Cluster barriers (hardware barriers, no polling) order the parts before the exchange
// and keep every CTA's shared memory alive until the others have read it.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// full cluster barrier: every thread of every CTA arrives (its shared-memory writes released to
// the cluster) and waits for all (acquire); also a barrier of this CTA's own threads
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive once this thread is done reading the other CTAs' shared memory: the release orders
// those reads before the arrival, so no CTA passes its final wait and exits while its shared
// memory is still being read (the wait follows the global stores)
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ float2 ld_dsmem(const float2* local_ptr, unsigned rank) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(local_ptr);
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(addr), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(remote) : "memory");
  return v;
}

// every round of H_{2^LAL} over the rows of the tile in shared memory, results written back (the
// caller synchronises after the last round)
template <int THREADS, int EPT, int LAL, int LB, int P>
__device__ __forceinline__ void hrounds_local(float2 (&r)[EPT], float2* s) {
  using Rd = WRound<LAL, P>;
  constexpr int R = 1 << Rd::RB;
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int v;
    const int t0 = wgroup<THREADS, LB, Rd::SH, Rd::RB>(q, v);
#pragma unroll
    for (int k = 0; k < R; ++k) r[q * R + k] = s[wsp<LB>(t0 + (k << Rd::SH), v)];
    wht_group<float2, R>(&r[q * R]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < EPT / R; ++q) {
    int v;
    const int t0 = wgroup<THREADS, LB, Rd::SH, Rd::RB>(q, v);
#pragma unroll
    for (int k = 0; k < R; ++k) s[wsp<LB>(t0 + (k << Rd::SH), v)] = r[q * R + k];
  }
  if constexpr (P + 1 < Rd::NR) {
    __syncthreads();
    hrounds_local<THREADS, EPT, LAL, LB, P + 1>(r, s);
  }
}

template <int LA, int LB, int CL>
__host__ __device__ constexpr int hfc_threads() { return 1 << (LA - ilog2c(CL) + LB - 4); }

template <int LA, int LB, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(hfc_threads<LA, LB, CL>(), CL)
    kron_hfc_kernel(const __grid_constant__ KronHFArgs a) {
  constexpr int LAL = LA - ilog2c(CL), THREADS = hfc_threads<LA, LB, CL>(), EPT = 16;
  constexpr int ROWS = 1 << LAL, COLS = 1 << LB, CPC = COLS / CL;   // rows per CTA, columns per CTA
  constexpr int RSTEP = THREADS / CPC, NK = ROWS / RSTEP;           // NK = 16 / CL rows per thread
  static_assert(LAL >= 2 && THREADS >= 32 && CPC >= 1 && RSTEP >= 1 && NK * RSTEP == ROWS, "cluster tile shape");
  using S = Sched<LB>;
  constexpr int LR0 = S::lr(0), LRL = S::lr(S::NR - 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const unsigned rank = cluster_rank();
  const int64_t tile = blockIdx.x / CL;
  const int64_t col = tile / a.nmid, mid = tile % a.nmid;
  const float2* in = a.in + col * a.in_ld + (mid << LB) + (int64_t)rank * ROWS * a.sa;
  float2* out = a.out + col * a.out_ld + (mid << LB);
  float2 r[EPT];
  pdl_launch_dependents();
  pdl_wait();
  // Fourier along this CTA's rows: first pass straight from HBM
  {
    constexpr int R = 1 << LR0, M = 1 << (LB - LR0);
#pragma unroll
    for (int q = 0; q < EPT / R; ++q) {
      int j, v;
      bfly2<false, THREADS, LB, LAL, LR0>(q, j, v);
      const float2* p = in + (int64_t)v * a.sa + j;
#pragma unroll
      for (int k = 0; k < R; ++k) r[q * R + k] = gld(p + k * M);
    }
  }
  // L2 prefetch of this CTA's rows of the tile a residency wave later, while this one computes
  if (a.pf_tiles > 0 && tile + a.pf_tiles < a.ntiles) {
    constexpr int LINES = ROWS * COLS * 8 / 128;  // 128-byte lines of this CTA's rows
    const int64_t nt = tile + a.pf_tiles;
    const int64_t ncol = nt / a.nmid, nmid = nt % a.nmid;
    const float2* nin = a.in + ncol * a.in_ld + (nmid << LB) + (int64_t)rank * ROWS * a.sa;
    for (int l = threadIdx.x; l < LINES; l += THREADS) {
      constexpr int LPR = COLS * 8 / 128;  // lines per row
      const float2* pl = nin + (int64_t)(l / LPR) * a.sa + (l % LPR) * 16;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(pl)));
    }
  }
  p2_run<float2, false, THREADS, EPT, LB, LAL, 0, false, true>(r, s, a.dir, a.tw);
  __syncthreads();
  p2_write<float2, false, THREADS, EPT, LB, LAL, LRL, LB - LRL>(r, s);
  __syncthreads();
  hrounds_local<THREADS, EPT, LAL, LB, 0>(r, s);
  // the top digits across the cluster: part p = the rows of CTA p, for this CTA's columns
  const int c = (int)rank * CPC + (int)(threadIdx.x % CPC);
  const int i0 = (int)(threadIdx.x / CPC);
  float2 x[NK][CL];
  cluster_sync();
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    const float2* mine = s + wsp<LB>(i0 + k * RSTEP, c);
#pragma unroll
    for (int p = 0; p < CL; ++p) x[k][p] = p == (int)rank ? *mine : ld_dsmem(mine, (unsigned)p);
  }
  cluster_arrive_release();
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    wht_group<float2, CL>(x[k]);
#pragma unroll
    for (int p = 0; p < CL; ++p) x[k][p] = cscale(x[k][p], a.scale);
  }
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    const int i = i0 + k * RSTEP;
#pragma unroll
    for (int p = 0; p < CL; ++p) {
      float2* q = out + (int64_t)(p * ROWS + i) * a.sa + c;
      float2 y = x[k][p];
      if (a.beta) y = cadd(y, gld(q));
      gst(q, y);
    }
  }
  // the other CTAs read this CTA's shared memory until they have arrived
  cluster_wait();
}

template <int LA, int LB, int CL>
fm_status hfc_start(KronHFArgs a, cudaStream_t st) {
  constexpr int E = 1 << (LA - ilog2c(CL) + LB);
  constexpr size_t smem = (size_t)(E + E / 16 + 1) * sizeof(float2);
  auto kern = kron_hfc_kernel<LA, LB, CL>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned> attr_set{0};
  if (dev < 32 && !(attr_set.load() & (1u << dev))) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("kron_hf cluster smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_set.fetch_or(1u << dev);
  }
  if (a.ntiles == 0) return FM_OK;
  if (a.ntiles > 0x1fffffffLL) { set_error("kron_hf cluster: too many tiles"); return FM_ERR_UNSUPPORTED; }
  if (a.pair == 3) {
    // prefetch distance: half of the tiles resident on the GPU (two CTAs per SM, CL per tile);
    // measured on GB300 for the 2^24 x 4 Kron workload: half a wave 265 us per launch, a whole
    // wave 267, two waves 279, no prefetch 277
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      set_error("kron_hf cluster: SM count query failed");
      return FM_ERR_CUDA;
    }
    a.pf_tiles = (int64_t)nsm / CL;
  }
  static const std::string label =
      "kron_hfc_kernel<" + std::to_string(LA) + "," + std::to_string(LB) + ",cluster=" + std::to_string(CL) + ">";
  return pdl_go(label.c_str(), kern, dim3((unsigned)(CL * a.ntiles)), dim3(hfc_threads<LA, LB, CL>()), smem, st, a);
}

template <int LA, int LB>
fm_status hf_start(const KronHFArgs& a, cudaStream_t st);

// the forms a tile shape admits: CTA pairs for every shape, quads where a CTA keeps whole warps
template <int LA, int LB>
fm_status hf_pick(const KronHFArgs& a, cudaStream_t st) {
  if (a.pair == 2) {
    if constexpr (LA + LB >= 11) return hfc_start<LA, LB, 4>(a, st);
  }
  if (a.pair == 3) return hfc_start<LA, LB, 2>(a, st);
  if (a.pair >= 1) return hfc_start<LA, LB, 2>(a, st);
  return hf_start<LA, LB>(a, st);
}

template <int LA, int LB>
fm_status hf_start(const KronHFArgs& a, cudaStream_t st) {
  constexpr int E = 1 << (LA + LB);
  constexpr size_t smem = (size_t)(E + E / 16 + 1) * sizeof(float2);
  auto kern = kron_hf_kernel<LA, LB>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned> attr_set{0};
  if (dev < 32 && !(attr_set.load() & (1u << dev))) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("kron_hf smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_set.fetch_or(1u << dev);
  }
  if (a.ntiles == 0) return FM_OK;
  if (a.ntiles > 0x7fffffffLL) { set_error("kron_hf: too many tiles"); return FM_ERR_UNSUPPORTED; }
  static const std::string label = "kron_hf_kernel<" + std::to_string(LA) + "," + std::to_string(LB) + ">";
  return pdl_go(label.c_str(), kern, dim3((unsigned)a.ntiles), dim3(1 << (LA + LB - 4)), smem, st, a);
}

}  // namespace

bool kron_hf_ok(int la, int lb) { return la >= 4 && la <= 8 && lb >= 4 && lb <= 8 && la + lb >= 10 && la + lb <= 14; }

fm_status kron_hf_launch(const KronHFArgs& a, int la, int lb, cudaStream_t st) {
#define FM_HF(A, B) \
  if (la == A && lb == B) return hf_pick<A, B>(a, st);
  FM_HF(4, 6) FM_HF(5, 5) FM_HF(6, 4)
  FM_HF(4, 7) FM_HF(5, 6) FM_HF(6, 5) FM_HF(7, 4)
  FM_HF(4, 8) FM_HF(5, 7) FM_HF(6, 6) FM_HF(7, 5) FM_HF(8, 4)
  FM_HF(5, 8) FM_HF(6, 7) FM_HF(7, 6) FM_HF(8, 5)
  FM_HF(6, 8) FM_HF(7, 7) FM_HF(8, 6)
#undef FM_HF
  set_error("kron_hf: no kernel for 2^%d x 2^%d", la, lb);
  return FM_ERR_UNSUPPORTED;
}

}  // namespace fm
