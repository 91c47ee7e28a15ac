// Fast Walsh-Hadamard transform for the Sylvester Hadamard operator (CUDA-core paths).
//
// H_n = H_2 (x) H_2 (x) ... (x) H_2 in natural order, H[i, j] = (-1)^popcount(i & j),
// so the transform is a sequence of +- butterflies, one per index bit, in any order.
// A CTA holds a tile of V vectors of length Lp in shared memory and applies in-place
// radix-16 passes (four bits per pass, done in registers).  A column longer than one tile
// (n = C * Lp) is split by its C top index values: with x = [x_0; ...; x_{C-1}] the output
// block r is H_Lp (sum_s H_C[r, s] x_s), so CTA r combines the C input blocks while
// loading and transforms its own block; the C CTAs of a column read the same lines at
// the same time, so HBM sees each input byte about once.
//
// Element types: f32 -> f32, c64 -> c64 (as two real channels), int8 -> int32 (exact).
#include <algorithm>

#include "fm_device.cuh"
#include "fm_internal.h"
#include "fwht.h"

namespace fm {

__device__ __forceinline__ float wadd(float a, float b) { return a + b; }
__device__ __forceinline__ float wsub(float a, float b) { return a - b; }
__device__ __forceinline__ int wadd(int a, int b) { return a + b; }
__device__ __forceinline__ int wsub(int a, int b) { return a - b; }
__device__ __forceinline__ float2 wadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 wsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename W> __device__ __forceinline__ W wzero();
template <> __device__ __forceinline__ float wzero<float>() { return 0.f; }
template <> __device__ __forceinline__ int wzero<int>() { return 0; }
template <> __device__ __forceinline__ float2 wzero<float2>() { return make_float2(0.f, 0.f); }

template <typename Tin, typename W> __device__ __forceinline__ W wload(const Tin* p);
template <> __device__ __forceinline__ float wload<float, float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float2 wload<float2, float2>(const float2* p) { return *p; }
template <> __device__ __forceinline__ int wload<int8_t, int>(const int8_t* p) { return (int)*p; }
template <> __device__ __forceinline__ int wload<int, int>(const int* p) { return *p; }

template <typename W, int R>
__device__ __forceinline__ void wht_regs(W* x) {
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if ((i & h) == 0) {
        W a = x[i], b = x[i + h];
        x[i] = wadd(a, b);
        x[i + h] = wsub(a, b);
      }
    }
  }
}

// One in-place pass over index bits [sh, sh + RB) of every vector in the tile.
template <typename W, int RB, int THREADS, int E>
__device__ __forceinline__ void wht_pass(W* s, int sh, int logLp, int logV, int vfast) {
  constexpr int R = 1 << RB;
  const int V = 1 << logV;
  for (int b = threadIdx.x; b < (E >> RB); b += THREADS) {
    int v, lo, hi;
    if (vfast) {
      v = b & (V - 1);
      const int rest = b >> logV;
      lo = rest & ((1 << sh) - 1);
      hi = rest >> sh;
    } else {
      lo = b & ((1 << sh) - 1);
      const int rest = b >> sh;
      const int nhi_log = logLp - sh - RB;
      hi = rest & ((1 << nhi_log) - 1);
      v = rest >> nhi_log;
    }
    const int t0 = (hi << (sh + RB)) + lo;
    W x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int t = t0 + (k << sh);
      x[k] = s[spad(vfast ? ((t << logV) + v) : ((v << logLp) + t))];
    }
    wht_regs<W, R>(x);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int t = t0 + (k << sh);
      s[spad(vfast ? ((t << logV) + v) : ((v << logLp) + t))] = x[k];
    }
  }
}

template <typename W>
__host__ __device__ constexpr size_t fwht_vinfo_offset(int E) {
  return (((size_t)(E + E / 16 + 1) * sizeof(W)) + 15) & ~(size_t)15;
}

struct WVec {
  int64_t in_off;   // -1 if absent
  int64_t out_off;
};

template <typename Tin, typename W, typename Tout, int THREADS, int EPT>
__global__ void __launch_bounds__(THREADS) fwht_tile_kernel(const __grid_constant__ FwhtArgs a) {
  constexpr int E = THREADS * EPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* s = reinterpret_cast<W*>(smem_raw);
  // per-vector table after the padded tile, on a 16-byte boundary (it holds int64 fields)
  WVec* vinfo = reinterpret_cast<WVec*>(smem_raw + fwht_vinfo_offset<W>(E));
  const int logLp = a.logLp, logV = a.logV, V = 1 << a.logV;
  const int C = 1 << a.logC;
  // blockIdx.x = tile * C + part
  const int part = (int)(blockIdx.x & (C - 1));
  const int64_t tile = (int64_t)blockIdx.x >> a.logC;
  const int64_t g0 = tile * V;
  const int64_t nvec = a.ncols * a.outer * a.inner;
  const int vfast = V >= 16;
  pdl_launch_dependents();

  for (int v = threadIdx.x; v < V; v += THREADS) {
    WVec vi;
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

  const Tin* in = reinterpret_cast<const Tin*>(a.in);
  Tout* out = reinterpret_cast<Tout*>(a.out);
  const int64_t Lp = (int64_t)1 << logLp;
  // ---- load and combine the C blocks with row `part` of H_C
  for (int e = threadIdx.x; e < E; e += THREADS) {
    int t, v;
    if (vfast) { v = e & (V - 1); t = e >> logV; }
    else { t = e & ((1 << logLp) - 1); v = e >> logLp; }
    const WVec vi = vinfo[v];
    W acc = wzero<W>();
    if (vi.in_off >= 0) {
      for (int sblk = 0; sblk < C; ++sblk) {
        W x = wload<Tin, W>(in + vi.in_off + ((int64_t)sblk * Lp + t) * a.in_tstride);
        acc = (__popc(sblk & part) & 1) ? wsub(acc, x) : wadd(acc, x);
      }
    }
    s[spad(vfast ? ((t << logV) + v) : ((v << logLp) + t))] = acc;
  }
  __syncthreads();

  // ---- in-place passes, up to four bits each
  for (int sh = 0; sh < logLp; sh += 4) {
    const int rb = min(4, logLp - sh);
    switch (rb) {
      case 4: wht_pass<W, 4, THREADS, E>(s, sh, logLp, logV, vfast); break;
      case 3: wht_pass<W, 3, THREADS, E>(s, sh, logLp, logV, vfast); break;
      case 2: wht_pass<W, 2, THREADS, E>(s, sh, logLp, logV, vfast); break;
      default: wht_pass<W, 1, THREADS, E>(s, sh, logLp, logV, vfast); break;
    }
    __syncthreads();
  }

  // ---- store block `part`
  for (int e = threadIdx.x; e < E; e += THREADS) {
    int t, v;
    if (vfast) { v = e & (V - 1); t = e >> logV; }
    else { t = e & ((1 << logLp) - 1); v = e >> logLp; }
    const WVec vi = vinfo[v];
    if (vi.out_off < 0) continue;
    W y = s[spad(vfast ? ((t << logV) + v) : ((v << logLp) + t))];
    Tout* p = out + vi.out_off + ((int64_t)part * Lp + t) * a.out_tstride;
    if (a.beta) y = wadd(y, *p);
    *p = y;
  }
}

// ------------------------------------------------------------------ long contiguous columns
// n = C * 2^14 with plain column blocks (f32 or int8 -> int32).  CTA r of a column owns
// block r (2^14 elements, 64 KB of FP32/int32 in shared memory) and 512 threads with 32
// elements each.  Element e of the block has bits 0..13; the transform is done in three
// register rounds over bit groups {0,1,2,12,13}, {3..7} and {8..11} with two shared-memory
// exchanges in between.  The first round loads straight from HBM with one 32-byte vector
// load per block and register group (all C blocks combined with row r of H_C as they
// arrive); the last round stores straight to HBM (an aligned pair of elements per thread,
// 256 contiguous bytes per warp and instruction).  Shared-memory word of element e: bits 3-4 XOR bits 8-9 and bit 2 XOR bit 5,
// which keeps 16-byte groups intact and makes the round-A 16-byte stores and the round-B
// and round-C accesses bank-conflict free.
__device__ __forceinline__ int lswz(int e) { return e ^ (((e >> 8) & 3) << 3) ^ (((e >> 5) & 1) << 2); }

template <typename W> struct Vec4;
template <> struct Vec4<float> { typedef float4 t; };
template <> struct Vec4<int> { typedef int4 t; };
template <typename W> struct Vec2;
template <> struct Vec2<float> { typedef float2 t; };
template <> struct Vec2<int> { typedef int2 t; };

// Coherent global loads (never the read-only .nc path): with programmatic dependent launch
// the kernel is resident while the previous grid still writes its input, and a
// non-coherent load may be served before the griddepcontrol.wait that orders them.
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
// Byte i of w sign-extended to 32 bits in one byte permute: selector nibble 0 copies byte
// i, nibbles 1-3 (msb set) replicate its sign bit.
template <int I>
__device__ __forceinline__ int sext8(unsigned w) {
  constexpr unsigned sel = I | ((8u | I) << 4) | ((8u | I) << 8) | ((8u | I) << 12);
  unsigned d;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(w), "n"(sel));
  return (int)d;
}
__device__ __forceinline__ void ld8(const int8_t* p, int (&v)[8]) {
  uint2 u;
  asm volatile("ld.global.v2.u32 {%0, %1}, [%2];" : "=r"(u.x), "=r"(u.y) : "l"(p));
  v[0] = sext8<0>(u.x);
  v[1] = sext8<1>(u.x);
  v[2] = sext8<2>(u.x);
  v[3] = sext8<3>(u.x);
  v[4] = sext8<0>(u.y);
  v[5] = sext8<1>(u.y);
  v[6] = sext8<2>(u.y);
  v[7] = sext8<3>(u.y);
}
__device__ __forceinline__ float2 make_vec2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ int2 make_vec2(int a, int b) { return make_int2(a, b); }
__device__ __forceinline__ float4 make_vec4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ int4 make_vec4(int a, int b, int c, int d) { return make_int4(a, b, c, d); }

template <typename Tin, typename W, int C>
__global__ void __launch_bounds__(512, 2) fwht_long_kernel(const Tin* in, int64_t in_ld, W* out, int64_t out_ld,
                                                           int beta, int64_t ncols, int64_t pf_cols) {
  typedef typename Vec4<W>::t V4;
  constexpr int LP = 1 << 14;
  __shared__ __align__(32) W s[LP];
  const int part = (int)(blockIdx.x % C);
  const int64_t col = blockIdx.x / C;
  const int t = threadIdx.x;
  const Tin* x = in + col * in_ld + 8 * t;
  W r[32];
  pdl_launch_dependents();
  pdl_wait();

  // round A: e = c + 8 t + 4096 q, registers hold bits {0,1,2} (c) and {12,13} (q)
#pragma unroll
  for (int q = 0; q < 4; ++q) ld8(x + 4096 * q, *reinterpret_cast<W(*)[8]>(&r[8 * q]));
#pragma unroll
  for (int sb = 1; sb < C; ++sb) {
    const bool neg = __popc(sb & part) & 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      W v[8];
      ld8(x + (int64_t)sb * LP + 4096 * q, v);
#pragma unroll
      for (int c = 0; c < 8; ++c) r[8 * q + c] = neg ? r[8 * q + c] - v[c] : r[8 * q + c] + v[c];
    }
  }
  // L2 prefetch of block `part` of the column pf_cols further on (one residency wave: the CTAs
  // that will read it start about when this one's successors do), one line per thread
  if (pf_cols > 0 && col + pf_cols < ncols) {
    constexpr int LINES = LP * (int)sizeof(Tin) / 128;
    if (t < LINES) {
      const Tin* pl = in + (col + pf_cols) * in_ld + (int64_t)part * LP + t * (128 / (int)sizeof(Tin));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(pl)));
    }
  }
  wht_regs<W, 32>(r);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    *reinterpret_cast<V4*>(&s[lswz(8 * t + 4096 * q)]) = make_vec4(r[8 * q], r[8 * q + 1], r[8 * q + 2], r[8 * q + 3]);
    *reinterpret_cast<V4*>(&s[lswz(8 * t + 4 + 4096 * q)]) =
        make_vec4(r[8 * q + 4], r[8 * q + 5], r[8 * q + 6], r[8 * q + 7]);
  }
  __syncthreads();

  // round B: e = a + 8 k + 256 b with a = t & 7, b = t >> 3; registers hold bits 3..7 (k)
  {
    const int base = (t & 7) + 256 * (t >> 3);
#pragma unroll
    for (int k = 0; k < 32; ++k) r[k] = s[lswz(base + 8 * k)];
    wht_regs<W, 32>(r);
#pragma unroll
    for (int k = 0; k < 32; ++k) s[lswz(base + 8 * k)] = r[k];
  }
  __syncthreads();

  // round C: e = c + 2 l + 256 m + 4096 h with l = t & 127, h = t >> 7; registers hold bits
  // 8..11 (m) for both values of bit 0 (c, carried untransformed), so that every
  // shared-memory read and HBM write moves an aligned pair of elements
  {
    typedef typename Vec2<W>::t V2;
    const int l = t & 127, h = t >> 7;
    const int e0 = 2 * l + 4096 * h;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const V2 v = *reinterpret_cast<const V2*>(&s[lswz(e0 + 256 * m)]);
      r[m] = v.x;
      r[16 + m] = v.y;
    }
    wht_regs<W, 16>(r);
    wht_regs<W, 16>(r + 16);
    W* y = out + col * out_ld + (int64_t)part * LP + e0;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      V2* p = reinterpret_cast<V2*>(y + 256 * m);
      V2 v = make_vec2(r[m], r[16 + m]);
      if (beta) {
        const V2 o = *p;
        v = make_vec2(v.x + o.x, v.y + o.y);
      }
      *p = v;
    }
  }
}

template <typename Tin, typename W>
static fm_status fwht_long(const FwhtArgs& a, cudaStream_t st) {
  const int logC = a.logL - 14;
  const Tin* in = reinterpret_cast<const Tin*>(a.in);
  W* out = reinterpret_cast<W*>(a.out);
  const int64_t blocks = a.ncols << logC;
  if (blocks == 0) return FM_OK;
  const char* nm = "fwht_long_kernel";
  const dim3 grid((unsigned)blocks), blk(512);
  // prefetch distance: the columns resident on the GPU (two CTAs per SM, 2^logC per column),
  // one residency wave; measured on GB300 for 2^16 x 256 FP32: a quarter wave 33.7 us per
  // launch, half 33.2, one 32.1, one and a half 33.6, two 35.3, none 37.0.  a.prefetch 0 turns
  // it off
  int64_t pf = 0;
  if (a.prefetch) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      set_error("fwht_long: SM count query failed");
      return FM_ERR_CUDA;
    }
    pf = std::max<int64_t>(1, ((int64_t)nsm * 2) >> logC);
  }
  const int64_t nc = a.ncols;
  switch (logC) {
    case 0: return pdl_go(nm, fwht_long_kernel<Tin, W, 1>, grid, blk, 0, st, in, a.in_ld, out, a.out_ld, a.beta, nc, pf);
    case 1: return pdl_go(nm, fwht_long_kernel<Tin, W, 2>, grid, blk, 0, st, in, a.in_ld, out, a.out_ld, a.beta, nc, pf);
    case 2: return pdl_go(nm, fwht_long_kernel<Tin, W, 4>, grid, blk, 0, st, in, a.in_ld, out, a.out_ld, a.beta, nc, pf);
    default: break;
  }
  set_error("fwht_long: unsupported length");
  return FM_ERR_UNSUPPORTED;
}

// Plain contiguous column blocks of length 2^14..2^16 with 16-byte aligned columns.
static bool long_path_ok(const FwhtArgs& a, int in_size) {
  if (a.logL < 14 || a.logL > 16 || a.outer != 1 || a.inner != 1) return false;
  if (a.in_tstride != 1 || a.out_tstride != 1) return false;
  // 8-element (32 B for FP32, 8 B for int8) vector loads, 16-byte output words
  if (((uintptr_t)a.in % (8 * in_size)) || ((uintptr_t)a.out % 16)) return false;
  if (a.in_ld % 8 || a.out_ld % 4) return false;
  return true;
}

template <typename Tin, typename W, typename Tout, int THREADS, int EPT>
static fm_status fwht_cfg(FwhtArgs a, cudaStream_t st) {
  constexpr int E = THREADS * EPT;
  // tile: Lp = min(L, E) elements per vector, V = E / Lp vectors, C = L / Lp parts
  int logE = 0;
  while ((1 << logE) < E) ++logE;
  a.logLp = a.logL < logE ? a.logL : logE;
  a.logC = a.logL - a.logLp;
  a.logV = logE - a.logLp;
  if (a.logC > 4) { set_error("fwht: length 2^%d too long", a.logL); return FM_ERR_UNSUPPORTED; }
  const int64_t nvec = a.ncols * a.outer * a.inner;
  const int64_t tiles = (nvec + (1 << a.logV) - 1) >> a.logV;
  const int64_t blocks = tiles << a.logC;
  if (blocks > 0x7fffffffLL) { set_error("fwht: too many tiles"); return FM_ERR_UNSUPPORTED; }
  const size_t smem = fwht_vinfo_offset<W>(E) + ((size_t)1 << a.logV) * sizeof(WVec);
  auto kern = fwht_tile_kernel<Tin, W, Tout, THREADS, EPT>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned long long> attr_bytes[32];
  if (dev < 32 && attr_bytes[dev].load() < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error("fwht smem attribute: %s", cudaGetErrorString(e)); return FM_ERR_CUDA; }
    attr_bytes[dev].store(smem);
  }
  if (blocks == 0) return FM_OK;
  return pdl_go("fwht_tile_kernel", kern, dim3((unsigned)blocks), dim3(THREADS), smem, st, a);
}

fm_status fwht_launch(FwhtArgs a, fm_dtype in_dt, cudaStream_t st) {
  if (a.logL < 1) { set_error("fwht: n must be >= 2"); return FM_ERR_UNSUPPORTED; }
  if (in_dt == FM_F32 && long_path_ok(a, 4)) return fwht_long<float, float>(a, st);
  if (in_dt == FM_I8 && long_path_ok(a, 1)) return fwht_long<int8_t, int>(a, st);
  if (fwht2_ok(a)) return fwht2_launch(a, in_dt, st);
  switch (in_dt) {
    case FM_F32: return fwht_cfg<float, float, float, 512, 32>(a, st);
    case FM_C64: return fwht_cfg<float2, float2, float2, 512, 16>(a, st);
    case FM_I8: return fwht_cfg<int8_t, int, int, 512, 32>(a, st);
    case FM_I32: return fwht_cfg<int, int, int, 512, 32>(a, st);  // second pass of long int8 columns
    default: break;
  }
  set_error("fwht: dtype %d not supported", (int)in_dt);
  return FM_ERR_DTYPE;
}

}  // namespace fm
