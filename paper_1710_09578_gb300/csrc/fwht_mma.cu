// Walsh-Hadamard transform on BF16 tensor-core tiles (Hadamard modes FM_HAD_BF16 and
// FM_HAD_BF16X2).
//
// With the index bits grouped in digits of four, H_n is a product of Kronecker factors
// I (x) H_16 (x) I, one per digit, and each factor is a dense contraction: viewing the
// block as X[16][m] (the digit as the row index), the stage computes Y = H_16 X.  H_16
// has entries +-1, exact in BF16, so a warp runs the stage as mma.m16n8k16 products of
// the 16x16 matrix with 16x8 slices of X, accumulated in FP32.  When the number of bits
// is not a multiple of four the last digit overlaps the previous one and its matrix is
// H_{2^r} (x) I_{2^(4-r)}, which transforms only the r bits not done yet.
//   FM_HAD_BF16    X is rounded to BF16 (round to nearest even) before every stage;
//   FM_HAD_BF16X2  X = hi + lo with hi = bf16(x), lo = bf16(x - hi) (x - hi is exact in
//                  FP32) and the stage accumulates H hi + H lo, so each stage loses only
//                  the rounding of lo (about 2^-18 relative).
// A block of up to 2^14 elements lives in shared memory in FP32 between stages.  For
// longer columns (2^15, 2^16 = C blocks) CTA r loads the C blocks and combines them with
// row r of H_C in FP32 while loading (the top one or two index bits, a few adds per
// element), then transforms its own block on the tensor cores.
#include <cuda_bf16.h>

#include <atomic>

#include "fm_device.cuh"
#include "fm_internal.h"
#include "fwht.h"

namespace fm {

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<uint32_t*>(&p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Entry (row, col) of H_{2^r} (x) I_{2^(4-r)} on a 4-bit digit whose low `id` = 4 - r bits
// are already transformed (id = 0 gives H_16).
__device__ __forceinline__ float hdigit(int row, int col, int id) {
  const int m = (1 << id) - 1;
  if ((row & m) != (col & m)) return 0.f;
  return (__popc((row >> id) & (col >> id)) & 1) ? -1.f : 1.f;
}

template <int SPLIT>
__global__ void __launch_bounds__(512) fwht_mma_kernel(const float* in, int64_t in_ld,
                                                       float* out, int64_t out_ld, int beta,
                                                       int logLp, int nparts) {
  extern __shared__ __align__(16) float s[];
  const int Lp = 1 << logLp;
  const int part = (int)(blockIdx.x % nparts);
  const int64_t col = blockIdx.x / nparts;
  const float* x = in + col * in_ld;
  float* y = out + col * out_ld + (int64_t)part * Lp;
  pdl_launch_dependents();
  pdl_wait();
  for (int i = threadIdx.x; i < Lp; i += blockDim.x) {
    float acc = 0.f;
    for (int sb = 0; sb < nparts; ++sb) {
      const float v = x[(int64_t)sb * Lp + i];
      acc = (__popc(sb & part) & 1) ? acc - v : acc + v;
    }
    s[i] = acc;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int ncol = Lp >> 4;                   // columns of the 16 x ncol view
  for (int s0 = 0; s0 < logLp; s0 += 4) {
    const int d0 = s0 + 4 <= logLp ? s0 : logLp - 4;  // digit = bits [d0, d0 + 4)
    const int id = s0 - d0;                             // bits of the digit already done
    uint32_t A[4];
    A[0] = pack_bf16(hdigit(g, 2 * tq, id), hdigit(g, 2 * tq + 1, id));
    A[1] = pack_bf16(hdigit(g + 8, 2 * tq, id), hdigit(g + 8, 2 * tq + 1, id));
    A[2] = pack_bf16(hdigit(g, 2 * tq + 8, id), hdigit(g, 2 * tq + 9, id));
    A[3] = pack_bf16(hdigit(g + 8, 2 * tq + 8, id), hdigit(g + 8, 2 * tq + 9, id));
    const int lowm = (1 << d0) - 1;
    for (int n0 = warp * 8; n0 < ncol; n0 += nwarps * 8) {
      // B: rows k = 2tq, 2tq+1, 2tq+8, 2tq+9 of column n = n0 + g
      const int nb = n0 + g;
      const bool vb = nb < ncol;
      const int baseb = ((nb >> d0) << (d0 + 4)) | (nb & lowm);
      float xb[4] = {0.f, 0.f, 0.f, 0.f};
      if (vb) {
        xb[0] = s[baseb + ((2 * tq) << d0)];
        xb[1] = s[baseb + ((2 * tq + 1) << d0)];
        xb[2] = s[baseb + ((2 * tq + 8) << d0)];
        xb[3] = s[baseb + ((2 * tq + 9) << d0)];
      }
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      const uint32_t h0 = pack_bf16(xb[0], xb[1]), h1 = pack_bf16(xb[2], xb[3]);
      mma_bf16(d, A, h0, h1);
      if (SPLIT) {
        const __nv_bfloat162 q0 = *reinterpret_cast<const __nv_bfloat162*>(&h0);
        const __nv_bfloat162 q1 = *reinterpret_cast<const __nv_bfloat162*>(&h1);
        const uint32_t l0 = pack_bf16(xb[0] - __low2float(q0), xb[1] - __high2float(q0));
        const uint32_t l1 = pack_bf16(xb[2] - __low2float(q1), xb[3] - __high2float(q1));
        mma_bf16(d, A, l0, l1);
      }
      // D: rows g, g+8 of columns n0 + 2tq, n0 + 2tq + 1 (the warp read all of B first)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int nd = n0 + 2 * tq + c;
        if (nd < ncol) {
          const int based = ((nd >> d0) << (d0 + 4)) | (nd & lowm);
          s[based + (g << d0)] = d[c];
          s[based + ((g + 8) << d0)] = d[2 + c];
        }
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < Lp; i += blockDim.x) y[i] = beta ? y[i] + s[i] : s[i];
}

// ---------------------------------------------------------------- long columns
// n = C * 2^14 (C = 1, 2, 4), plain column blocks.  CTA r of a column loads the C blocks
// combined with row r of H_C (as the FP32 kernel does) into a 2^14-element FP32 tile in
// shared memory, then transforms it in two register rounds of eight index bits each.
// A warp holds a 16 x 16 sub-tile T (two 4-bit digits) as the A operand of
// mma.m16n8k16: one digit is transformed as T.H (two MMAs against the halves of the
// constant B = H_16), the product is rounded to BF16, transposed in registers with
// movmatrix, and the other digit is transformed the same way; the result comes out
// transposed, which only changes where it is written back.  Round 1 takes bits 0-3 and
// 4-7 of each 256-element run; round 2 takes bits 8-11 and the digit {0,1,12,13} whose
// matrix is I_4 (x) H_4 (bits 0, 1 ride along untransformed).  Shared-memory words are
// swizzled (bits 2-4 XOR higher bits) so the fragment reads, the transposed write-backs
// and the linear 16-byte reads for the output are all free of bank conflicts.

// word of element e in the swizzled 2^14 tile (bits 0-1 unchanged: pairs and quads of
// consecutive elements stay contiguous)
__device__ __forceinline__ int tsw(int e) {
  const int x = ((((e >> 8) ^ (e >> 10)) & 1) << 2) | ((((e >> 9) ^ (e >> 5)) & 1) << 3) |
                ((((e >> 12) ^ (e >> 6)) & 1) << 4);
  return e ^ x;
}

__device__ __forceinline__ uint32_t movtrans(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

__device__ __forceinline__ float bf16_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }

// B fragments (two 16 x 8 halves) of the 16 x 16 digit matrix hdigit(., ., id)
struct DigitB {
  uint32_t lo0, lo1, hi0, hi1;
  __device__ __forceinline__ DigitB(int id, int g, int tq) {
    lo0 = pack_bf16(hdigit(2 * tq, g, id), hdigit(2 * tq + 1, g, id));
    lo1 = pack_bf16(hdigit(2 * tq + 8, g, id), hdigit(2 * tq + 9, g, id));
    hi0 = pack_bf16(hdigit(2 * tq, g + 8, id), hdigit(2 * tq + 1, g + 8, id));
    hi1 = pack_bf16(hdigit(2 * tq + 8, g + 8, id), hdigit(2 * tq + 9, g + 8, id));
  }
};

// y (A-fragment order: (g, 2tq..), (g+8, 2tq..), (g, 2tq+8..), (g+8, 2tq+8..)) <- x . M
// for the 16 x 16 fragment x held as FP32 pairs; SPLIT adds the product of the BF16
// residual x - bf16(x).
template <int SPLIT>
__device__ __forceinline__ void frag_mul(float (&y)[8], const float (&x)[8], const DigitB& B) {
  uint32_t a[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = pack_bf16(x[2 * i], x[2 * i + 1]);
    if (SPLIT) l[i] = pack_bf16(x[2 * i] - bf16_lo(a[i]), x[2 * i + 1] - bf16_hi(a[i]));
  }
  float dl[4] = {0.f, 0.f, 0.f, 0.f}, dh[4] = {0.f, 0.f, 0.f, 0.f};
  mma_bf16(dl, a, B.lo0, B.lo1);
  mma_bf16(dh, a, B.hi0, B.hi1);
  if (SPLIT) {
    mma_bf16(dl, l, B.lo0, B.lo1);
    mma_bf16(dh, l, B.hi0, B.hi1);
  }
  y[0] = dl[0]; y[1] = dl[1]; y[2] = dl[2]; y[3] = dl[3];
  y[4] = dh[0]; y[5] = dh[1]; y[6] = dh[2]; y[7] = dh[3];
}

// z <- (M2 . (x . M1)^T)^T computed as (x M1)^T M2: both digits of the sub-tile; z comes
// out in A-fragment order of the TRANSPOSED tile.
template <int SPLIT>
__device__ __forceinline__ void frag_two_digits(float (&z)[8], const float (&x)[8], const DigitB& B1,
                                                const DigitB& B2) {
  float y[8];
  frag_mul<SPLIT>(y, x, B1);
  // transpose: blocks (0,0), (1,0), (0,1), (1,1) of the 16 x 16 tile are fragment words
  // 0, 1, 2, 3; the transposed tile takes words 0, 2, 1, 3, each transposed
  uint32_t h[4], l[4], th[4], tl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = pack_bf16(y[2 * i], y[2 * i + 1]);
    if (SPLIT) l[i] = pack_bf16(y[2 * i] - bf16_lo(h[i]), y[2 * i + 1] - bf16_hi(h[i]));
  }
  th[0] = movtrans(h[0]); th[1] = movtrans(h[2]); th[2] = movtrans(h[1]); th[3] = movtrans(h[3]);
  if (SPLIT) {
    tl[0] = movtrans(l[0]); tl[1] = movtrans(l[2]); tl[2] = movtrans(l[1]); tl[3] = movtrans(l[3]);
  }
  float dl[4] = {0.f, 0.f, 0.f, 0.f}, dh[4] = {0.f, 0.f, 0.f, 0.f};
  mma_bf16(dl, th, B2.lo0, B2.lo1);
  mma_bf16(dh, th, B2.hi0, B2.hi1);
  if (SPLIT) {
    mma_bf16(dl, tl, B2.lo0, B2.lo1);
    mma_bf16(dh, tl, B2.hi0, B2.hi1);
  }
  z[0] = dl[0]; z[1] = dl[1]; z[2] = dl[2]; z[3] = dl[3];
  z[4] = dh[0]; z[5] = dh[1]; z[6] = dh[2]; z[7] = dh[3];
}

// threads per CTA and resident CTAs per SM of the long-column kernel
// Coherent 16-byte global load (not the read-only .nc path, which may be served before the
// griddepcontrol.wait that orders this kernel after the grid writing its input).
__device__ __forceinline__ float4 ld4(const float* p) {
  float4 r;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
  return r;
}

constexpr int kTcThreads = 512, kTcMinBlocks = 2;

template <int SPLIT, int C>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks)
    fwht_tc_kernel(const float* in, int64_t in_ld, float* out, int64_t out_ld, int beta) {
  constexpr int LP = 1 << 14, NT = kTcThreads, NW = NT / 32, NCH = LP / 4 / NT;
  extern __shared__ __align__(16) float s[];
  const int part = (int)(blockIdx.x % C);
  const int64_t col = blockIdx.x / C;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const float* x = in + col * in_ld;
  pdl_launch_dependents();
  pdl_wait();

  // the C blocks combined with row `part` of H_C, 16 bytes per thread and load
#pragma unroll 1
  for (int i0 = 0; i0 < NCH; i0 += 2) {
    float4 v[2][C];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int sb = 0; sb < C; ++sb)
        v[i][sb] = ld4(x + (int64_t)sb * LP + 4 * (t + NT * (i0 + i)));
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4 acc = v[i][0];
#pragma unroll
      for (int sb = 1; sb < C; ++sb) {
        const float sg = (__popc(sb & part) & 1) ? -1.f : 1.f;
        acc.x += sg * v[i][sb].x;
        acc.y += sg * v[i][sb].y;
        acc.z += sg * v[i][sb].z;
        acc.w += sg * v[i][sb].w;
      }
      *reinterpret_cast<float4*>(&s[tsw(4 * (t + NT * (i0 + i)))]) = acc;
    }
  }
  __syncthreads();

  const DigitB H16(0, g, tq), H4I4(2, g, tq);
  // The swizzle XORs bits 2-4 of an element index with bits 5, 6, 8, 9, 10, 12; split into
  // the part from the sub-tile index (once per sub-tile) and the part from the lane (once
  // per thread), every fragment address below is one base plus a constant.
  // round 1: sub-tile w = elements w*256 + 16 row + col (row: bits 4-7, col: bits 0-3)
  const int xr1 = (16 * g + 2 * tq) ^ ((((g >> 1) & 1) << 3) | (((g >> 2) & 1) << 4));
  const int xw1 = (32 * tq + g) ^ (((tq & 1) << 3) | (((tq >> 1) & 1) << 4));
#pragma unroll 1
  for (int w = warp; w < 64; w += NW) {
    const int b = w << 8;
    const int mb = (((w ^ (w >> 2)) & 1) << 2) | (((w >> 1) & 1) << 3) | (((w >> 4) & 1) << 4);
    const int X = xr1 ^ mb, Y = xw1 ^ mb;
    float xr[8], z[8];
    const float2 p0 = *reinterpret_cast<const float2*>(&s[b | X]);
    const float2 p1 = *reinterpret_cast<const float2*>(&s[b | (X ^ 128)]);
    const float2 p2 = *reinterpret_cast<const float2*>(&s[b | (X ^ 8)]);
    const float2 p3 = *reinterpret_cast<const float2*>(&s[b | (X ^ 136)]);
    xr[0] = p0.x; xr[1] = p0.y; xr[2] = p1.x; xr[3] = p1.y;
    xr[4] = p2.x; xr[5] = p2.y; xr[6] = p3.x; xr[7] = p3.y;
    frag_two_digits<SPLIT>(z, xr, H16, H16);
    // z = Z^T: Z^T rows g, g+8 are Z cols (bits 0-3), Z^T cols 2tq.. are Z rows (bits 4-7)
    s[b | Y] = z[0];
    s[b | (Y ^ 16)] = z[1];
    s[b | (Y ^ 8)] = z[2];
    s[b | (Y ^ 24)] = z[3];
    s[b | (Y ^ 128)] = z[4];
    s[b | (Y ^ 144)] = z[5];
    s[b | (Y ^ 136)] = z[6];
    s[b | (Y ^ 152)] = z[7];
  }
  __syncthreads();

  // round 2: sub-tile u (bits 2-7) = T[r][c], r = bits 8-11, c = (bit 0, bit 1, bit 12,
  // bit 13); first c with I_4 (x) H_4 (bits 0, 1 untouched), then r with H_16
  const int ar2 = (2 * (tq & 1)) | ((tq >> 1) << 12) | (g << 8);
  const int mr2 = (((g ^ (g >> 2)) & 1) << 2) | (((g >> 1) & 1) << 3) | (((tq >> 1) & 1) << 4);
  const int aw2 = (g & 3) | ((g >> 2) << 12) | ((2 * tq) << 8);
  const int mw2 = (((tq >> 1) & 1) << 2) | ((tq & 1) << 3) | (((g >> 2) & 1) << 4);
#pragma unroll 1
  for (int u = warp; u < 64; u += NW) {
    const int U = (u << 2) ^ ((((u >> 3) & 1) << 3) | (((u >> 4) & 1) << 4));
    const int A = ar2 | (U ^ mr2);
    float xr[8], z[8];
    const float2 p0 = *reinterpret_cast<const float2*>(&s[A]);
    const float2 p1 = *reinterpret_cast<const float2*>(&s[A + 2048]);
    const float2 p2 = *reinterpret_cast<const float2*>(&s[A + 8192]);
    const float2 p3 = *reinterpret_cast<const float2*>(&s[A + 10240]);
    xr[0] = p0.x; xr[1] = p0.y; xr[2] = p1.x; xr[3] = p1.y;
    xr[4] = p2.x; xr[5] = p2.y; xr[6] = p3.x; xr[7] = p3.y;
    frag_two_digits<SPLIT>(z, xr, H4I4, H16);
    // z = Z^T: rows g, g+8 are c values, cols 2tq.. are r values
    const int B0 = aw2 | (U ^ mw2), B1 = (aw2 + 256) | (U ^ mw2 ^ 4);
    s[B0] = z[0];
    s[B1] = z[1];
    s[B0 + 8192] = z[2];
    s[B1 + 8192] = z[3];
    s[B0 + 2048] = z[4];
    s[B1 + 2048] = z[5];
    s[B0 + 10240] = z[6];
    s[B1 + 10240] = z[7];
  }
  __syncthreads();

  float* y = out + col * out_ld + (int64_t)part * LP;
#pragma unroll 4
  for (int i = 0; i < NCH; ++i) {
    const int e = 4 * (t + NT * i);
    float4 v = *reinterpret_cast<const float4*>(&s[tsw(e)]);
    float4* p = reinterpret_cast<float4*>(y + e);
    if (beta) {
      const float4 o = *p;
      v.x += o.x;
      v.y += o.y;
      v.z += o.z;
      v.w += o.w;
    }
    *p = v;
  }
}

template <int SPLIT>
static fm_status fwht_tc_launch(const FwhtArgs& a, cudaStream_t st) {
  const int C = 1 << (a.logL - 14);
  const float* in = reinterpret_cast<const float*>(a.in);
  float* out = reinterpret_cast<float*>(a.out);
  const size_t smem = sizeof(float) << 14;
  auto kern = C == 1 ? fwht_tc_kernel<SPLIT, 1> : (C == 2 ? fwht_tc_kernel<SPLIT, 2> : fwht_tc_kernel<SPLIT, 4>);
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned> attr_set[3];
  const int ci = C == 1 ? 0 : (C == 2 ? 1 : 2);
  if (dev < 32 && !(attr_set[ci].load() & (1u << dev))) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      set_error("fwht_tc smem attribute");
      return FM_ERR_CUDA;
    }
    attr_set[ci].fetch_or(1u << dev);
  }
  return pdl_go("fwht_tc_kernel", kern, dim3((unsigned)(a.ncols * C)), dim3(kTcThreads), smem, st, in, a.in_ld, out,
                a.out_ld, a.beta);
}

fm_status fwht_mma_launch(FwhtArgs a, int split, cudaStream_t st) {
  if (a.logL < 4 || a.logL > 16) { set_error("BF16 Hadamard needs 4 <= log2n <= 16"); return FM_ERR_UNSUPPORTED; }
  if (a.outer != 1 || a.inner != 1 || a.in_tstride != 1 || a.out_tstride != 1) {
    set_error("BF16 Hadamard applies to plain column blocks only (not along a Kron axis)");
    return FM_ERR_UNSUPPORTED;
  }
  if (a.ncols == 0) return FM_OK;
  // long columns with 16-byte aligned blocks: the two-round register kernel
  if (a.logL >= 14 && !((uintptr_t)a.in % 16) && !((uintptr_t)a.out % 16) && !(a.in_ld % 4) && !(a.out_ld % 4))
    return split ? fwht_tc_launch<1>(a, st) : fwht_tc_launch<0>(a, st);
  const int logLp = a.logL < 14 ? a.logL : 14;
  const int C = 1 << (a.logL - logLp);
  const size_t smem = sizeof(float) << logLp;
  auto k0 = fwht_mma_kernel<0>;
  auto k1 = fwht_mma_kernel<1>;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::atomic<unsigned> attr_set{0};
  if (dev < 32 && !(attr_set.load() & (1u << dev))) {
    cudaError_t e0 = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    cudaError_t e1 = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    if (e0 != cudaSuccess || e1 != cudaSuccess) { set_error("fwht_mma smem attribute"); return FM_ERR_CUDA; }
    attr_set.fetch_or(1u << dev);
  }
  const float* in = reinterpret_cast<const float*>(a.in);
  float* out = reinterpret_cast<float*>(a.out);
  auto kern = split ? k1 : k0;
  return pdl_go("fwht_mma_kernel", kern, dim3((unsigned)(a.ncols * C)), dim3(512), smem, st, in, a.in_ld, out,
                a.out_ld, a.beta, logLp, C);
}

}  // namespace fm
