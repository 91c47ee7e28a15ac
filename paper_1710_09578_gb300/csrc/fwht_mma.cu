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
__global__ void __launch_bounds__(512) fwht_mma_kernel(const float* __restrict__ in, int64_t in_ld,
                                                       float* __restrict__ out, int64_t out_ld, int beta,
                                                       int logLp, int nparts) {
  extern __shared__ __align__(16) float s[];
  const int Lp = 1 << logLp;
  const int part = (int)(blockIdx.x % nparts);
  const int64_t col = blockIdx.x / nparts;
  const float* x = in + col * in_ld;
  float* y = out + col * out_ld + (int64_t)part * Lp;
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

fm_status fwht_mma_launch(FwhtArgs a, int split, cudaStream_t st) {
  if (a.logL < 4 || a.logL > 16) { set_error("BF16 Hadamard needs 4 <= log2n <= 16"); return FM_ERR_UNSUPPORTED; }
  if (a.outer != 1 || a.inner != 1 || a.in_tstride != 1 || a.out_tstride != 1) {
    set_error("BF16 Hadamard applies to plain column blocks only (not along a Kron axis)");
    return FM_ERR_UNSUPPORTED;
  }
  if (a.ncols == 0) return FM_OK;
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
  kern<<<(unsigned)(a.ncols * C), 512, smem, st>>>(in, a.in_ld, out, a.out_ld, a.beta, logLp, C);
  return after_launch("fwht_mma_kernel");
}

}  // namespace fm
