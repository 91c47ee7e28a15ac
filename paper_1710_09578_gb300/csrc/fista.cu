// Batched FISTA for l1-regularised least squares, min 1/2 ||A x - b||^2 + lambda ||x||_1
// (Eq. (8) with tau = 2 lambda), with A_i = P_i T_i (row selection of a real Toeplitz matrix)
// for thousands of independent instances in ONE persistent launch.
//
// The recovery loop of the paper (Sec. 3: ISTA, and the accelerated variant it uses for its
// reconstructions) spends its time in phi_A and beta_A; here both run in shared memory:
// T y is the non-circular convolution of y with t, evaluated through the circulant
// embedding of length L = 2n (Sec. 2.1.1).  y is real, so the length-L transform is done
// as one complex FFT of length n on z[k] = w[2k] + i w[2k+1] (w = [y; 0]): a post-step
// turns Z = FFT_n(z) into the half spectrum W[k] = E[k] + exp(-2 pi i k / L) O[k]
// (E, O the spectra of the even and odd samples), multiplies by the embedding spectrum,
// and a pre-step folds the product back into the spectrum of [v_even + i v_odd] for the
// inverse FFT of length n.  Each product with T or T^T therefore costs two complex FFTs of
// length n on a 2^14-element tile, i.e. up to 128 KB of shared memory per CTA.
//
// Work list: instances sorted by size, grouped so that a group of V = 2^14 / n instances of
// the same n fills one tile and runs in lock step (the FISTA momentum sequence t_k does not
// depend on the data, only L and lambda are per instance).  Each CTA takes the next group
// with an atomic counter (no waiting on other CTAs) and keeps it until all its steps are
// done: lambda = lambda_rel ||A^T b||_inf, L = min(safety ||A v_P||^2, max|c_hat|^2) after P
// power iterations from v_0 = ones / sqrt(n), K FISTA steps from x_0 = y_1 = 0, t_1 = 1, and
// the final objective.  x_k lives in the caller's x buffer, y_k in the batch's scratch
// (both small enough to stay in L2 while a group runs); norms, the Rayleigh quotient and the
// objective are accumulated in FP64, everything else is FP32.
#include <algorithm>
#include <vector>

#include "exec.h"
#include "fft2.cuh"
#include "pointwise.h"

namespace fm {

struct FInst {
  const float2* spec;   // FFT_L(c) / L of the circulant embedding (L = 2n entries)
  const int32_t* idx;   // m selected rows
  const int32_t* inv;   // n entries: r if row r selects position j, else -1
  int64_t b_off;        // offset of b_i in the packed b
  int64_t x_off;        // offset of x_i in the packed x (and of y_i in the scratch)
  int n, m, logn, pad;
  double cap;           // max_k |FFT_L(c)_k|^2
};

struct FGroup {
  int logn, count, first, pad;
};

struct FistaArgs {
  const FInst* inst;
  const int32_t* order;    // instance indices sorted by group
  const FGroup* groups;
  int ngroups;
  int single_group;        // >= 0: only this group (one launch per instance)
  const float* b;          // packed b (instance i at inst[i].b_off) ...
  float* x;                // ... and packed x (at inst[i].x_off), or
  const float* const* bp;  // per-instance pointers (device arrays of `count` entries)
  float* const* xp;
  float* y;                // FISTA momentum state y_{k+1}, packed like x
  float* pw;               // power-iteration iterate, packed like x (may equal y)
  const float2* tw;        // pass-twiddle tables of the FFT passes
  const float2* tw2;       // W_{2^15}^m, real-FFT pre/post steps
  int iters, power_iters;
  double lambda_rel, safety;
  int accel;
  int warm;                // 1: resume from x_k, y_{k+1} with L, lambda read from rep_L, rep_lambda
  int k0;                  // warm: steps already taken
  double* rep_L;
  double* rep_lambda;
  double* rep_obj;
  int32_t* rep_status;
  int* counter;
};

constexpr int kFThreads = 512, kFEpt = 32, kFE = kFThreads * kFEpt;  // 2^14 complex per tile
constexpr int kFMaxV = 64;                                                // n >= 256

struct VState {
  const float2* spec;
  const int32_t* idx;
  const int32_t* inv;
  const float* b;       // this instance's measurements
  float* x;             // its solution x_k
  float* y;             // its momentum state y_{k+1}
  float* pw;            // its power-iteration iterate
  int m, valid, inst, pad;
  float invL, thr;
  double cap, lam, L, acc;
  unsigned amax;
};

// Tile geometry of a group with transform length 2^LOGL: V = 2^(14 - LOGL) vectors.
template <int LOGL>
struct FGeo {
  static constexpr int LOGV = 14 - LOGL, V = 1 << LOGV, NC = 1 << LOGL;
  // elements of a vector contiguous in shared memory: the element-wise steps (spectral
  // step, row mask, update) walk consecutive elements of one vector, and in the transform
  // passes a warp's lanes take consecutive butterflies of one vector (of two for the radix-16
  // passes of n = 256, which have 16 butterflies per vector)
  static constexpr bool VF = false;
};

// x and y are rewritten by the kernel itself: read and write them through L2 (.cg), never
// through the read-only path.  The spectra, row maps, measurements b and twiddle tables are
// written before the launch and only read by it: those go through the read-only path (__ldg),
// which also leaves the compiler free to issue them early.
__device__ __forceinline__ float2 ld_state(const float* p) { return __ldcg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st_state(float* p, float2 v) { __stcg(reinterpret_cast<float2*>(p), v); }

// word of element t of vector v in the tile (the layout the transform passes use)
template <int LOGL>
__device__ __forceinline__ int zword(int t, int v) {
  constexpr bool VF = FGeo<LOGL>::VF;
  constexpr int LOGV = FGeo<LOGL>::LOGV;
  return sp2<VF, LOGL, LOGV, layout_of<kFEpt, LOGL, LOGV, VF>()>(t, v);
}
template <int LOGL>
__device__ __forceinline__ float2* zaddr(float2* s, int t, int v) {
  return &s[zword<LOGL>(t, v)];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums over the elements of each vector, in a fixed order (runs are bit-reproducible).  The
// element loops of a tile visit q = threadIdx.x + i * kFThreads over V * Nc = 2^14 elements, so
// the 32 lanes of a warp always hold 32 consecutive elements of one vector (Nc >= 256):
// vec_part stores the warp's sum at slot q / 32, vec_finish adds a vector's slots in order.
__device__ __forceinline__ void vec_part(double* part, int q, double val) {
  val = warp_sum(val);
  if ((threadIdx.x & 31) == 0) part[q >> 5] = val;
}
template <int LOGL>
__device__ __forceinline__ void vec_finish(VState* vs, const double* part) {
  constexpr int V = FGeo<LOGL>::V, W = (1 << LOGL) >> 5;
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += kFThreads) {
    double acc = 0.0;
    for (int w = 0; w < W; ++w) acc += part[v * W + w];
    vs[v].acc = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ void vec_max(VState* vs, int v, float val) {
  atomicMax(&vs[v].amax, __float_as_uint(fabsf(val)));
}

// Natural-order FFT of every vector of the tile, in place in shared memory (passes of the
// compile-time engine).  Entry and exit: synchronised, natural order in shared memory.
template <int LOGL>
__device__ __forceinline__ void tile_fft(float2* s, int dir, const float2* tw) {
  constexpr int LOGV = FGeo<LOGL>::LOGV;
  constexpr bool VF = FGeo<LOGL>::VF;
  using S = Sched<LOGL, ept_lmax<kFEpt>()>;
  constexpr int LR0 = S::lr(0), LRL = S::lr(S::NR - 1);
  float2 r[kFEpt];
  p2_read<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LR0>(r, s);
  p2_run<float2, VF, kFThreads, kFEpt, LOGL, LOGV, 0, false>(r, s, dir, tw);
  __syncthreads();
  p2_write<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LRL, LOGL - LRL>(r, s);
  __syncthreads();
}

// tile_fft(-1) whose first pass reads the residual u = P^T (P T y - b) instead of T y
// (the MODE_RESID row mask of mask_rows applied to each element as it is read).
template <int LOGL>
__device__ __forceinline__ void tile_fft_resid(float2* s, const VState* vs, const float2* tw) {
  constexpr int LOGV = FGeo<LOGL>::LOGV, Nc = 1 << LOGL;
  constexpr bool VF = FGeo<LOGL>::VF;
  using S = Sched<LOGL, ept_lmax<kFEpt>()>;
  constexpr int LR0 = S::lr(0), LRL = S::lr(S::NR - 1), R = 1 << LR0, M = 1 << (LOGL - LR0);
  float2 r[kFEpt];
  p2_read<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LR0>(r, s);
#pragma unroll
  for (int q = 0; q < kFEpt / R; ++q) {
    int j, v;
    bfly2<VF, kFThreads, LOGL, LOGV, LR0>(q, j, v);
    const bool valid = vs[v].valid;
    const int32_t* inv = vs[v].inv;
    const float* bb = vs[v].b;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int kk = j + k * M;
      float2 u = make_float2(0.f, 0.f);
      if (valid && kk < (Nc >> 1)) {
        const float2 z = r[q * R + k];
        const int2 rr = __ldg(reinterpret_cast<const int2*>(inv + 2 * kk));
        if (rr.x >= 0) u.x = z.x - __ldg(bb + rr.x);
        if (rr.y >= 0) u.y = z.y - __ldg(bb + rr.y);
      }
      r[q * R + k] = u;
    }
  }
  p2_run<float2, VF, kFThreads, kFEpt, LOGL, LOGV, 0, false>(r, s, -1, tw);
  __syncthreads();
  p2_write<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LRL, LOGL - LRL>(r, s);
  __syncthreads();
}

// tile_fft(+1) whose last pass, holding the gradient g = T^T u (unpacked pairs) in
// registers, takes the FISTA step there: x_k = soft(y_k - g / L, lambda / L) and
// y_{k+1} = x_k + beta (x_k - x_{k-1}) go to x and y, and pack(y_{k+1}) is what the pass
// writes back to the tile for the next step.
template <int LOGL>
__device__ __forceinline__ void tile_ifft_update(float2* s, const VState* vs, float beta, const float2* tw) {
  constexpr int LOGV = FGeo<LOGL>::LOGV, Nc = 1 << LOGL;
  constexpr bool VF = FGeo<LOGL>::VF;
  using S = Sched<LOGL, ept_lmax<kFEpt>()>;
  constexpr int LR0 = S::lr(0), LRL = S::lr(S::NR - 1), R = 1 << LRL, M = 1 << (LOGL - LRL);
  float2 r[kFEpt];
  p2_read<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LR0>(r, s);
  p2_run<float2, VF, kFThreads, kFEpt, LOGL, LOGV, 0, false>(r, s, +1, tw);
#pragma unroll
  for (int q = 0; q < kFEpt / R; ++q) {
    int j, v;
    bfly2<VF, kFThreads, LOGL, LOGV, LRL>(q, j, v);
    const bool valid = vs[v].valid;
    float* x = vs[v].x;
    float* y = vs[v].y;
    const float invL = vs[v].invL, thr = vs[v].thr;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int kk = j + k * M;
      float2 ny = make_float2(0.f, 0.f);
      if (valid && kk < (Nc >> 1)) {
        const float2 g = r[q * R + k];
        const int o = 2 * kk;
        const float2 yv = ld_state(y + o);
        const float2 xv = ld_state(x + o);
        const float z0 = yv.x - g.x * invL, z1 = yv.y - g.y * invL;
        const float m0 = fabsf(z0) - thr, m1 = fabsf(z1) - thr;
        const float x0 = m0 > 0.f ? copysignf(m0, z0) : 0.f;
        const float x1 = m1 > 0.f ? copysignf(m1, z1) : 0.f;
        ny = make_float2(x0 + beta * (x0 - xv.x), x1 + beta * (x1 - xv.y));
        st_state(x + o, make_float2(x0, x1));
        st_state(y + o, ny);
      }
      r[q * R + k] = ny;
    }
  }
  __syncthreads();
  p2_write<float2, VF, kFThreads, kFEpt, LOGL, LOGV, LRL, LOGL - LRL>(r, s);
  __syncthreads();
}

// Z <- pre-step( spectrum x post-step(Z) ) for every vector: see the file comment.
template <int LOGL>
__device__ void tile_spectral(float2* s, VState* vs, int adjoint, const float2* tw2) {
  constexpr int Nc = 1 << LOGL, half = Nc >> 1, V = FGeo<LOGL>::V;
  constexpr int tsh = 14 - LOGL;  // index scale into the W_{2^15} table for exp(-2 pi i k / (2 Nc))
#pragma unroll 2
  for (int q = threadIdx.x; q < V * half; q += kFThreads) {
    const int v = q >> (LOGL - 1), k = q & (half - 1);
    if (!vs[v].valid) continue;
    const int kp = Nc - k;
    float2* pk = zaddr<LOGL>(s, k, v);
    float2* pm = zaddr<LOGL>(s, kp & (Nc - 1), v);
    const float2 Zk = *pk, Zm = *pm;
    // E = (Zk + conj Zm)/2, O = (Zk - conj Zm)/(2i)
    const float2 E = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 O = make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
    // W_{2Nc}^(Nc - k) = -conj(W_{2Nc}^k): one table read for the pair
    const float2 wk = __ldg(tw2 + (k << tsh)), wkp = make_float2(-wk.x, wk.y);
    const float2 Wk = cadd(E, cmul(wk, O));
    const float2 Wkp = cadd(cconj(E), cmul(wkp, cconj(O)));
    float2 sk = __ldg(vs[v].spec + k), skp = __ldg(vs[v].spec + kp);
    if (adjoint) { sk = cconj(sk); skp = cconj(skp); }
    const float2 Vk = cscale(cmul(sk, Wk), 2.f), Vkp = cscale(cmul(skp, Wkp), 2.f);
    // Z'[k] = (V_k + conj V_kp)/2 + i exp(+2 pi i k / L) (V_k - conj V_kp)/2
    const float2 A1 = cscale(cadd(Vk, cconj(Vkp)), 0.5f), B1 = cscale(csub(Vk, cconj(Vkp)), 0.5f);
    *pk = cadd(A1, cmul_i(cmul(cconj(wk), B1), +1));
    if (k > 0) {
      const float2 A2 = cscale(cadd(Vkp, cconj(Vk)), 0.5f), B2 = cscale(csub(Vkp, cconj(Vk)), 0.5f);
      *pm = cadd(A2, cmul_i(cmul(cconj(wkp), B2), +1));
    }
  }
  // k = Nc / 2 pairs with itself: Z' = conj(c') Z with c' = 2 spec (conjugated for T^T)
  for (int v = threadIdx.x; v < V; v += kFThreads) {
    if (!vs[v].valid) continue;
    float2* p = zaddr<LOGL>(s, half, v);
    float2 c = cscale(__ldg(vs[v].spec + half), 2.f);
    if (adjoint) c = cconj(c);
    *p = cmul(cconj(c), *p);
  }
}

template <int LOGL>
__device__ __forceinline__ float unpack(const float2* s, int m, int v) {
  const float2 z = s[zword<LOGL>(m >> 1, v)];
  return (m & 1) ? z.y : z.x;
}

// Z <- pack([w; 0]) where w is the length-n real vector (vs[v].*src) of each vector
template <int LOGL>
__device__ void pack_from(float2* s, VState* vs, float* VState::*src) {
  constexpr int Nc = 1 << LOGL, V = FGeo<LOGL>::V;
  for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
    const int v = q >> LOGL, k = q & (Nc - 1);
    float2 z = make_float2(0.f, 0.f);
    if (vs[v].valid && k < (Nc >> 1)) z = ld_state(vs[v].*src + 2 * k);
    *zaddr<LOGL>(s, k, v) = z;
  }
}

// tile <- T w (adjoint: T^T w) for the packed w in the tile
template <int LOGL>
__device__ void apply_T(float2* s, VState* vs, int adjoint, const float2* tw, const float2* tw2) {
  __syncthreads();
  tile_fft<LOGL>(s, -1, tw);
  tile_spectral<LOGL>(s, vs, adjoint, tw2);
  __syncthreads();
  tile_fft<LOGL>(s, +1, tw);
}

// In place on the tile, which holds T w unpacked as pairs (w[2k], w[2k+1]) at position k:
// u = P^T (P T w - b) (MODE_RESID), u = P^T P T w (MODE_MASK) or u = P^T b (MODE_B), packed
// the same way for the next transform, zeros in the upper half; with sumsq the squares of
// the selected entries are added into vs[v].acc.
enum { MODE_MASK = 0, MODE_RESID = 1, MODE_B = 2 };
template <int LOGL, int MODE>
__device__ void mask_rows(float2* s, VState* vs, double* part, bool sumsq) {
  constexpr int Nc = 1 << LOGL, V = FGeo<LOGL>::V;
  for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
    const int v = q >> LOGL, k = q & (Nc - 1);
    float2* p = zaddr<LOGL>(s, k, v);
    float2 u = make_float2(0.f, 0.f);
    double ss = 0.0;
    if (vs[v].valid && k < (Nc >> 1)) {
      const float2 z = MODE == MODE_B ? make_float2(0.f, 0.f) : *p;
      const int2 r = __ldg(reinterpret_cast<const int2*>(vs[v].inv + 2 * k));
      const float* bb = vs[v].b;
      if (r.x >= 0) u.x = MODE == MODE_B ? __ldg(bb + r.x) : (MODE == MODE_RESID ? z.x - __ldg(bb + r.x) : z.x);
      if (r.y >= 0) u.y = MODE == MODE_B ? __ldg(bb + r.y) : (MODE == MODE_RESID ? z.y - __ldg(bb + r.y) : z.y);
      ss = (double)u.x * (double)u.x + (double)u.y * (double)u.y;
    }
    *p = u;
    if (sumsq) vec_part(part, q, ss);
  }
}

// t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, one compiled copy for every caller, so that a run
// resumed after k0 steps rebuilds exactly the t a continuous run would hold.
__device__ __noinline__ double fista_t_next(double t) { return 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)); }

// Every step of one group: lambda, L, K FISTA steps and the objective.  A warm start skips
// lambda and L (read back from the report of the run it resumes) and the zero start.
template <int LOGL>
__device__ void fista_group(const FistaArgs& a, const FGroup& G, float2* s, VState* vs, double* part, double* s_t) {
  constexpr int Nc = 1 << LOGL, V = FGeo<LOGL>::V;
  for (int v = threadIdx.x; v < V; v += kFThreads) {
    VState w = {};
    w.valid = v < G.count;
    if (w.valid) {
      const int ii = a.order[G.first + v];
      const FInst in = a.inst[ii];
      w.spec = in.spec;
      w.idx = in.idx;
      w.inv = in.inv;
      w.b = a.bp ? a.bp[ii] : a.b + in.b_off;
      w.x = a.xp ? a.xp[ii] : a.x + in.x_off;
      w.y = a.y + in.x_off;
      w.pw = a.pw + in.x_off;
      w.m = in.m;
      w.cap = in.cap;
      w.inst = ii;
      if (a.warm) {
        w.lam = a.rep_lambda[ii];
        w.L = a.rep_L[ii];
      }
    }
    vs[v] = w;
  }
  __syncthreads();

  if (!a.warm) {
    // ---- lambda = lambda_rel * ||A^T b||_inf
    mask_rows<LOGL, MODE_B>(s, vs, part, false);
    apply_T<LOGL>(s, vs, 1, a.tw, a.tw2);
    for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
      const int v = q >> LOGL;
      if (vs[v].valid) vec_max(vs, v, unpack<LOGL>(s, q & (Nc - 1), v));
    }
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += kFThreads) vs[v].lam = a.lambda_rel * (double)__uint_as_float(vs[v].amax);

    // ---- power iteration on A^T A from ones / sqrt(n), the iterate kept in pw
    {
      const float v0 = rsqrtf((float)Nc);
      for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
        const int v = q >> LOGL;
        if (vs[v].valid) __stcg(vs[v].pw + (q & (Nc - 1)), v0);
      }
    }
    for (int it = 0; it < a.power_iters; ++it) {
      __syncthreads();
      pack_from<LOGL>(s, vs, &VState::pw);
      apply_T<LOGL>(s, vs, 0, a.tw, a.tw2);
      mask_rows<LOGL, MODE_MASK>(s, vs, part, false);
      apply_T<LOGL>(s, vs, 1, a.tw, a.tw2);
      __syncthreads();
      for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
        const int v = q >> LOGL;
        const float w = unpack<LOGL>(s, q & (Nc - 1), v);
        vec_part(part, q, (double)w * (double)w);
      }
      vec_finish<LOGL>(vs, part);
      for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
        const int v = q >> LOGL;
        if (vs[v].valid) {
          const double nrm = sqrt(vs[v].acc);
          const float w = unpack<LOGL>(s, q & (Nc - 1), v);
          __stcg(vs[v].pw + (q & (Nc - 1)), nrm > 0.0 ? (float)((double)w / nrm) : 0.f);
        }
      }
    }
    // lam_hat = ||A v||^2, L = min(safety * lam_hat, cap)
    __syncthreads();
    pack_from<LOGL>(s, vs, &VState::pw);
    apply_T<LOGL>(s, vs, 0, a.tw, a.tw2);
    mask_rows<LOGL, MODE_MASK>(s, vs, part, true);
    vec_finish<LOGL>(vs, part);
    for (int v = threadIdx.x; v < V; v += kFThreads) {
      double L = a.safety * vs[v].acc;
      if (vs[v].cap < L) L = vs[v].cap;
      vs[v].L = L;
    }
  }
  for (int v = threadIdx.x; v < V; v += kFThreads) {
    const double L = vs[v].L;
    vs[v].invL = L > 0.0 ? (float)(1.0 / L) : 0.f;
    vs[v].thr = L > 0.0 ? (float)(vs[v].lam / L) : 0.f;
  }
  // ---- FISTA; the tile holds pack(y_k) at the top of a step.  Cold: x_0 = y_1 = 0, t_1 = 1.
  //      Warm: x and y hold x_k0 and y_{k0+1}; t_{k0+1} follows from t_1 = 1 by the recurrence.
  if (a.warm) {
    __syncthreads();
    pack_from<LOGL>(s, vs, &VState::y);
    if (threadIdx.x == 0) {
      double t = 1.0;
      if (a.accel)
        for (int k = 0; k < a.k0; ++k) t = fista_t_next(t);
      *s_t = t;
    }
  } else {
    for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
      const int v = q >> LOGL;
      if (vs[v].valid) {
        __stcg(vs[v].x + (q & (Nc - 1)), 0.f);
        __stcg(vs[v].y + (q & (Nc - 1)), 0.f);
      }
      *zaddr<LOGL>(s, q & (Nc - 1), v) = make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) *s_t = 1.0;
  }
  for (int k = 0; k < a.iters; ++k) {
    __syncthreads();
    const double t = *s_t;
    const double tn = a.accel ? fista_t_next(t) : 1.0;
    const float beta = a.accel ? (float)((t - 1.0) / tn) : 0.f;
    // A y_k, the residual (fused into the first pass of the next transform), A^T of it,
    // and the step (fused into the last pass of the inverse transform)
    apply_T<LOGL>(s, vs, 0, a.tw, a.tw2);
    tile_fft_resid<LOGL>(s, vs, a.tw);
    tile_spectral<LOGL>(s, vs, 1, a.tw2);
    __syncthreads();
    tile_ifft_update<LOGL>(s, vs, beta, a.tw);
    if (threadIdx.x == 0) *s_t = tn;
  }
  // ---- objective 1/2 ||A x - b||^2 + lambda ||x||_1 and status
  __syncthreads();
  pack_from<LOGL>(s, vs, &VState::x);
  apply_T<LOGL>(s, vs, 0, a.tw, a.tw2);
  mask_rows<LOGL, MODE_RESID>(s, vs, part, true);
  vec_finish<LOGL>(vs, part);
  for (int v = threadIdx.x; v < V; v += kFThreads) vs[v].cap = 0.5 * vs[v].acc;  // reuse cap: data term
  for (int q = threadIdx.x; q < V * Nc; q += kFThreads) {
    const int v = q >> LOGL;
    const float xv = vs[v].valid ? __ldcg(vs[v].x + (q & (Nc - 1))) : 0.f;
    vec_part(part, q, fabs((double)xv));
  }
  vec_finish<LOGL>(vs, part);
  for (int v = threadIdx.x; v < V; v += kFThreads) {
    if (!vs[v].valid) continue;
    const int ii = vs[v].inst;
    const double obj = vs[v].cap + vs[v].lam * vs[v].acc;
    if (a.rep_L) a.rep_L[ii] = vs[v].L;
    if (a.rep_lambda) a.rep_lambda[ii] = vs[v].lam;
    if (a.rep_obj) a.rep_obj[ii] = obj;
    if (a.rep_status) a.rep_status[ii] = isfinite(obj) ? 0 : (int)FM_ERR_NUMERIC;
  }
}

__global__ void __launch_bounds__(kFThreads, 1) fista_kernel(const __grid_constant__ FistaArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  VState* vs = reinterpret_cast<VState*>(smem_raw + fft_vinfo_offset<float2>(kFE));
  __shared__ int s_group;
  __shared__ double s_t;
  __shared__ double s_part[kFE / 32];   // per-warp partial sums (vec_part)
  bool first = true;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (a.single_group >= 0) s_group = first ? a.single_group : -1;
      else s_group = atomicAdd(a.counter, 1);
    }
    __syncthreads();
    const int gi = s_group;
    first = false;
    if (gi < 0 || gi >= a.ngroups) break;
    const FGroup G = a.groups[gi];
    switch (G.logn) {
      case 8: fista_group<8>(a, G, s, vs, s_part, &s_t); break;
      case 9: fista_group<9>(a, G, s, vs, s_part, &s_t); break;
      case 10: fista_group<10>(a, G, s, vs, s_part, &s_t); break;
      case 11: fista_group<11>(a, G, s, vs, s_part, &s_t); break;
      case 12: fista_group<12>(a, G, s, vs, s_part, &s_t); break;
      case 13: fista_group<13>(a, G, s, vs, s_part, &s_t); break;
      default: fista_group<14>(a, G, s, vs, s_part, &s_t); break;
    }
  }
}

}  // namespace fm

using namespace fm;

struct fm_batch_s {
  std::vector<fm_op_s*> ops;
  int64_t count = 0, total_rows = 0, total_cols = 0;
  int device = 0;
  FInst* inst = nullptr;
  int32_t* order = nullptr;
  FGroup* groups = nullptr;        // persistent work list, largest instances first
  int32_t* order_asc = nullptr;    // ... and its smallest-first form (fm_batch_tune)
  FGroup* groups_asc = nullptr;
  int order_mode = 0;              // 0 largest first, 1 smallest first
  FGroup* single = nullptr;        // one group per instance (per-instance launches)
  std::vector<int32_t> single_index;  // instance -> its entry in `single`
  int ngroups = 0, nsingle = 0;
  float* y = nullptr;
  float2* tw2 = nullptr;
  int* counter = nullptr;
  int sms = 1;
};

static void batch_free(fm_batch_s* B) {
  void* bufs[] = {B->inst, B->order, B->groups, B->order_asc, B->groups_asc, B->single, B->y, B->tw2, B->counter};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (auto* o : B->ops) op_release(o);
  delete B;
}

static size_t fista_smem() { return fft_vinfo_offset<float2>(kFE) + sizeof(VState) * kFMaxV; }

extern "C" {

fm_status fm_batch_create(const fm_op* A, int64_t count, void* stream, fm_batch* out) {
  clear_error();
  if (!out || !A || count < 1) { set_error("need at least one operator"); return FM_ERR_INVALID_ARG; }
  std::vector<FInst> h(count);
  int64_t brow = 0, xcol = 0;
  for (int64_t i = 0; i < count; ++i) {
    const fm_op_s* op = A[i];
    if (!op || op->kind != K_PRODUCT || op->kids.size() != 2 || op->kids[0]->kind != K_PARTIAL ||
        op->kids[1]->kind != K_TOEPLITZ) {
      set_error("instance %lld: expected Product(Partial, Toeplitz)", (long long)i);
      return FM_ERR_UNSUPPORTED;
    }
    const fm_op_s* P = op->kids[0];
    const fm_op_s* T = op->kids[1];
    const int64_t n = T->cols;
    if (!T->real || T->rows != n || P->cols != n || n < 256 || n > 16384 || (n & (n - 1)) || T->L != 2 * n) {
      set_error("instance %lld: need a real n x n Toeplitz with n a power of two in [2^8, 2^14]", (long long)i);
      return FM_ERR_UNSUPPORTED;
    }
    int logn = 0;
    while ((1LL << logn) < n) ++logn;
    h[i].spec = T->spec32;
    h[i].idx = P->idx;
    h[i].inv = P->inv;
    h[i].b_off = brow;
    h[i].x_off = xcol;
    h[i].n = (int)n;
    h[i].m = (int)P->rows;
    h[i].logn = logn;
    h[i].cap = T->cap;
    brow += P->rows;
    xcol += n;
  }
  // groups of equal n, largest first
  std::vector<int32_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = (int32_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t p, int32_t q) { return h[p].logn > h[q].logn; });
  auto make_groups = [&](const std::vector<int32_t>& ord) {
    std::vector<FGroup> g;
    for (int64_t i = 0; i < count;) {
      const int logn = h[ord[i]].logn;
      const int V = 1 << (14 - logn);
      int c = 0;
      while (i + c < count && c < V && h[ord[i + c]].logn == logn) ++c;
      g.push_back({logn, c, (int)i, 0});
      i += c;
    }
    return g;
  };
  const std::vector<FGroup> groups = make_groups(order);
  std::vector<int32_t> order_asc(count);
  for (int64_t i = 0; i < count; ++i) order_asc[i] = (int32_t)i;
  std::stable_sort(order_asc.begin(), order_asc.end(), [&](int32_t p, int32_t q) { return h[p].logn < h[q].logn; });
  const std::vector<FGroup> groups_asc = make_groups(order_asc);
  std::vector<FGroup> single(count);
  std::vector<int32_t> single_index(count);
  for (int64_t r = 0; r < count; ++r) {
    single[r] = {h[order[r]].logn, 1, (int)r, 0};
    single_index[order[r]] = (int32_t)r;
  }
  fm_batch_s* B = new (std::nothrow) fm_batch_s();
  if (!B) return FM_ERR_OOM;
  cudaGetDevice(&B->device);
  for (int64_t i = 0; i < count; ++i) {
    op_retain(A[i]);
    B->ops.push_back(A[i]);
  }
  B->count = count;
  B->total_rows = brow;
  B->total_cols = xcol;
  B->ngroups = (int)groups.size();
  B->nsingle = (int)count;
  B->single_index = single_index;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMalloc(&B->inst, sizeof(FInst) * count);
  if (e == cudaSuccess) e = cudaMalloc(&B->order, sizeof(int32_t) * count);
  if (e == cudaSuccess) e = cudaMalloc(&B->groups, sizeof(FGroup) * groups.size());
  if (e == cudaSuccess) e = cudaMalloc(&B->single, sizeof(FGroup) * count);
  if (e == cudaSuccess) e = cudaMalloc(&B->order_asc, sizeof(int32_t) * count);
  if (e == cudaSuccess) e = cudaMalloc(&B->groups_asc, sizeof(FGroup) * groups_asc.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(B->order_asc, order_asc.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(B->groups_asc, groups_asc.data(), sizeof(FGroup) * groups_asc.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B->y, sizeof(float) * xcol);
  if (e == cudaSuccess) e = cudaMalloc(&B->tw2, sizeof(float2) * 32768);
  if (e == cudaSuccess) e = cudaMalloc(&B->counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(B->inst, h.data(), sizeof(FInst) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->order, order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(B->groups, groups.data(), sizeof(FGroup) * groups.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->single, single.data(), sizeof(FGroup) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("batch setup: %s", cudaGetErrorString(e));
    batch_free(B);
    return e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;
  }
  fm_status s = twiddle_launch(32768, B->tw2, nullptr, st);
  if (s == FM_OK) {
    DeviceTables* t;
    s = device_tables(B->device, &t);
  }
  if (s == FM_OK) {
    e = cudaFuncSetAttribute(fista_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fista_smem());
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("batch setup: %s", cudaGetErrorString(e));
      s = FM_ERR_CUDA;
    }
  }
  if (s != FM_OK) {
    batch_free(B);
    return s;
  }
  *out = B;
  return FM_OK;
}

void fm_batch_release(fm_batch B) {
  if (B) batch_free(B);
}

fm_status fm_batch_sizes(fm_batch B, int64_t* rows, int64_t* cols) {
  if (!B || !rows || !cols) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  *rows = B->total_rows;
  *cols = B->total_cols;
  return FM_OK;
}

static fm_status check_params(const fm_fista_params* p, const fm_fista_report* rep) {
  if (p->iters < 0 || p->power_iters < 1 || !(p->safety > 0.0) || !(p->lambda_rel >= 0.0) ||
      (p->mode != 0 && p->mode != 1) || (p->warm != 0 && p->warm != 1) || p->k0 < 0) {
    set_error("bad FISTA parameters");
    return FM_ERR_INVALID_ARG;
  }
  if (p->warm && (!rep || !rep->L || !rep->lambda)) {
    set_error("a warm start reads L and lambda of the run it resumes from rep->L and rep->lambda");
    return FM_ERR_INVALID_ARG;
  }
  return FM_OK;
}

// Launch the solve of every instance of B (bp, xp: per-instance pointer arrays on the device,
// or NULL for the packed b and x).
static fm_status fista_run(fm_batch B, const float* b, float* x, const float* const* bp, float* const* xp,
                           float* y, const fm_fista_params* p, const fm_fista_report* rep, cudaStream_t st) {
  int dev = 0;
  FM_CUDA(cudaGetDevice(&dev));
  if (dev != B->device) { set_error("batch lives on device %d, current is %d", B->device, dev); return FM_ERR_INVALID_ARG; }
  DeviceTables* tabs = device_tables_if_ready(dev);
  if (!tabs) { set_error("device tables missing"); return FM_ERR_INVALID_ARG; }
  FistaArgs a;
  a.inst = B->inst;
  a.order = B->order;
  a.b = b;
  const bool asc = B->order_mode == 1 && p->mode == 0;
  if (asc) a.order = B->order_asc;
  a.x = x;
  a.bp = bp;
  a.xp = xp;
  a.y = y ? y : B->y;
  a.pw = B->y;
  a.tw = tabs->twp32;
  a.tw2 = B->tw2;
  a.iters = p->iters;
  a.power_iters = p->power_iters;
  a.lambda_rel = p->lambda_rel;
  a.safety = p->safety;
  a.accel = p->accel ? 1 : 0;
  a.warm = p->warm;
  a.k0 = p->k0;
  a.rep_L = rep ? rep->L : nullptr;
  a.rep_lambda = rep ? rep->lambda : nullptr;
  a.rep_obj = rep ? rep->objective : nullptr;
  a.rep_status = rep ? rep->status : nullptr;
  a.counter = B->counter;
  const size_t smem = fista_smem();
  if (p->mode == 0) {
    a.groups = asc ? B->groups_asc : B->groups;
    a.ngroups = B->ngroups;
    a.single_group = -1;
    FM_CUDA(cudaMemsetAsync(B->counter, 0, sizeof(int), st));
    const int grid = std::min(B->ngroups, B->sms);
    const int ts = g_trace_on.load(std::memory_order_relaxed) ? trace_open(st) : -1;
    fista_kernel<<<grid, kFThreads, smem, st>>>(a);
    if (ts >= 0) trace_close(ts, st, "fista_kernel");
    return after_launch("fista_kernel");
  }
  // one instance per launch, in the caller's order
  a.groups = B->single;
  a.ngroups = B->nsingle;
  for (int64_t i = 0; i < B->count; ++i) {
    a.single_group = B->single_index[i];
    const int ts = g_trace_on.load(std::memory_order_relaxed) ? trace_open(st) : -1;
    fista_kernel<<<1, kFThreads, smem, st>>>(a);
    if (ts >= 0) trace_close(ts, st, "fista_kernel");
    FM_TRY(after_launch("fista_kernel"));
  }
  return FM_OK;
}

fm_status fm_fista_batch(fm_batch B, const float* b, float* x, float* y, const fm_fista_params* p,
                         const fm_fista_report* rep, void* stream) {
  clear_error();
  if (!B || !b || !x || !p) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  if ((uintptr_t)x % 8 || (uintptr_t)y % 8) { set_error("x and y must be 8-byte aligned"); return FM_ERR_INVALID_ARG; }
  FM_TRY(check_params(p, rep));
  if (p->warm && !y) { set_error("a warm start needs the momentum state y of the run it resumes"); return FM_ERR_INVALID_ARG; }
  return fista_run(B, b, x, nullptr, nullptr, y, p, rep, (cudaStream_t)stream);
}

fm_status fm_batch_set_order(fm_batch B, int32_t order) {
  clear_error();
  if (!B || (order != 0 && order != 1)) { set_error("order 0 (largest first) or 1 (smallest first)"); return FM_ERR_INVALID_ARG; }
  B->order_mode = order;
  return FM_OK;
}

fm_status fm_batch_tune(fm_batch B, const float* b, float* x, const fm_fista_params* p, void* stream, float* ms,
                        int32_t* chosen) {
  clear_error();
  if (!B || !b || !x || !p) { set_error("null pointer"); return FM_ERR_INVALID_ARG; }
  FM_TRY(check_params(p, nullptr));
  if (p->warm || p->mode != 0) { set_error("tune a cold persistent solve (warm = 0, mode = 0)"); return FM_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FM_CUDA(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  fm_status s = e == cudaSuccess ? FM_OK : FM_ERR_CUDA;
  float t[2] = {0.f, 0.f};
  const int start = B->order_mode;
  for (int m = 0; m < 2 && s == FM_OK; ++m) {
    B->order_mode = m;
    s = fista_run(B, b, x, nullptr, nullptr, nullptr, p, nullptr, st);     // warm-up
    if (s == FM_OK && cudaEventRecord(e0, st) != cudaSuccess) s = FM_ERR_CUDA;
    if (s == FM_OK) s = fista_run(B, b, x, nullptr, nullptr, nullptr, p, nullptr, st);
    if (s == FM_OK && cudaEventRecord(e1, st) != cudaSuccess) s = FM_ERR_CUDA;
    if (s == FM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[m], e0, e1) != cudaSuccess))
      s = FM_ERR_CUDA;
  }
  if (s == FM_ERR_CUDA) set_error("fm_batch_tune: CUDA error while timing");
  B->order_mode = s == FM_OK ? (t[1] < t[0] ? 1 : 0) : start;
  if (ms) { ms[0] = t[0]; ms[1] = t[1]; }
  if (chosen) *chosen = B->order_mode;
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return s;
}

fm_status fm_fista(const fm_op* A, int64_t batch, const float* const* b, float* const* x, const fm_fista_params* p,
                   const fm_fista_report* rep, void* stream) {
  clear_error();
  if (!A || !b || !x || !p || batch < 1) { set_error("null pointer or empty batch"); return FM_ERR_INVALID_ARG; }
  FM_TRY(check_params(p, rep));
  if (p->warm) { set_error("fm_fista starts cold; resume a run through fm_fista_batch"); return FM_ERR_UNSUPPORTED; }
  for (int64_t i = 0; i < batch; ++i) {
    if (!b[i] || !x[i]) { set_error("instance %lld: null b or x", (long long)i); return FM_ERR_INVALID_ARG; }
    if ((uintptr_t)x[i] % 8) { set_error("instance %lld: x must be 8-byte aligned", (long long)i); return FM_ERR_INVALID_ARG; }
  }
  cudaStream_t st = (cudaStream_t)stream;
  fm_batch B = nullptr;
  FM_TRY(fm_batch_create(A, batch, stream, &B));
  void* ptrs = nullptr;
  cudaError_t e = cudaMalloc(&ptrs, 2 * sizeof(void*) * (size_t)batch);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ptrs, b, sizeof(void*) * batch, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void**)ptrs + batch, x, sizeof(void*) * batch, cudaMemcpyHostToDevice, st);
  fm_status s = FM_OK;
  if (e != cudaSuccess) {
    set_error("fm_fista: pointer upload: %s", cudaGetErrorString(e));
    s = e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;
  }
  if (s == FM_OK)
    s = fista_run(B, nullptr, nullptr, (const float* const*)ptrs, (float* const*)((void**)ptrs + batch), nullptr,
                  p, rep, st);
  e = cudaStreamSynchronize(st);
  if (s == FM_OK && e != cudaSuccess) {
    set_error("fm_fista: %s", cudaGetErrorString(e));
    s = FM_ERR_CUDA;
  }
  if (ptrs) cudaFree(ptrs);
  fm_batch_release(B);
  return s;
}

}  // extern "C"
