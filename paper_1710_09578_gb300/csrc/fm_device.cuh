// Device helpers shared by the kernels of the structured-operator library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fm {

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

__device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }

// Programmatic dependent launch: pdl_wait() blocks until the previous grid of the stream has
// completed with its writes visible (a no-op when the launch did not allow an early start);
// pdl_launch_dependents() lets the next grid start once every CTA of this one has called it.
// A kernel launched this way reads data that the previous grid writes only through coherent
// loads (ld.global): a read-only .nc load (ld.global.nc, __ldg, or one the compiler derives
// from a const __restrict__ pointer) may be served before the wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmake(a.x * s, a.y * s); }
// a * (dir * i): dir = -1 gives a * (-i), dir = +1 gives a * i.
template <typename C> __device__ __forceinline__ C cmul_i(C a, int dir) {
  return dir > 0 ? cmake(-a.y, a.x) : cmake(a.y, -a.x);
}

// In-register DFTs of size 2, 4, 8 with y_k = sum_r a_r exp(dir * 2 pi i r k / R), natural order.
template <typename C> __device__ __forceinline__ void dft2(C* a) {
  C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}
template <typename C> __device__ __forceinline__ void dft4(C* a, int dir) {
  C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  C t2 = cadd(a[1], a[3]), t3 = cmul_i(csub(a[1], a[3]), dir);
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}
template <typename C> __device__ __forceinline__ void dft8(C* a, int dir) {
  typedef decltype(a[0].x) T;
  const T h = (T)0.70710678118654752440084436210484903928;
  C e[4] = {a[0], a[2], a[4], a[6]};
  C o[4] = {a[1], a[3], a[5], a[7]};
  dft4(e, dir);
  dft4(o, dir);
  // o_k * exp(dir * 2 pi i k / 8)
  C o1 = cscale(cadd(o[1], cmul_i(o[1], dir)), h);
  C o2 = cmul_i(o[2], dir);
  C o3 = cscale(csub(cmul_i(o[3], dir), o[3]), h);
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], o1);
  a[5] = csub(e[1], o1);
  a[2] = cadd(e[2], o2);
  a[6] = csub(e[2], o2);
  a[3] = cadd(e[3], o3);
  a[7] = csub(e[3], o3);
}

// x * W_16^m with W_16 = exp(dir * 2 pi i / 16), for the nine exponents of a 4 x 4 split.
template <typename C, int M>
__device__ __forceinline__ C w16(C x, int dir) {
  typedef decltype(x.x) T;
  constexpr int m = M % 16;
  if constexpr (m == 0) return x;
  else if constexpr (m == 4) return cmul_i(x, dir);
  else if constexpr (m == 8) return cmake(-x.x, -x.y);
  else if constexpr (m == 12) return cmul_i(x, -dir);
  else {
    // cos and sin of 2 pi m / 16 for m = 1, 2, 3, 6, 9 (the only other exponents used)
    const T c1 = (T)0.92387953251128675612818318939678828682, s1 = (T)0.38268343236508977172845998403039886676;
    const T h = (T)0.70710678118654752440084436210484903928;
    T c, sn;
    if constexpr (m == 1) { c = c1; sn = s1; }
    else if constexpr (m == 2) { c = h; sn = h; }
    else if constexpr (m == 3) { c = s1; sn = c1; }
    else if constexpr (m == 6) { c = -h; sn = h; }
    else { c = -c1; sn = -s1; }  // m == 9
    const T sd = dir > 0 ? sn : -sn;
    return cmake(x.x * c - x.y * sd, x.x * sd + x.y * c);
  }
}

// In-register DFT of size 16 (natural order in and out) as 4 x 4: DFTs of length 4 over
// the stride-4 subsequences, twiddles W_16^(i k1), DFTs of length 4 across them; the
// result index k1 + 4 k2 is a renaming of registers.
template <typename C> __device__ __forceinline__ void dft16(C* a, int dir) {
  C b[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    C t[4] = {a[i], a[i + 4], a[i + 8], a[i + 12]};
    dft4(t, dir);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) b[4 * i + k1] = t[k1];
  }
  b[5] = w16<C, 1>(b[5], dir);
  b[6] = w16<C, 2>(b[6], dir);
  b[7] = w16<C, 3>(b[7], dir);
  b[9] = w16<C, 2>(b[9], dir);
  b[10] = w16<C, 4>(b[10], dir);
  b[11] = w16<C, 6>(b[11], dir);
  b[13] = w16<C, 3>(b[13], dir);
  b[14] = w16<C, 6>(b[14], dir);
  b[15] = w16<C, 9>(b[15], dir);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[4] = {b[k1], b[4 + k1], b[8 + k1], b[12 + k1]};
    dft4(t, dir);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
  }
}

// x * W_32^m with W_32 = exp(dir * 2 pi i / 32), m = 0 .. 15.
template <typename C, int M>
__device__ __forceinline__ C w32(C x, int dir) {
  typedef decltype(x.x) T;
  if constexpr (M == 0) return x;
  else if constexpr (M == 8) return cmul_i(x, dir);
  else if constexpr (M == 4 || M == 12) {
    const T h = (T)0.70710678118654752440084436210484903928;
    return M == 4 ? cscale(cadd(x, cmul_i(x, dir)), h) : cscale(csub(cmul_i(x, dir), x), h);
  } else {
    // cos and sin of pi m / 16 from those of pi / 16, pi / 8 and 3 pi / 16 by symmetry
    const T c1 = (T)0.98078528040323044912618223613424, s1 = (T)0.19509032201612826784828486847702;
    const T c2 = (T)0.92387953251128675612818318939679, s2 = (T)0.38268343236508977172845998403040;
    const T c3 = (T)0.83146961230254523707878837761791, s3 = (T)0.55557023301960222474283081394853;
    constexpr int q = M < 8 ? M : 16 - M;  // cos(pi (16 - q) / 16) = -cos(pi q / 16), sin equal
    T c, sn;
    if constexpr (q == 1) { c = c1; sn = s1; }
    else if constexpr (q == 2) { c = c2; sn = s2; }
    else if constexpr (q == 3) { c = c3; sn = s3; }
    else if constexpr (q == 5) { c = s3; sn = c3; }
    else if constexpr (q == 6) { c = s2; sn = c2; }
    else { c = s1; sn = c1; }  // q == 7
    if constexpr (M > 8) c = -c;
    const T sd = dir > 0 ? sn : -sn;
    return cmake(x.x * c - x.y * sd, x.x * sd + x.y * c);
  }
}

// In-register DFT of size 32 (natural order in and out): DFTs of length 16 over the even and
// the odd elements, then y_k = E_k + W_32^k O_k and y_(k+16) = E_k - W_32^k O_k.
template <typename C, int K = 0>
__device__ __forceinline__ void dft32_combine(C* a, const C* e, const C* o, int dir) {
  if constexpr (K < 16) {
    const C t = w32<C, K>(o[K], dir);
    a[K] = cadd(e[K], t);
    a[K + 16] = csub(e[K], t);
    dft32_combine<C, K + 1>(a, e, o, dir);
  }
}
template <typename C> __device__ __forceinline__ void dft32(C* a, int dir) {
  C e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = a[2 * i];
    o[i] = a[2 * i + 1];
  }
  dft16(e, dir);
  dft16(o, dir);
  dft32_combine<C>(a, e, o, dir);
}

// Global-space loads and stores.  With the state space explicit (rather than a generic
// address that might point into shared memory) the instruction scheduler may move a load
// ahead of unrelated shared-memory stores, so a thread can have all the loads of a tile in
// flight at once.  The loads are volatile so that the compiler never executes one
// speculatively, outside the bounds check that guards it.
__device__ __forceinline__ float gld(const float* p) {
  float r;
  asm volatile("ld.global.f32 %0, [%1];" : "=f"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ double gld(const double* p) {
  double r;
  asm volatile("ld.global.f64 %0, [%1];" : "=d"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ float2 gld(const float2* p) {
  float2 r;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ double2 gld(const double2* p) {
  double2 r;
  asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ int gld(const int32_t* p) {
  int r;
  asm volatile("ld.global.s32 %0, [%1];" : "=r"(r) : "l"(p));
  return r;
}
__device__ __forceinline__ void gst(float* p, float v) {
  asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void gst(double* p, double v) {
  asm volatile("st.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void gst(float2* p, float2 v) {
  asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void gst(double2* p, double2 v) {
  asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v.x), "d"(v.y) : "memory");
}

// Pass-twiddle tables: for a radix-2^lr pass of a Stockham transform whose butterflies span
// 2^s = Ns * R elements, row i < Ns holds W_{2^s}^(i k), k = 0 .. R - 1 (W = exp(-2 pi i / 2^s)),
// so a butterfly j reads row j mod Ns as R contiguous entries.  One block of 2^s entries per
// (s, lr), s = 1 .. 14, lr = 1 .. min(4, s), in that order.
__host__ __device__ constexpr int64_t pass_tw_offset(int s, int lr) {
  int64_t off = 0;
  for (int q = 1; q < s; ++q) off += (int64_t)(q < 4 ? q : 4) << q;
  return off + ((int64_t)(lr - 1) << s);
}
constexpr int64_t kPassTwEntries = pass_tw_offset(15, 1);

// Shared-memory index with one pad slot every 16 elements (breaks power-of-two strides).
__device__ __forceinline__ int spad(int lin) { return lin + (lin >> 4); }

}  // namespace fm
