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

// Shared-memory index with one pad slot every 16 elements (breaks power-of-two strides).
__device__ __forceinline__ int spad(int lin) { return lin + (lin >> 4); }

}  // namespace fm
