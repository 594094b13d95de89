// Small complex helpers for float2 / double2 interleaved storage.
#pragma once
#include <cuda_runtime.h>

template <class T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <class T> using cplx = typename CT<T>::type;

template <class T> __host__ __device__ __forceinline__ cplx<T> mkc(T re, T im) {
  cplx<T> z;
  z.x = re;
  z.y = im;
  return z;
}
// acc -= a * b
template <class T> __device__ __forceinline__ void csub_mul(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x -= a.x * b.x - a.y * b.y;
  acc.y -= a.x * b.y + a.y * b.x;
}
// acc += a * b
template <class T> __device__ __forceinline__ void cadd_mul(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}
template <class T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a / b with Smith's scaling (no spurious overflow for |b| >> 1 or << 1)
template <class T> __device__ __forceinline__ cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  if (fabs(b.x) >= fabs(b.y)) {
    T r = b.y / b.x, d = b.x + b.y * r;
    return mkc<T>((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    T r = b.x / b.y, d = b.x * r + b.y;
    return mkc<T>((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
template <class T> __device__ __forceinline__ T cabs1(cplx<T> a) { return fabs(a.x) + fabs(a.y); }

__device__ __forceinline__ float2 to_c(double2 z, float) { return make_float2((float)z.x, (float)z.y); }
__device__ __forceinline__ double2 to_c(double2 z, double) { return z; }
__device__ __forceinline__ double2 to_d(float2 z) { return make_double2((double)z.x, (double)z.y); }
__device__ __forceinline__ double2 to_d(double2 z) { return z; }

// Compensated accumulation (Ogita, Rump, Oishi 2005, Dot2): s + c carries the sum of
// the exact products as if accumulated in twice the working precision; each product
// is split exactly by FMA (TwoProd), each addition by TwoSum.  The _rn intrinsics keep
// the compiler from contracting the transformations into FMAs.
__device__ __forceinline__ void dot2_add(double& s, double& c, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double e = fma(a, b, -p);
  const double t = __dadd_rn(s, p);
  const double z = __dsub_rn(t, s);
  c = __dadd_rn(c, __dadd_rn(__dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(p, z)), e));
  s = t;
}

// Relaxed-ordering loads that bypass L1 (data written by other CTAs).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <class T> __device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }
