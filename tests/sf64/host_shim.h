// Host definitions of the few CUDA intrinsics sf64.cuh uses, so the host
// test suite can compile it with g++. The single-precision approximations
// are perturbed by up to 2 ulp on purpose, to exercise the Newton steps
// with a seed no better than the hardware's.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdint>
#define __device__
#define __forceinline__ inline
#define SF_CALL __attribute__((noinline))
static inline long long __double_as_longlong(double d) { long long v; memcpy(&v, &d, 8); return v; }
static inline double __longlong_as_double(long long v) { double d; memcpy(&d, &v, 8); return d; }
static inline unsigned __float_as_uint(float f) { unsigned v; memcpy(&v, &f, 4); return v; }
static inline float __uint_as_float(unsigned v) { float f; memcpy(&f, &v, 4); return f; }
static inline unsigned long long vbe_umulhi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
static inline long long vbe_smulhi(long long a, long long b) { return (long long)(((__int128)a * b) >> 64); }
static inline int vbe_clz64(unsigned long long x) { return x ? __builtin_clzll(x) : 64; }
static unsigned g_perturb = 12345;
static inline float perturb(float r) {
  g_perturb = g_perturb * 1103515245u + 12345u;
  unsigned b = __float_as_uint(r);
  int d = (int)((g_perturb >> 16) % 5) - 2;  // -2..2 ulp
  return __uint_as_float(b + d);
}
static inline float vbe_rcp_approx(float x) { return perturb(1.0f / x); }
static inline float vbe_rsqrt_approx(float x) { return perturb(1.0f / std::sqrt(x)); }
