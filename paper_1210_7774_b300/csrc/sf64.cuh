// Float64 division, square root, exp and log evaluated with 64-bit integer
// arithmetic, for GPUs whose FP64 pipe is narrow (on B300 it retires two
// lanes per clock per SM, 1/64 of the FP32 rate, while the integer and FP32
// pipes are wide). Every function returns the same result class as the
// IEEE operation it replaces and falls back to the native operation for
// operands it does not handle (zeros, subnormals, infinities, NaNs, results
// outside the normal range), so the fallback is rare on real data.
//
// Methods (written from the mathematics; no vendor library code):
//  * division and square root: a reciprocal (resp. reciprocal square root)
//    seeded by the single-precision hardware approximation and refined by
//    two Newton-Raphson steps in 64-bit fixed point (error < 2^-60), a
//    quotient (root) estimate from it, then the exact integer remainder
//    decides the correctly rounded (round-to-nearest-even) result
//    (Markstein's remainder-based correction, IBM J. Res. Dev. 34(1), 1990);
//  * exp: table-driven reduction x = (64k + j) ln2/64 + r, |r| <= ln2/64,
//    exp(x) = 2^k 2^(j/64) e^r with a degree-8 Taylor polynomial in
//    fixed point (Tang, ACM TOMS 15(2), 1989);
//  * log: x = 2^e m, m in [0.75, 1.5), m = F (1 + f) with F = j/128 from
//    a table, log x = e ln2 + log F + log1p(f) with a degree-9 series in
//    fixed point (Tang, ACM TOMS 16(4), 1990); near x = 1 the series is
//    evaluated relative to |x - 1| so there is no cancellation.
// exp and log are accurate to about 0.5 ulp (not always correctly
// rounded); division and square root are correctly rounded.
//
// The file is plain CUDA C++; the host test suite compiles it with g++ and
// compares against the host's IEEE arithmetic.
#ifndef VBE_SF64_CUH
#define VBE_SF64_CUH

#include "sf64_tables.h"

// the four entry points are real calls: inlined, a kernel that uses them
// several times grows large and compiles slowly
#ifndef SF_CALL
#define SF_CALL __noinline__
#endif

typedef unsigned long long sf_u64;
typedef long long sf_i64;

#define SF_M52 0x000FFFFFFFFFFFFFull
#define SF_H52 0x0010000000000000ull
#define SF_SIGN 0x8000000000000000ull

// The native operations, for the cases the integer routines below leave to
// the FP64 pipe (special operands, results outside the normal range). They
// are kept out of line so that none of their code is scheduled into the
// integer paths.
__device__ SF_CALL double vbe_ddiv_native(double a, double b) { return a / b; }
__device__ SF_CALL double vbe_dsqrt_native(double a) { return sqrt(a); }
__device__ SF_CALL double vbe_dexp_native(double x) { return exp(x); }
__device__ SF_CALL double vbe_dlog_native(double x) { return log(x); }

// The bits of a double, opaque to the compiler: a test on them (a zero
// numerator, say) would otherwise be turned back into a float64 compare on
// the FP64 pipe (measured: one such compare per divide).
__device__ __forceinline__ sf_u64 sf_bits(double a) {
#ifdef __CUDA_ARCH__
  sf_u64 u;
  asm("mov.b64 %0, %1;" : "=l"(u) : "d"(a));
  return u;
#else
  return (sf_u64)__double_as_longlong(a);
#endif
}

// ------------------------------------------------------------ division

__device__ SF_CALL double vbe_ddiv(double a, double b) {
  const sf_u64 ua = sf_bits(a), ub = sf_bits(b);
  const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  const sf_u64 sign = (ua ^ ub) & SF_SIGN;
  // a zero numerator over a normal or infinite divisor: a signed zero
  // (frequent in practice, e.g. momenta of a fluid at rest)
  if ((ua << 1) == 0 && eb != 0 && ((ub << 12) == 0 || eb != 0x7ff)) return __longlong_as_double((sf_i64)sign);
  if (ea == 0 || ea == 0x7ff || eb == 0 || eb == 0x7ff) return vbe_ddiv_native(a, b);
  const sf_u64 ma = (ua & SF_M52) | SF_H52, mb = (ub & SF_M52) | SF_H52;
  if ((ub & SF_M52) == 0) {  // b = +-2^k: the quotient is exact
    const int er = ea - eb + 1023;
    if (er < 1 || er > 2046) return vbe_ddiv_native(a, b);
    return __longlong_as_double((sf_i64)(sign | ((sf_u64)er << 52) | (ua & SF_M52)));
  }
  const int s = ma < mb ? 53 : 52;
  int er = ea - eb + 1023 - (s - 52);
  if (er < 1 || er > 2046) return vbe_ddiv_native(a, b);
  // x = 1/d, d = mb / 2^53 in (0.5, 1); X = x 2^62 (Q2.62), D = d 2^64 (Q0.64)
  const sf_u64 D = mb << 11;
  const float df = __uint_as_float((126u << 23) | (unsigned)((mb >> 29) & 0x7fffffu));
  const unsigned xb = __float_as_uint(vbe_rcp_approx(df));
  const int xe = (int)(xb >> 23) - 88;
  if (xe < 30 || xe > 41) return vbe_ddiv_native(a, b);
  sf_u64 X = (sf_u64)((xb & 0x7fffffu) | 0x800000u) << xe;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const sf_u64 T = vbe_umulhi(D, X);  // d x, Q2.62
    const sf_u64 E = (2ull << 62) - T;   // 2 - d x
    X = (vbe_umulhi(X, E) << 2) | ((X * E) >> 62);
  }
  // R = 2^116 / mb ~ 2 X; quotient estimate of (ma << s) / mb
  const sf_u64 R = X << 1;
  const sf_u64 hi = vbe_umulhi(ma, R), lo = ma * R;
  sf_u64 q = s == 52 ? hi : ((hi << 1) | (lo >> 63));
  // exact remainder (|rem| < 2^55, so the low 64 bits hold it)
  sf_i64 rem = (sf_i64)((ma << s) - q * mb);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (rem < 0) {
      q -= 1;
      rem += (sf_i64)mb;
    } else if (rem >= (sf_i64)mb) {
      q += 1;
      rem -= (sf_i64)mb;
    }
  }
  // round to nearest, ties to even: compare 2 rem with mb
  const sf_u64 r2 = (sf_u64)rem << 1;
  if (r2 > mb || (r2 == mb && (q & 1))) q += 1;
  if (q == (SF_H52 << 1)) {
    q = SF_H52;
    er += 1;
    if (er > 2046) return vbe_ddiv_native(a, b);
  }
  return __longlong_as_double((sf_i64)(sign | ((sf_u64)er << 52) | (q & SF_M52)));
}

// --------------------------------------------------------- square root

__device__ SF_CALL double vbe_dsqrt(double a) {
  const sf_u64 ua = (sf_u64)__double_as_longlong(a);
  const int ea = (int)((ua >> 52) & 0x7ff);
  if ((ua & SF_SIGN) || ea == 0 || ea == 0x7ff) return vbe_dsqrt_native(a);
  sf_u64 m = (ua & SF_M52) | SF_H52;  // a = m 2^(ea - 1075)
  int e = ea - 1023;                   // a = (m 2^-52) 2^e
  if (e & 1) {
    m <<= 1;
    e -= 1;
  }
  // t = m 2^-52 in [1, 4); T = t 2^62
  const sf_u64 T = m << 10;
  const unsigned hb = (unsigned)(m >> 53);  // t in [2, 4)
  const float tf = __uint_as_float(((127u + hb) << 23) | (unsigned)((m >> (29 + hb)) & 0x7fffffu));
  const unsigned yb = __float_as_uint(vbe_rsqrt_approx(tf));
  const int ye = (int)(yb >> 23) - 88;
  if (ye < 30 || ye > 41) return vbe_dsqrt_native(a);
  sf_u64 Y = (sf_u64)((yb & 0x7fffffu) | 0x800000u) << ye;  // y = 1/sqrt(t) in (0.5, 1], Q2.62
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const sf_u64 Y2 = (vbe_umulhi(Y, Y) << 2) | ((Y * Y) >> 62);   // y^2
    const sf_u64 TY2 = (vbe_umulhi(T, Y2) << 2) | ((T * Y2) >> 62);  // t y^2 ~ 1
    const sf_u64 F = (3ull << 62) - TY2;                              // 3 - t y^2
    Y = (vbe_umulhi(Y, F) << 1) | ((Y * F) >> 63);                   // y (3 - t y^2) / 2
  }
  const sf_u64 S = (vbe_umulhi(T, Y) << 2) | ((T * Y) >> 62);  // sqrt(t), Q2.62, in [1, 2)
  sf_u64 q = S >> 10;                                            // ~ sqrt(m 2^52), 53 bits
  // exact remainder N - q^2 with N = m << 52 (|rem| < 2^60)
  sf_i64 rem = (sf_i64)((m << 52) - q * q);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (rem < 0) {
      rem += (sf_i64)(2 * q - 1);
      q -= 1;
    } else if (rem > (sf_i64)(2 * q)) {
      q += 1;
      rem -= (sf_i64)(2 * q - 1);
    }
  }
  if (rem > (sf_i64)q) q += 1;  // (q + 1/2)^2 = q^2 + q + 1/4 is never an integer: no ties
  const int er = e / 2 + 1023;
  if (q == (SF_H52 << 1)) return vbe_dsqrt_native(a);  // cannot happen for a normal input; stay safe
  return __longlong_as_double((sf_i64)(((sf_u64)er << 52) | (q & SF_M52)));
}

// --------------------------------------------- multiply, add, compare

// a * b, correctly rounded (round to nearest, ties to even)
__device__ __forceinline__ double vbe_dmul(double a, double b) {
  const sf_u64 ua = (sf_u64)__double_as_longlong(a), ub = (sf_u64)__double_as_longlong(b);
  const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  int e = ea + eb - 1023;
  if (ea == 0 || ea == 0x7ff || eb == 0 || eb == 0x7ff || e < 1 || e > 2045) return a * b;
  const sf_u64 A = ((ua & SF_M52) | SF_H52) << 11, mb = (ub & SF_M52) | SF_H52;
  const sf_u64 hi = vbe_umulhi(A, mb), lo = A * mb;  // P = ma mb: hi = P >> 53, lo = P << 11
  sf_u64 q, round, sticky;
  if (hi >> 52) {  // P in [2^105, 2^106)
    q = hi;
    round = lo >> 63;
    sticky = (lo << 1) != 0;
    e += 1;
  } else {
    q = (hi << 1) | (lo >> 63);
    round = (lo >> 62) & 1;
    sticky = (lo << 2) != 0;
  }
  q += round & (sticky | (q & 1));
  if (q == (SF_H52 << 1)) {
    q >>= 1;
    e += 1;
  }
  if (e > 2046) return a * b;
  return __longlong_as_double((sf_i64)(((ua ^ ub) & SF_SIGN) | ((sf_u64)e << 52) | (q & SF_M52)));
}

// a * c where c is a constant: when c = +-2^k and the product is a normal
// number (or a is a signed zero) the product is exact and is formed by moving
// the exponent field on the integer pipes; any other case is the hardware
// multiply. Whether c is a power of two is uniform across the kernel.
__device__ __forceinline__ double vbe_dmul_k(double a, double c) {
  const sf_u64 uc = (sf_u64)__double_as_longlong(c);
  const int ec = (int)((uc >> 52) & 0x7ff);
  if ((uc & SF_M52) == 0 && ec != 0 && ec != 0x7ff) {
    const sf_u64 ua = (sf_u64)__double_as_longlong(a), sg = uc & SF_SIGN;
    const int ea = (int)((ua >> 52) & 0x7ff), k = ec - 1023;
    if ((unsigned)(ea + k - 1) < 0x7feu && ea != 0 && ea != 0x7ff)
      return __longlong_as_double((sf_i64)((ua ^ sg) + ((sf_u64)(sf_i64)k << 52)));
    if ((ua << 1) == 0) return __longlong_as_double((sf_i64)(ua ^ sg));
  }
  return a * c;
}

// a + b, correctly rounded (round to nearest, ties to even)
__device__ __forceinline__ double vbe_dadd(double a, double b) {
  sf_u64 ua = (sf_u64)__double_as_longlong(a), ub = (sf_u64)__double_as_longlong(b);
  int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  if (ea == 0 || ea == 0x7ff || eb == 0 || eb == 0x7ff) return a + b;
  if ((ua & ~SF_SIGN) < (ub & ~SF_SIGN)) {  // |a| >= |b| from here on
    const sf_u64 t = ua;
    ua = ub;
    ub = t;
    const int te = ea;
    ea = eb;
    eb = te;
  }
  const int d = ea - eb;
  const sf_u64 ma = ((ua & SF_M52) | SF_H52) << 10;  // leading bit at 62, 10 guard bits
  const sf_u64 mb = ((ub & SF_M52) | SF_H52) << 10;
  const sf_u64 mbs = d >= 64 ? 0 : (mb >> d);
  const sf_u64 st = d >= 64 ? 1 : (d > 0 && (mb << (64 - d)) != 0);  // bits of b shifted out
  int e = ea;
  sf_u64 m;
  if (((ua ^ ub) & SF_SIGN) == 0) {
    m = ma + mbs;
    if (m >> 63) {
      m = (m >> 1) | (m & 1);
      e += 1;
    }
    m |= st;
  } else {
    m = ma - mbs - st;  // floor of the exact difference
    if (m == 0) return 0.0;
    const int lz = vbe_clz64(m) - 1;
    m = (m << lz) | st;
    e -= lz;
  }
  // keep bits 62..10; bits 9..0 decide the rounding (sticky in bit 0)
  sf_u64 q = m >> 10;
  const sf_u64 rest = m & 0x3ff;
  if (rest > 0x200 || (rest == 0x200 && (q & 1))) q += 1;
  if (q == (SF_H52 << 1)) {
    q >>= 1;
    e += 1;
  }
  if (e < 1 || e > 2046) return a + b;
  return __longlong_as_double((sf_i64)((ua & SF_SIGN) | ((sf_u64)e << 52) | (q & SF_M52)));
}

__device__ __forceinline__ double vbe_dsub(double a, double b) {
  return vbe_dadd(a, __longlong_as_double(__double_as_longlong(b) ^ (sf_i64)SF_SIGN));
}

// IEEE ordering on bit patterns: NaN compares false (NOT_EQUAL true), -0 == +0
__device__ __forceinline__ sf_i64 sf_key(sf_u64 u) {
  return (u & SF_SIGN) ? -(sf_i64)(u & ~SF_SIGN) : (sf_i64)u;
}
__device__ __forceinline__ bool sf_isnan(sf_u64 u) { return (u & ~SF_SIGN) > 0x7ff0000000000000ull; }
__device__ __forceinline__ bool vbe_dlt(double a, double b) {
  const sf_u64 ua = (sf_u64)__double_as_longlong(a), ub = (sf_u64)__double_as_longlong(b);
  return !sf_isnan(ua) && !sf_isnan(ub) && sf_key(ua) < sf_key(ub);
}
__device__ __forceinline__ bool vbe_dle(double a, double b) {
  const sf_u64 ua = (sf_u64)__double_as_longlong(a), ub = (sf_u64)__double_as_longlong(b);
  return !sf_isnan(ua) && !sf_isnan(ub) && sf_key(ua) <= sf_key(ub);
}
__device__ __forceinline__ bool vbe_deq(double a, double b) {
  const sf_u64 ua = (sf_u64)__double_as_longlong(a), ub = (sf_u64)__double_as_longlong(b);
  return !sf_isnan(ua) && !sf_isnan(ub) && sf_key(ua) == sf_key(ub);
}
__device__ __forceinline__ double vbe_dneg(double a) {
  return __longlong_as_double(__double_as_longlong(a) ^ (sf_i64)SF_SIGN);
}
__device__ __forceinline__ double vbe_dabs(double a) {
  return __longlong_as_double(__double_as_longlong(a) & (sf_i64)~SF_SIGN);
}
// v 2^-53 for an integer 0 <= v < 2^53 (exact)
__device__ __forceinline__ double vbe_u53_to_unit(sf_u64 v) {
  if (v == 0) return 0.0;
  const int lz = vbe_clz64(v);  // >= 11
  return __longlong_as_double((sf_i64)(((sf_u64)(1033 - lz) << 52) | ((v << (lz - 11)) & SF_M52)));
}

// ---------------------------------------------------- 128-bit helpers

struct sf_i128 {  // two's complement, value = hi * 2^64 + lo
  sf_i64 hi;
  sf_u64 lo;
};

__device__ __forceinline__ sf_i128 sf_sub(sf_i128 a, sf_i128 b) {
  sf_i128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (sf_i64)(a.lo < b.lo);
  return r;
}

__device__ __forceinline__ sf_i128 sf_add(sf_i128 a, sf_i128 b) {
  sf_i128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (sf_i64)(r.lo < a.lo);
  return r;
}

__device__ __forceinline__ sf_i128 sf_neg(sf_i128 a) {
  sf_i128 z = {0, 0};
  return sf_sub(z, a);
}

// k * (hi, lo) for a signed 32-bit k and a non-negative 128-bit (hi, lo)
__device__ __forceinline__ sf_i128 sf_mul_small(int k, sf_u64 hi, sf_u64 lo) {
  const sf_u64 ak = (sf_u64)(k < 0 ? -(sf_i64)k : (sf_i64)k);
  sf_i128 p;
  p.lo = ak * lo;
  p.hi = (sf_i64)(ak * hi + vbe_umulhi(ak, lo));
  return k < 0 ? sf_neg(p) : p;
}

// round a positive mantissa word v (value v * 2^scale_exp) to 53 bits and
// pack it with the sign; returns false when the exponent leaves the normal
// range (the caller then uses the native operation)
__device__ __forceinline__ bool sf_pack(sf_u64 v, int scale_exp, sf_u64 sign, double* out) {
  const int lead = 63 - vbe_clz64(v);
  const int sh = lead - 52;
  sf_u64 q = sh >= 0 ? (v >> sh) : (v << -sh);
  if (sh > 0) q += (v >> (sh - 1)) & 1;  // round half up (below 0.51 ulp with the error budget)
  int e = lead + scale_exp;
  if (q == (SF_H52 << 1)) {
    q >>= 1;
    e += 1;
  }
  const int eb = e + 1023;
  if (eb < 1 || eb > 2046) return false;
  *out = __longlong_as_double((sf_i64)(sign | ((sf_u64)eb << 52) | (q & SF_M52)));
  return true;
}

// ------------------------------------------------------------------ exp

__device__ SF_CALL double vbe_dexp(double x) {
  const sf_u64 ux = (sf_u64)__double_as_longlong(x);
  const int ex = (int)((ux >> 52) & 0x7ff);
  if (ex < 1023 - 40 || ex > 1031) return vbe_dexp_native(x);  // |x| < 2^-40, |x| >= 512, inf, nan
  // k ~ round(x 64 / ln2) in single precision (off by at most one)
  const float xf = __uint_as_float((unsigned)((ux >> 32) & 0x80000000u) |
                                   ((unsigned)(ex - 1023 + 127) << 23) | (unsigned)((ux >> 29) & 0x7fffffu));
  const float kf = xf * 92.33248261689366f + 12582912.0f;  // 1.5 * 2^23 rounds to an integer
  const int k = (int)(__float_as_uint(kf) - 0x4B400000u);
  // X = x 2^112 exactly (53-bit mantissa shifted by ex - 963 in [20, 68])
  const sf_u64 M = (ux & SF_M52) | SF_H52;
  const int sh = ex - 963;
  sf_i128 X;
  X.lo = sh >= 64 ? 0 : (M << sh);
  X.hi = (sf_i64)(sh >= 64 ? (M << (sh - 64)) : (M >> (64 - sh)));
  if (ux & SF_SIGN) X = sf_neg(X);
  // r = x - k ln2/64 at scale 2^-112, then R = r 2^68 (|r| < 0.017)
  const sf_i128 r = sf_sub(X, sf_mul_small(k, VBE_LN2_64TH_HI, VBE_LN2_64TH_LO));
  const sf_i64 R = (sf_i64)(((sf_u64)r.hi << 20) | (r.lo >> 44));
  // e^r = sum r^n / n!, n <= 8, Horner in Q2.62
  sf_i64 P = (sf_i64)((1ull << 62) / 40320);
  P = (sf_i64)((1ull << 62) / 5040) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)((1ull << 62) / 720) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)((1ull << 62) / 120) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)((1ull << 62) / 24) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)((1ull << 62) / 6) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)(1ull << 61) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)(1ull << 62) + (vbe_smulhi(P, R) >> 4);
  P = (sf_i64)(1ull << 62) + (vbe_smulhi(P, R) >> 4);
  // 2^(j/64) e^r, value V 2^-61
  const int j = k & 63, m = k >> 6;
  const sf_u64 V = vbe_umulhi(VBE_EXP2_TAB[j], (sf_u64)P);
  double out;
  if (!sf_pack(V, m - 61, 0, &out)) return vbe_dexp_native(x);
  return out;
}

// ------------------------------------------------------------------ log

// Q(u) = log1p(u) / u = 1 - u/2 + u^2/3 - ... + u^8/9 for |u| < 0.006, u
// and the result at scale 2^-62
__device__ __forceinline__ sf_i64 sf_log1p_q(sf_i64 u) {
  sf_i64 Q = (sf_i64)((1ull << 62) / 9);
  Q = -(sf_i64)((1ull << 62) / 8) + (vbe_smulhi(Q, u) << 2);
  Q = (sf_i64)((1ull << 62) / 7) + (vbe_smulhi(Q, u) << 2);
  Q = -(sf_i64)((1ull << 62) / 6) + (vbe_smulhi(Q, u) << 2);
  Q = (sf_i64)((1ull << 62) / 5) + (vbe_smulhi(Q, u) << 2);
  Q = -(sf_i64)((1ull << 62) / 4) + (vbe_smulhi(Q, u) << 2);
  Q = (sf_i64)((1ull << 62) / 3) + (vbe_smulhi(Q, u) << 2);
  Q = -(sf_i64)(1ull << 61) + (vbe_smulhi(Q, u) << 2);
  Q = (sf_i64)(1ull << 62) + (vbe_smulhi(Q, u) << 2);
  return Q;
}

__device__ __forceinline__ sf_i128 sf_from_i64(sf_i64 v) {
  sf_i128 r;
  r.lo = (sf_u64)v;
  r.hi = v < 0 ? -1 : 0;
  return r;
}

__device__ SF_CALL double vbe_dlog(double x) {
  const sf_u64 ux = (sf_u64)__double_as_longlong(x);
  const int ex = (int)((ux >> 52) & 0x7ff);
  if ((ux & SF_SIGN) || ex == 0 || ex == 0x7ff) return vbe_dlog_native(x);
  const sf_u64 M = (ux & SF_M52) | SF_H52;
  int e = ex - 1023;
  // x = 2^e m with m in [0.75, 1.5); Mq = m 2^63; m - 1 = Fint 2^-fs exactly
  sf_u64 Mq;
  sf_i64 Fint;
  int fs;
  if (M >= 0x18000000000000ull) {
    e += 1;
    Mq = M << 10;
    Fint = (sf_i64)M - (sf_i64)(SF_H52 << 1);
    fs = 53;
  } else {
    Mq = M << 11;
    Fint = (sf_i64)M - (sf_i64)SF_H52;
    fs = 52;
  }
  const int jj = (int)((Mq + (1ull << 55)) >> 56);  // round(128 m) in [96, 192]
  if (jj == 128 && e == 0) {
    // near 1: log x = f Q(f), f = m - 1, evaluated relative to |f|
    if (Fint == 0) return 0.0;
    const sf_i64 Q = sf_log1p_q(Fint << (62 - fs));
    const sf_u64 af = (sf_u64)(Fint < 0 ? -Fint : Fint);
    const int z = vbe_clz64(af);
    double out;
    if (!sf_pack(vbe_umulhi(af << z, (sf_u64)Q), 2 - fs - z, Fint < 0 ? SF_SIGN : 0, &out)) return vbe_dlog_native(x);
    return out;
  }
  const int i = jj - 96;
  // u = m / F - 1 with F = jj / 128, at scale 2^-64 (|u| < 0.0053)
  const sf_u64 ph = vbe_umulhi(Mq, VBE_LOG_INV[i]), pl = Mq * VBE_LOG_INV[i];  // m/F at 2^-126
  const sf_i64 u64 = (sf_i64)((((ph - (1ull << 62)) << 2)) | (pl >> 62));
  const sf_i64 Q = sf_log1p_q(u64 >> 2);
  // log1p(u) = u Q at scale 2^-64
  const sf_i64 L1 = (sf_i64)(((sf_u64)vbe_smulhi(u64, Q) << 2) | (((sf_u64)u64 * (sf_u64)Q) >> 62));
  // S = e ln2 + log F + log1p(u), 128-bit at scale 2^-64
  sf_i128 S = sf_mul_small(e, 0, VBE_LN2_HI);
  S = sf_add(S, sf_from_i64(sf_mul_small(e, 0, VBE_LN2_LO).hi));
  S = sf_add(S, sf_from_i64(VBE_LOG_TAB[i]));
  S = sf_add(S, sf_from_i64(L1));
  const sf_u64 sign = S.hi < 0 ? SF_SIGN : 0;
  if (sign) S = sf_neg(S);
  if (S.hi == 0 && S.lo == 0) return vbe_dlog_native(x);
  double out;
  bool ok;
  if (S.hi != 0) {
    const int z = vbe_clz64((sf_u64)S.hi);
    const sf_u64 v = z == 0 ? (sf_u64)S.hi : (((sf_u64)S.hi << z) | (S.lo >> (64 - z)));
    ok = sf_pack(v, -z, sign, &out);
  } else {
    ok = sf_pack(S.lo, -64, sign, &out);
  }
  return ok ? out : vbe_dlog_native(x);
}

#endif  // VBE_SF64_CUH
