// Exhaustive-style checks of sf64.cuh against the host's IEEE arithmetic.
// Usage: check <op> <count> <seed>; prints mismatches and max ulp error.
#include "host_shim.h"
#include "../../paper_1210_7774_b300/csrc/sf64_tables.h"
#include "../../paper_1210_7774_b300/csrc/sf64.cuh"
#include <cstdio>
#include <cstdlib>
#include <random>

static double rnd_double(std::mt19937_64& g, int emin, int emax) {
  unsigned long long m = g() & SF_M52;
  int e = emin + (int)(g() % (unsigned)(emax - emin + 1));
  unsigned long long s = (g() & 1) ? SF_SIGN : 0;
  return __longlong_as_double((long long)(s | ((unsigned long long)(e + 1023) << 52) | m));
}

static long long ulps(double a, double b) {
  long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if (ia < 0) ia = (long long)0x8000000000000000ull - ia;
  if (ib < 0) ib = (long long)0x8000000000000000ull - ib;
  long long d = ia - ib;
  return d < 0 ? -d : d;
}

int main(int argc, char** argv) {
  const char* op = argv[1];
  long long n = atoll(argv[2]);
  std::mt19937_64 g(atoll(argv[3]));
  long long bad = 0, maxu = 0, nonzero = 0;
  for (long long i = 0; i < n; ++i) {
    double a, b, got, want;
    int mode = (int)(g() % 8);
    if (!strcmp(op, "div")) {
      a = mode == 0 ? rnd_double(g, -1030, 1030) : rnd_double(g, -60, 60);
      b = mode == 1 ? rnd_double(g, -1030, 1030) : rnd_double(g, -60, 60);
      if (mode == 2) b = __longlong_as_double(__double_as_longlong(b) & ~0xFFFFFll);  // short mantissas
      if (mode == 3) a = b * (1.0 + (double)(g() % 1000) * 0x1p-52);                    // near-1 quotients
      if (mode == 4) { a = (double)(g() % 100000 + 1); b = (double)(g() % 1000 + 1); }   // exact quotients
      if (mode == 5) a = (g() & 1) ? -0.0 : 0.0;                                         // zero numerators
      if (mode == 6) {                                                                   // special operands
        const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1.0, -1.0, 0x1p-1074, -0x1p-1060};
        a = (g() & 1) ? sp[g() % 9] : a;
        b = sp[g() % 9];
      }
      got = vbe_ddiv(a, b);
      want = a / b;
      if (got == 0 && want == 0 && std::signbit(got) != std::signbit(want)) { got = 1; want = 2; }
    } else if (!strcmp(op, "sqrt")) {
      a = mode == 0 ? rnd_double(g, -1022, 1023) : std::fabs(rnd_double(g, -80, 80));
      if (mode == 1) { double r = (double)(g() % 94906265); a = r * r; }                  // perfect squares
      if (mode == 2) { double r = std::fabs(rnd_double(g, -20, 20)); a = r * r; }
      a = std::fabs(a);
      got = vbe_dsqrt(a);
      want = std::sqrt(a);
    } else if (!strcmp(op, "mul") || !strcmp(op, "add") || !strcmp(op, "sub")) {
      a = mode == 0 ? rnd_double(g, -1030, 1030) : rnd_double(g, -60, 60);
      b = mode == 1 ? rnd_double(g, -1030, 1030) : rnd_double(g, -60, 60);
      if (mode == 2) b = a * (1.0 + (double)((int)(g() % 64) - 32) * 0x1p-52);   // near-cancellation
      if (mode == 3) b = -a;                                                       // exact zero
      if (mode == 4) b = std::ldexp(b, -(int)(g() % 70));                         // wide exponent gaps
      if (mode == 5) { a = (double)(int64_t)(g() % 2000001) - 1000000; b = (double)(int64_t)(g() % 2001) - 1000; }
      if (mode == 6) { a = 0x1p1023 * (1 + (g() % 100) * 0x1p-52); b = a; }       // overflow edge
      if (!strcmp(op, "mul")) { got = vbe_dmul(a, b); want = a * b; }
      else if (!strcmp(op, "add")) { got = vbe_dadd(a, b); want = a + b; }
      else { got = vbe_dsub(a, b); want = a - b; }
      if (got == 0 && want == 0 && std::signbit(got) != std::signbit(want)) { got = 1; want = 2; }
    } else if (!strcmp(op, "mulk")) {
      // products by constants: powers of two (the integer path) and others
      a = mode == 0 ? rnd_double(g, -1030, 1030) : rnd_double(g, -60, 60);
      const int k = (int)(g() % 2101) - 1050;
      b = std::ldexp((g() & 1) ? -1.0 : 1.0, k < -1074 ? -1074 : k);
      if (mode == 1) b = std::ldexp((g() & 1) ? -1.0 : 1.0, (int)(g() % 9) - 4);
      if (mode == 2) a = std::ldexp(1.0 + (double)(g() % 1024) * 0x1p-10, (int)(g() % 40) - 1060);  // subnormal results
      if (mode == 3) a = std::ldexp(1.0 + (double)(g() % 1024) * 0x1p-10, (int)(g() % 40) + 990);   // overflow edge
      if (mode == 4) b = rnd_double(g, -8, 8);                                                        // not a power of two
      if (mode == 5) {
        const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 0x1p-1074, -0x1p-1060, 0x1p1023};
        a = sp[g() % 8];
        if (g() & 1) b = sp[g() % 8];
      }
      got = vbe_dmul_k(a, b);
      want = a * b;
      if (got == 0 && want == 0 && std::signbit(got) != std::signbit(want)) { got = 1; want = 2; }
    } else if (!strcmp(op, "cmp")) {
      const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1.0, -1.0, 0x1p-1074};
      a = mode < 2 ? sp[g() % 8] : rnd_double(g, -5, 5);
      b = mode < 3 ? sp[g() % 8] : (mode == 4 ? a : rnd_double(g, -5, 5));
      int gv = vbe_dlt(a, b) + 2 * vbe_dle(a, b) + 4 * vbe_deq(a, b) + 8 * vbe_dlt(b, a);
      int wv = (a < b) + 2 * (a <= b) + 4 * (a == b) + 8 * (b < a);
      got = gv; want = wv;
    } else if (!strcmp(op, "u53")) {
      unsigned long long v = g() >> (11 + (g() % 40));
      if (mode == 0) v = 0;
      got = vbe_u53_to_unit(v); want = (double)v * 0x1p-53;
      a = (double)v; b = 0;
    } else if (!strcmp(op, "exp")) {
      a = mode < 4 ? std::ldexp((double)(g() >> 11) * 0x1p-53 * 2 - 1, 10) : rnd_double(g, -45, 9);
      if (mode == 5) a = -std::fabs(a);
      got = vbe_dexp(a);
      want = (double)expl((long double)a);
    } else if (!strcmp(op, "log")) {
      a = mode < 3 ? std::fabs(rnd_double(g, -1022, 1023)) : std::fabs(rnd_double(g, -3, 3));
      if (mode == 3) a = 1.0 + ((double)(g() >> 11) * 0x1p-53 - 0.5) * 0x1p-6;   // near 1
      if (mode == 4) a = 1.0 + ((double)(g() >> 11) * 0x1p-53 - 0.5) * 0x1p-30;  // very near 1
      if (mode == 5) a = (double)(g() % 1000 + 96) / 128.0 * (1.0 + ((double)(g() >> 11) * 0x1p-53 - 0.5) * 0x1p-20);
      got = vbe_dlog(a);
      want = (double)logl((long double)a);
    } else {
      fprintf(stderr, "unknown op\n");
      return 2;
    }
    long long u = (std::isnan(got) && std::isnan(want)) ? 0 : ulps(got, want);
    if (u > maxu) maxu = u;
    if (u) ++nonzero;
    const long long tol = (!strcmp(op, "exp") || !strcmp(op, "log")) ? 1 : 0;
    if (u > tol) {
      if (bad < 5) printf("MISMATCH %s(%a, %a): got %a want %a\n", op, a, b, got, want);
      ++bad;
    }
  }
  printf("%s n=%lld mismatches=%lld max_ulp=%lld nonzero_ulp=%lld\n", op, n, bad, maxu, nonzero);
  return bad ? 1 : 0;
}
