// dd.cuh -- double-double arithmetic for the one-time weight solve.
//
// A value is hi + lo with |lo| <= ulp(hi)/2 (about 32 significant digits).
// The error-free transformations are Knuth's TwoSum, Dekker's
// Fast-TwoSum and the FMA-based TwoProduct; addition, multiplication,
// division and square root follow the classic double-double algorithms of
// Dekker (1971) as popularised by Hida, Li & Bailey's QD library, written
// out here for this library.  exp and erf are evaluated from their Taylor /
// Maclaurin series (the arguments in the weight solve are below 1 in
// magnitude), with exp's argument first halved k times and the result
// squared back k times.
#pragma once

namespace kfvm {

struct dd {
  double hi, lo;
};

__host__ __device__ inline dd dd_make(double a) { return dd{a, 0.0}; }

__device__ inline dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return dd{s, e};
}

__device__ inline dd fast_two_sum(double a, double b) {  // requires |a| >= |b|
  double s = __dadd_rn(a, b);
  double e = __dsub_rn(b, __dsub_rn(s, a));
  return dd{s, e};
}

__device__ inline dd two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  double e = __fma_rn(a, b, -p);
  return dd{p, e};
}

__device__ inline dd operator+(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ inline dd operator-(dd x) { return dd{-x.hi, -x.lo}; }
__device__ inline dd operator-(dd x, dd y) { return x + (-y); }

__device__ inline dd operator*(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  p.lo = __fma_rn(x.hi, y.lo, p.lo);
  p.lo = __fma_rn(x.lo, y.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ inline dd operator*(dd x, double y) {
  dd p = two_prod(x.hi, y);
  p.lo = __fma_rn(x.lo, y, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ inline dd operator/(dd x, dd y) {
  double q1 = __ddiv_rn(x.hi, y.hi);
  dd r = x - y * q1;
  double q2 = __ddiv_rn(r.hi, y.hi);
  r = r - y * q2;
  double q3 = __ddiv_rn(r.hi, y.hi);
  dd q = fast_two_sum(q1, q2);
  return q + dd_make(q3);
}

__device__ inline dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd{0.0, 0.0};
  double x = __dsqrt_rn(a.hi);
  // one Newton step in double-double: x + (a - x^2) / (2x)
  dd xx = dd_make(x);
  dd r = (a - xx * xx) / dd_make(2.0 * x);
  return xx + r;
}

__device__ inline bool dd_lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ inline dd dd_abs(dd a) { return (a.hi < 0.0 || (a.hi == 0.0 && a.lo < 0.0)) ? -a : a; }

// pi to double-double precision: 3.14159265358979323846264338327950288...
__device__ inline dd dd_pi() { return dd{3.141592653589793116, 1.2246467991473532e-16}; }

// exp(x) for |x| <= 4: halve the argument 6 times, Taylor series to 1e-34, square back.
__device__ inline dd dd_exp(dd x) {
  const int k = 6;
  dd y = x * (1.0 / 64.0);  // exact scaling by a power of two
  dd term = dd_make(1.0), sum = dd_make(1.0);
  for (int n = 1; n <= 16; ++n) {
    term = term * y / dd_make((double)n);
    sum = sum + term;
  }
  for (int i = 0; i < k; ++i) sum = sum * sum;
  return sum;
}

// erf(x) for |x| <= 1.5 from its Maclaurin series 2/sqrt(pi) sum (-1)^n x^(2n+1) / (n! (2n+1)).
__device__ inline dd dd_erf(dd x) {
  dd x2 = x * x;
  dd p = x;  // (-1)^n x^(2n+1) / n!
  dd sum = x;
  for (int n = 1; n <= 60; ++n) {
    p = -(p * x2) / dd_make((double)n);
    dd t = p / dd_make((double)(2 * n + 1));
    sum = sum + t;
    if (fabs(t.hi) < 1e-36 * fabs(sum.hi)) break;
  }
  return sum * (dd_make(2.0) / dd_sqrt(dd_pi()));
}

}  // namespace kfvm
