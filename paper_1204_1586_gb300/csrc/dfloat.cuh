// Double-float ("double-single") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, giving a
// significand of about 48 bits.  Built from error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2): s + e == a + b exactly;
//   TwoProd via FMA (Dekker 1971 with a fused multiply-add): p + e == a * b exactly;
// with the add/multiply/divide/sqrt compositions of the double-double
// literature (Hida, Li, Bailey, "Algorithms for quad-double precision
// floating point arithmetic", 2001), written here for float pairs.
// The _rn intrinsics keep the compiler from fusing the compensation terms.
#pragma once

namespace cpg {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// a * b for a float b (one fewer cross term).
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// acc + a * b with a, b floats: the product is exact before the addition.
__device__ __forceinline__ df df_add_prod_ff(df acc, float a, float b) { return df_add(acc, two_prod(a, b)); }

__device__ __forceinline__ df df_sqrt(df a) {
  if (a.hi <= 0.0f) return df{0.0f, 0.0f};
  const float s = __fsqrt_rn(a.hi);
  const df r = df_sub(a, two_prod(s, s));        // a - s^2
  return quick_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}

// 1 / sqrt(a) for a > 0: FP32 reciprocal-sqrt seed y0, then one Newton step
// y = y0 + y0 (1 - a y0^2) / 2.  The residual e = 1 - a y0^2 is formed in
// double-float (y0^2 exactly by TwoProd); the small correction y0 e / 2 needs
// only float precision, so the result carries about twice the seed's bits.
__device__ __forceinline__ df df_rsqrt(df a) {
  const float y0 = rsqrtf(a.hi);
  const df e = df_sub(df_make(1.f), df_mul(a, two_prod(y0, y0)));
  return quick_two_sum(y0, __fmul_rn(__fmul_rn(y0, e.hi), 0.5f));
}

// 1 / a for a normal, positive or negative (not zero, not subnormal): the
// hardware's approximate reciprocal y0 of a.hi (relative error e ~ 2^-23),
// then the Newton-Raphson correction carried to second order,
//   1 / a = y0 / (1 - e) = y0 (1 + e + e^2 + ...),  e = 1 - a y0,
// where e is formed by two fused multiply-adds (1 - a.hi y0 is exact in one
// FMA because a.hi y0 is within 2^-22 of 1; a.lo y0 is then subtracted), so
// the truncation is e^3 ~ 2^-69 and the result carries the double-float's
// precision.  The dependent chain is one approximate reciprocal and five FP32
// operations.
__device__ __forceinline__ df df_rcp(df a) {
  float y0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a.hi));
  float e = __fmaf_rn(-a.hi, y0, 1.f);
  e = __fmaf_rn(-a.lo, y0, e);
  const float c = __fmaf_rn(e, e, e);  // e + e^2
  return quick_two_sum(y0, __fmul_rn(y0, c));
}

// Compensated accumulation of a sum of products (Ogita, Rump, Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005, algorithm Dot2): each
// product is split exactly by TwoProd, the running float sum s is advanced by
// TwoSum, and every rounding error (of the products and of the additions) is
// added into the float c.  The result s + c is as accurate as a dot product
// evaluated in twice the working precision and then rounded; the dependent
// chain through s is one addition per term (c never feeds back into s).
struct dot2 {
  float s = 0.f, c = 0.f;
  // += a * b for floats a, b.
  __device__ __forceinline__ void add_ff(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, ep));
  }
  // += a * b for a float a and a double-float b (a * b.lo, two orders below
  // a * b.hi, goes into the error term by one fused multiply-add).
  __device__ __forceinline__ void add_fd(float a, df b) {
    add_ff(a, b.hi);
    c = __fmaf_rn(a, b.lo, c);
  }
  // += x^2 for a double-float x (2 x.hi x.lo into the error term; x.lo^2 is
  // below the result's precision).
  __device__ __forceinline__ void add_sq(df x) {
    add_ff(x.hi, x.hi);
    c = __fmaf_rn(__fmul_rn(2.f, x.hi), x.lo, c);
  }
  __device__ __forceinline__ df value() const { return two_sum(s, c); }
};

__device__ __forceinline__ double df_to_double(df a) { return double(a.hi) + double(a.lo); }

__device__ __forceinline__ df df_from_double(double d) {
  const float hi = float(d);
  return df{hi, float(d - double(hi))};
}

__device__ __forceinline__ df df_shfl_xor(df a, int o, int width = 32) {
  return df{__shfl_xor_sync(0xffffffffu, a.hi, o, width), __shfl_xor_sync(0xffffffffu, a.lo, o, width)};
}

}  // namespace cpg
