// Float-float ("df") arithmetic for the value kernels.
//
// FP64 on this part issues at 1/73 of the FP32 rate, and every conversion that involves a 64-bit type
// (double <-> float, int64 <-> float) runs at the FP64 rate too. The value kernels therefore keep
// all arithmetic on the FP32 and INT32 pipes: an unevaluated sum hi + lo of two floats carries ~48
// significant bits, which meets the 1e-12 relative parity bound with a wide margin.
//
// Building blocks are the classic error-free transformations: Knuth's two-sum, the FMA form of
// Dekker's two-product, and the fast two-sum for ordered operands (Dekker 1971; Knuth TAOCP vol. 2).
// Rounded intrinsics (__fadd_rn, __fmul_rn) keep the compiler from contracting them into FMAs.
//
// Doubles enter through an exact split into three floats done with integer operations only (see
// split3), and leave as one correctly rounded FP64 add of the two parts (df_to_double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

// 8-byte aligned so that one 64-bit shared-memory access moves a pair
struct __align__(8) df2 {
  float h, l;
};

__device__ __forceinline__ df2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df2 df_from(float a) { return {a, 0.0f}; }

// Error bounds below are for pairs with |lo| <= u |hi| (u = 2^-24; the routines here return such pairs,
// except df_from_double_shift: |lo| < 2u |hi|), to first order in u, with no result leaving the normal
// float range.
// df_add: |error| <= 3 u^2 (|a| + |b|): the leading parts' sum is exact (two-sum); the trailing parts' sum
// (size <= u (|a| + |b|)) and its sum with the two-sum's error (size <= 2u (|a| + |b|)) round once each; the
// final fast two-sum is exact. There is no bound relative to |a + b| itself when they cancel.
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const df2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }
// One step of a running sum: the operations of df_add, renormalised every step, so that the sum of m
// terms c_j stays within 3 u^2 sum_j (|partial sum before j| + |c_j|) <= 3 m u^2 sum_j |c_j| (u = 2^-24).
// (Carrying the trailing part unnormalised would let it grow with every step and the bound with m^2.)
__device__ __forceinline__ df2 df_acc(df2 a, df2 b) { return df_add(a, b); }

// df_mul: |error| <= 6 u^2 |a b|: the residual of a.h b.h is exact (FMA); adding a.h b.l, then a.l b.h,
// rounds sums of size <= 2u |ab| and 3u |ab|; the dropped a.l b.l is <= u^2 |ab|.
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// df_mul_f: |error| <= 2 u^2 |a b| (one rounding of a sum of size <= 2u |ab|).
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return fast_two_sum(p, e);
}
// scaling by a power of two (exact; any other factor needs df_mul_f)
__device__ __forceinline__ df2 df_scale(df2 a, float pow2) { return {__fmul_rn(a.h, pow2), __fmul_rn(a.l, pow2)}; }

// 1/a: a float reciprocal r refined by one Newton step carried in df. Relative error <= 9 u^2: with
// eps = a r - 1 (|eps| <= 2u), the step drops eps^2 (4 u^2) and rounds 1 - a.h r (u^2), the sum with a.l r
// (2 u^2) and r t (2 u^2). For |a.l| up to 2u |a.h| (a pair that is not renormalised) the bound is 16 u^2.
__device__ __forceinline__ df2 df_recip(df2 a) {
  const float r = __frcp_rn(a.h);
  float t = __fmaf_rn(-a.h, r, 1.0f);
  t = __fmaf_rn(-a.l, r, t);
  return fast_two_sum(r, __fmul_rn(r, t));
}

// Sum over m of a_m * b_m for df vectors. |error| <= g_D u^2 sum_m |a_m b_m| with g_2 = 19, g_3 = 36,
// g_4 = 56: the leading products and their running sum are exact (residuals and two-sum errors); everything
// else gathers in one float t, whose 4D - 2 roundings are each at most u times a partial sum of terms of
// total size <= (D + 2) u sum |a_m b_m| (counted term by term, by position); the dropped a.l b.l add u^2,
// and the final fast two-sum, inexact only when the leading sum has cancelled below |t|, at most u |t|.
template <int D>
__device__ __forceinline__ df2 df_dot(const df2 (&a)[D], const df2 (&b)[D]) {
  // leading products exact (product + FMA residual), their sum by two-sum; residuals, cross terms and
  // the sum's own errors gathered in one float; one renormalisation at the end
  float s = __fmul_rn(a[0].h, b[0].h);
  float t = __fmaf_rn(a[0].h, b[0].h, -s);
  t = __fmaf_rn(a[0].h, b[0].l, t);
  t = __fmaf_rn(a[0].l, b[0].h, t);
#pragma unroll
  for (int m = 1; m < D; ++m) {
    const float p = __fmul_rn(a[m].h, b[m].h);
    const float e = __fmaf_rn(a[m].h, b[m].h, -p);
    const df2 u = two_sum(s, p);
    s = u.h;
    t = __fadd_rn(t, __fadd_rn(u.l, e));
    t = __fmaf_rn(a[m].h, b[m].l, t);
    t = __fmaf_rn(a[m].l, b[m].h, t);
  }
  return fast_two_sum(s, t);
}
// a0 b0 - a1 b1, the same way
__device__ __forceinline__ df2 df_dot2m(df2 a0, df2 b0, df2 a1, df2 b1) {
  const df2 A[2] = {a0, df_neg(a1)}, B[2] = {b0, b1};
  return df_dot<2>(A, B);
}

// ---- doubles in -----------------------------------------------------------------------------------

// Float with the given (unbiased) power of two, for exponents in the normal float range.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Exact split x = a + b + c into three floats with the sign of x, from the IEEE bits only:
// a = the leading 24 significant bits (truncated), b = the next 23, c = the last 6.
// Exact for |x| in [2^-80, 2^127] and for 0; smaller magnitudes flush b and c to zero and tiny x to 0.
struct f3 {
  float a, b, c;
};
__device__ __forceinline__ f3 split3(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ff);
  const uint32_t sign = hi & 0x80000000u;
  f3 r;
  if (E < 897 || E > 1150) {  // outside the float range for the leading part (includes 0 and subnormals)
    r.a = 0.0f;
    r.b = 0.0f;
    r.c = 0.0f;
    return r;
  }
  r.a = __uint_as_float(sign | ((uint32_t)(E - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  const uint32_t R = lo & 0x1fffffffu;  // 29 remaining bits, weight 2^(E-1075)
  const uint32_t bi = R >> 6, ci = R & 63u;
  const float bf = __fsub_rn(__uint_as_float(0x4b000000u | bi), 8388608.0f);  // exact, bi < 2^23
  const float cf = __fsub_rn(__uint_as_float(0x4b000000u | ci), 8388608.0f);
  const int e0 = E - 1075;
  const float s1 = (e0 + 6 >= -126) ? pow2f(e0 + 6) : 0.0f;
  const float s0 = (e0 >= -126) ? pow2f(e0) : 0.0f;
  const float sg = sign ? -1.0f : 1.0f;
  r.b = __fmul_rn(__fmul_rn(bf, s1), sg);
  r.c = __fmul_rn(__fmul_rn(cf, s0), sg);
  return r;
}

// df approximation of a double (relative error <= u^2 = 2^-48: the middle and last parts, 29 bits in all,
// rounded to one float), renormalised
__device__ __forceinline__ df2 df_from_double(double x) {
  const f3 s = split3(x);
  return fast_two_sum(s.a, __fadd_rn(s.b, s.c));
}

// df approximation of a double that need not be exact (relative error <= u^2 = 2^-48): the leading 24 bits
// from the IEEE bits, the remaining 29 bits through one int32->float conversion.
__device__ __forceinline__ df2 df_from_double_fast(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ff);
  if (E < 897 || E > 1150) return df2{(float)0.0f, 0.0f};
  const uint32_t sign = hi & 0x80000000u;
  const float a = __uint_as_float(sign | ((uint32_t)(E - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  const int e0 = E - 1075;
  const float r = (e0 >= -126) ? __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), pow2f(e0)) : 0.0f;
  return fast_two_sum(a, sign ? -r : r);
}

// ---- element-frame conversions ----------------------------------------------------------------------

// |x| as an ordered integer: the IEEE high word without the sign (compares like |x| to 2^-20 relative).
__device__ __forceinline__ uint32_t abs_hiword(double x) { return (uint32_t)__double2hiint(x) & 0x7fffffffu; }

// Unbiased exponent of the largest magnitude among doubles whose abs_hiword maximum is m (m = 0: all
// zero, gives -1023).
__device__ __forceinline__ int exponent_of_hiword(uint32_t m) { return (int)(m >> 20) - 1023; }

// x * 2^-s as a float pair, from the IEEE bits with integer operations only: the leading part is the
// top 24 significant bits (truncated, exponent shifted by s), the trailing part the remaining 29 bits
// through one int32 -> float conversion (rounded to 24 bits: 5 bits dropped, an error of at most 16 units
// of the double's last place), so the pair carries x 2^-s to u^2 = 2^-48 relative. Both parts have the
// sign of x and |lo| < ulp(hi) <= 2u |hi| (the leading part is truncated, not rounded). Gives 0 when x 2^-s is below 2^-126 (for
// the element's own edges, which are scaled so that the largest component is in [1, 2), that is below
// 2^-126 of the element's size).
__device__ __forceinline__ df2 df_from_double_shift(double x, int s) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const int E = (int)((hw >> 20) & 0x7ffu);
  const int fe = E - s - 896;  // float exponent field of the leading part
  const uint32_t sg = hw & 0x80000000u;
  df2 r = {0.0f, 0.0f};
  if (E != 0 && fe > 0 && fe < 255) {
    r.h = __uint_as_float(sg | ((uint32_t)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const int pe = fe - 52;  // float exponent field of the weight of the double's last bit
    if (pe > 0) r.l = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float(sg | ((uint32_t)pe << 23)));
  }
  return r;
}

// v * 2^e for a float pair (exact while both parts stay normal); e in [-126, 127].
__device__ __forceinline__ df2 df_ldexp(df2 v, int e) {
  const float p = __int_as_float((e + 127) << 23);
  return {__fmul_rn(v.h, p), __fmul_rn(v.l, p)};
}

// The range the float-float results keep their precision in. A result's trailing part may be far below
// its leading part; once it leaves the normal float range (2^-126) it is lost, an absolute error of up to
// 2^-126, which is below 2^-42 of a result of magnitude 2^-84 or more. So a result is in range when its
// terms are of magnitude in [2^-84, 2^120] (sums of a row's contributions then stay finite); a product
// of nonzero factors must not be 0 (it flushed). The check is made on the magnitude of a result's terms,
// never on a sum of signed terms: such a sum may cancel far below its terms (a normal of an axis-aligned
// face whose exact component is 0 comes out as a residue of its terms' roundings), which loses nothing
// against the terms the error is measured by. Scale exponents (the power of two an element's normalised
// result is multiplied by) are kept within [-100, 100].
__device__ __forceinline__ bool df_prod_in_range(df2 v, bool nonzero_factors) {
  const float a = fabsf(v.h);
  return a <= 0x1p120f && (a >= 0x1p-84f || (a == 0.0f && !nonzero_factors));
}
// A term magnitude m (a float product of the magnitudes of a result's factors, formed in the element's
// frame) that the result is then scaled by 2^e: in range when m 2^e is within [2^-84, 2^120] and m itself
// is normal (a subnormal or zero m from nonzero factors has flushed already); m = 0 from a zero factor
// is in range.
__device__ __forceinline__ bool mag_in_range(float m, int e, bool nonzero_factors) {
  const float a = fabsf(m);
  if (a == 0.0f) return !nonzero_factors;
  if (!(a <= 0x1p127f) || a < 0x1p-126f) return false;
  const int x = (int)((__float_as_uint(a) >> 23) & 0xffu) - 127 + e;
  return x >= -84 && x < 120;
}
__device__ __forceinline__ bool scale_in_range(int e) { return e >= -100 && e <= 100; }
// Binary exponent of |a| for a normal float (0 and subnormals give -127), and the range test of a term
// whose factors' exponents sum to x (the same [2^-84, 2^120] range, up to a factor 2 per factor).
__device__ __forceinline__ int fexp(float a) { return (int)((__float_as_uint(a) >> 23) & 0xffu) - 127; }
__device__ __forceinline__ bool exp_in_range(int x) { return x >= -84 && x < 120; }

// xj - xi as df, from exact three-float splits: the difference of the leading parts and of the
// middle parts are formed exactly with two-sum, so the result is within 4 u^2 |xj - xi| + 2^-67 max|x|
// however close xi and xj are (three roundings of trailing sums of size <= 2u |xj - xi|, and the
// difference of the last parts, each below 2^-45 |x|); the second term stays below u^2 |xj - xi| while
// the coordinates are within 2^19 edge lengths of the origin.
__device__ __forceinline__ df2 f3_diff(const f3& xj, const f3& xi) {
  const df2 A = two_sum(xj.a, -xi.a);
  const df2 B = two_sum(xj.b, -xi.b);
  const float C = __fsub_rn(xj.c, xi.c);
  const df2 S = two_sum(A.h, B.h);
  return fast_two_sum(S.h, __fadd_rn(__fadd_rn(S.l, A.l), __fadd_rn(B.l, C)));
}

// ---- doubles out ----------------------------------------------------------------------------------

// The exact double of a float, assembled from its bits with 32-bit integer operations (no conversion
// instruction). Zero and float subnormals give a signed zero (they only ever appear as the low part
// of a float-float, below any result's precision); infinities and NaNs keep their class.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t sg = u & 0x80000000u;
  const uint32_t m = u & 0x7fffffu;
  uint32_t hi = sg | ((e + 896u) << 20) | (m >> 3);
  uint32_t lo = m << 29;
  hi = (e == 0u) ? sg : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sg | 0x7ff00000u | (m ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// hi + lo rounded to the nearest double: both parts are exact doubles, so one FP64 add rounds their
// sum correctly. The FP64 unit is otherwise idle in these kernels.
__device__ __forceinline__ double df_to_double(df2 v) { return __dadd_rn(f2d_bits(v.h), f2d_bits(v.l)); }

// ---- sin(pi r), cos(pi r) ---------------------------------------------------------------------------

// The table passed to the functions below holds sin(pi k / 2048) and cos(pi k / 2048), k = 0..1024,
// each as a (hi, lo) float pair: float4(sin.hi, sin.lo, cos.hi, cos.lo).
constexpr int kSinTabN = 1024;

// sin(theta) and cos(theta) for a small df theta (|theta| < pi/512): theta - theta^3/6 + theta^5/120 with the
// cubic term in float-float, 1 - theta^2/2 + theta^4/24 with theta^2 in float-float (the next terms are below
// 2^-57 relative); no term cancels another.
__device__ __forceinline__ void df_sincos_series(df2 th, df2& s, df2& c) {
  df2 sq = two_prod(th.h, th.h);
  sq.l = __fmaf_rn(2.0f * th.h, th.l, sq.l);
  const float t2 = sq.h;
  const df2 SIXTH = {0.1666666716337204f, -4.9670538793e-09f};
  const df2 c3 = df_mul(df_mul(th, sq), SIXTH);  // theta^3 / 6
  const float t5 = __fmul_rn(__fmul_rn(th.h, __fmul_rn(t2, t2)), 1.0f / 120.0f);
  s = df_add(th, df2{-c3.h, __fsub_rn(t5, c3.l)});
  const df2 one_m = two_sum(1.0f, -0.5f * sq.h);
  c = fast_two_sum(one_m.h, __fadd_rn(one_m.l, __fadd_rn(-0.5f * sq.l, __fmul_rn(__fmul_rn(t2, t2), 1.0f / 24.0f))));
}

// sin(pi r) and cos(pi r) for a df r with |r| <= 1/2, table-driven: r = k/2048 + d with k = rint(2048 r),
// |d| <= 1/4096, the Taylor series of sin and cos of theta = pi d combined with the table's sin, cos(pi k/2048)
// by the angle-addition formulas. Where the two terms of an addition have opposite signs (d against k for the
// sine; d with k for the cosine) their magnitudes add up to at most (|k| + 1/2) / (|k| - 1/2) times the
// result's: 3 at |k| = 1 (sine) or 1023 (cosine), 7/5 from |k| = 3 on (and 1 at k = 0, where the sine is the
// series itself). df_sincospi_small uses this step for every r (one path, no branches: it is evaluated at
// every quadrature point); the staged per-vertex values (sincospi_half) take the series directly at both
// ends, where the ratio would exceed 7/5.
// The table step: sin and cos of pi (k/2048 + d) for |k| <= 1024 and |d| <= 1/4096, d a float pair
// accurate to 2^-48 of itself.
__device__ __forceinline__ void df_sincospi_table(int k, df2 dlt, const float4* __restrict__ tab, df2& s, df2& c) {
  const df2 PI = {3.14159274101257324f, -8.74227765734758577e-8f};
  const df2 th = df_mul(PI, dlt);
  const float t2 = __fmul_rn(th.h, th.h);
  // sin(theta) = theta (1 - theta^2/6 + theta^4/120)
  const float q = __fmul_rn(t2, __fmaf_rn(t2, -1.0f / 120.0f, 1.0f / 6.0f));
  const df2 sn = fast_two_sum(th.h, __fmaf_rn(-th.h, q, th.l));
  // cos(theta) = 1 - theta^2/2 + theta^4/24, with theta^2 in df
  df2 sq = two_prod(th.h, th.h);
  sq.l = __fmaf_rn(2.0f * th.h, th.l, sq.l);
  const df2 one_m = two_sum(1.0f, -0.5f * sq.h);
  const float tail = __fadd_rn(-0.5f * sq.l, __fmul_rn(__fmul_rn(t2, t2), 1.0f / 24.0f));
  const df2 cs = fast_two_sum(one_m.h, __fadd_rn(one_m.l, tail));
  const int ak = min(k < 0 ? -k : k, kSinTabN);  // |k| <= 1024 for |r| <= 1/2; the bound keeps the read in the table
  const float4 e = tab[ak];
  df2 Sk = {e.x, e.y}, Ck = {e.z, e.w};
  if (k < 0) Sk = df_neg(Sk);
  s = df_add(df_mul(Sk, cs), df_mul(Ck, sn));
  c = df_sub(df_mul(Ck, cs), df_mul(Sk, sn));
}

__device__ __forceinline__ void df_sincospi_small(df2 r, const float4* __restrict__ tab, df2& s, df2& c) {
  const float kf = rintf(__fmul_rn(r.h, 2048.0f));
  df_sincospi_table((int)kf, fast_two_sum(__fsub_rn(r.h, __fmul_rn(kf, 1.0f / 2048.0f)), r.l), tab, s, c);
}

// sin(pi x) and cos(pi x) for a df x of any size (reduction as in df_sinpi below).
__device__ __forceinline__ void df_sincospi(df2 x, const float4* __restrict__ tab, df2& s, df2& c) {
  const float n = rintf(x.h);
  df2 r = fast_two_sum(__fsub_rn(x.h, n), x.l);
  const float n2 = rintf(r.h);
  r = fast_two_sum(__fsub_rn(r.h, n2), r.l);
  df_sincospi_small(r, tab, s, c);
  if ((__float2int_rn(n) + __float2int_rn(n2)) & 1) {
    s = df_neg(s);
    c = df_neg(c);
  }
}

// sin(pi x) for a df x of any size: x = n + r exactly with n = rint(x.h), then the parity of n.
__device__ __forceinline__ df2 df_sinpi(df2 x, const float4* __restrict__ tab) {
  const float n = rintf(x.h);
  df2 r = fast_two_sum(__fsub_rn(x.h, n), x.l);
  // x.h - n is exact (Sterbenz, or n == 0); r.h + r.l may still reach just past 1/2
  const float n2 = rintf(r.h);
  r = fast_two_sum(__fsub_rn(r.h, n2), r.l);
  df2 s, c;
  df_sincospi_small(r, tab, s, c);
  return ((__float2int_rn(n) + __float2int_rn(n2)) & 1) ? df_neg(s) : s;
}

}  // namespace fem
