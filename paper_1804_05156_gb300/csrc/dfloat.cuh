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
// split3), and leave through an integer reassembly of hi + lo into IEEE double bits (df_to_double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

struct df2 {
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

__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  const df2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }
// accumulate without renormalising (the result's lo may exceed half an ulp of hi; renormalise later)
__device__ __forceinline__ df2 df_acc(df2 a, df2 b) {
  const df2 s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ df2 df_norm(df2 a) { return fast_two_sum(a.h, a.l); }

__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return fast_two_sum(p, e);
}
// scaling by a power of two (exact; any other factor needs df_mul_f)
__device__ __forceinline__ df2 df_scale(df2 a, float pow2) { return {__fmul_rn(a.h, pow2), __fmul_rn(a.l, pow2)}; }

// 1/a: a float reciprocal refined by one Newton step carried in df (error ~2^-46 relative)
__device__ __forceinline__ df2 df_recip(df2 a) {
  const float r = __frcp_rn(a.h);
  float t = __fmaf_rn(-a.h, r, 1.0f);
  t = __fmaf_rn(-a.l, r, t);
  return fast_two_sum(r, __fmul_rn(r, t));
}

// Sum over m of a_m * b_m for df vectors, relative error ~2^-46 against sum_m |a_m b_m|.
template <int D>
__device__ __forceinline__ df2 df_dot(const df2 (&a)[D], const df2 (&b)[D]) {
  df2 s = df_mul(a[0], b[0]);
#pragma unroll
  for (int m = 1; m < D; ++m) s = df_add(s, df_mul(a[m], b[m]));
  return s;
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

// df approximation of a double (relative error <= 2^-47): the first two parts of split3, renormalised
__device__ __forceinline__ df2 df_from_double(double x) {
  const f3 s = split3(x);
  return fast_two_sum(s.a, __fadd_rn(s.b, s.c));
}

// xj - xi as df, from exact three-float splits: the difference of the leading parts and of the
// middle parts are formed exactly with two-sum, so the result is accurate to ~2^-47 of |xj - xi|
// however close xi and xj are.
__device__ __forceinline__ df2 f3_diff(const f3& xj, const f3& xi) {
  const df2 A = two_sum(xj.a, -xi.a);
  const df2 B = two_sum(xj.b, -xi.b);
  const float C = __fsub_rn(xj.c, xi.c);
  const df2 S = two_sum(A.h, B.h);
  return fast_two_sum(S.h, __fadd_rn(__fadd_rn(S.l, A.l), __fadd_rn(B.l, C)));
}

// ---- doubles out ----------------------------------------------------------------------------------

// hi + lo rounded to a double (error <= 1 ulp), with 32-bit integer operations and one float->int32
// conversion; no FP64 instruction.
__device__ __forceinline__ double df_to_double(df2 v) {
  v = fast_two_sum(v.h, v.l);
  const uint32_t hb = __float_as_uint(v.h);
  const int eh = (int)((hb >> 23) & 0xff);
  if (eh == 0 || eh == 255) {  // zero, float subnormal or non-finite hi: hi alone decides
    if (eh == 255) {
      const uint32_t m = hb & 0x7fffffu;
      return __hiloint2double((int)((hb & 0x80000000u) | 0x7ff00000u | (m ? 0x80000u : 0u)), 0);
    }
    // subnormal or zero float: exact as a double through the bits
    if ((hb & 0x7fffffffu) == 0) return __hiloint2double((int)(hb & 0x80000000u), 0);
    const uint32_t m = hb & 0x7fffffu;
    const int lz = __clz(m) - 8;                       // shift to bring the leading 1 to bit 23
    const uint32_t mm = (m << lz) & 0x7fffffu;
    const int E = 1023 - 126 - lz;
    return __hiloint2double((int)((hb & 0x80000000u) | ((uint32_t)E << 20) | (mm >> 3)), (int)(mm << 29));
  }
  // mantissa of hi as a 53-bit integer: (1.m23) << 29; unit = 2^(eh - 127 - 52)
  uint32_t mhi = ((hb & 0x7fffffu) | 0x800000u) >> 3;  // top 21 bits -> bits 0..20 of the high word
  uint32_t mlo = (hb & 7u) << 29;
  // lo in the same units: |lo| <= 2^-24 |hi| -> |L| < 2^29
  const int k = 179 - eh;  // lo * 2^k is in those units
  float lf = v.l;
  int kk = k;
  // apply 2^k in two steps so each factor stays a normal float
  const int k1 = kk / 2, k2 = kk - k1;
  lf = __fmul_rn(__fmul_rn(lf, pow2f(k1)), pow2f(k2));
  const int L = __float2int_rn(lf);
  const bool neg = (hb & 0x80000000u) != 0;
  // magnitude M = mant(hi) + (neg ? -L : L) as a 64-bit value in two 32-bit words
  const int Ls = neg ? -L : L;
  uint64_t M = ((uint64_t)mhi << 32) | mlo;
  M = (uint64_t)((int64_t)M + (int64_t)Ls);
  int E = eh - 127 + 1023;
  if (M >> 53) {  // carried into bit 53: renormalise with round-half-even
    const uint64_t odd = M & 1u;
    M = (M >> 1) + (odd & ((M >> 1) & 1u));
    E += 1;
  } else if (!(M >> 52)) {  // borrowed below bit 52
    M <<= 1;
    E -= 1;
  }
  const uint64_t bits = ((uint64_t)(neg ? 1u : 0u) << 63) | ((uint64_t)E << 52) | (M & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// ---- sin(pi r), cos(pi r) ---------------------------------------------------------------------------

// The table passed to the functions below holds sin(pi k / 2048) and cos(pi k / 2048), k = 0..1024,
// each as a (hi, lo) float pair: float4(sin.hi, sin.lo, cos.hi, cos.lo).
constexpr int kSinTabN = 1024;

// sin(pi r) and cos(pi r) for a df r with |r| <= 1/2 (table-driven: r = k/2048 + d, then the Taylor
// series of sin and cos of theta = pi d, |theta| <= pi/4096, combined by the angle-addition formulas).
__device__ __forceinline__ void df_sincospi_small(df2 r, const float4* __restrict__ tab, df2& s, df2& c) {
  const float kf = rintf(__fmul_rn(r.h, 2048.0f));
  const df2 dlt = fast_two_sum(__fsub_rn(r.h, __fmul_rn(kf, 1.0f / 2048.0f)), r.l);
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
  const int k = (int)kf;
  const int ak = k < 0 ? -k : k;
  const float4 e = tab[ak];
  df2 Sk = {e.x, e.y}, Ck = {e.z, e.w};
  if (k < 0) Sk = df_neg(Sk);
  s = df_add(df_mul(Sk, cs), df_mul(Ck, sn));
  c = df_sub(df_mul(Ck, cs), df_mul(Sk, sn));
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
