// Float-float (unevaluated pair of floats) arithmetic for the float64-accurate
// passes.  GB300 executes float64 at 1/64 of the float32 rate: a float64
// instruction occupies a sub-partition's float64 pipe for about 64 cycles even
// when one lane is active, so the per-entry float64-accurate work of the
// polish passes is written with float32 instructions instead.
#pragma once

#include "common.cuh"

namespace ibsn {

// a * b (float-float times float-float), about 2^-47 relative
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_scale2(FF a, float pow2) { return FF{a.hi * pow2, a.lo * pow2}; }

// 2^(j/64), j = 0..63, each rounded to a float-float pair (hi = fl32, lo =
// fl32 of the remainder); derived from ln 2 = sum_k 1/(k 2^k) in 80-digit
// decimal arithmetic.  The CPU test re-derives them.
__device__ const float2 kExp2Tab64[64] = {
    {0x1p+0f, 0.0f},
    {0x1.02c9a4p+0f, -0x1.887fap-28f},
    {0x1.059b0ep+0f, -0x1.9d4f52p-25f},
    {0x1.087452p+0f, -0x1.e2990ep-26f},
    {0x1.0b5586p+0f, 0x1.9f3122p-25f},
    {0x1.0e3ec4p+0f, -0x1.a585ccp-25f},
    {0x1.11301ep+0f, -0x1.fdb496p-25f},
    {0x1.1429aap+0f, 0x1.d525bcp-25f},
    {0x1.172b84p+0f, -0x1.c15742p-27f},
    {0x1.1a35bep+0f, 0x1.6df96ep-25f},
    {0x1.1d4874p+0f, -0x1.d2e8cap-25f},
    {0x1.2063b8p+0f, 0x1.0c519ap-25f},
    {0x1.2387a6p+0f, 0x1.ceac48p-25f},
    {0x1.26b456p+0f, 0x1.789f38p-26f},
    {0x1.29e9ep+0f, -0x1.5c0424p-25f},
    {0x1.2d285ap+0f, 0x1.b900c2p-26f},
    {0x1.306fep+0f, 0x1.4636e2p-25f},
    {0x1.33c08cp+0f, -0x1.b37d2p-25f},
    {0x1.371a74p+0f, -0x1.18aac6p-25f},
    {0x1.3a7db4p+0f, -0x1.634c02p-25f},
    {0x1.3dea64p+0f, 0x1.824684p-25f},
    {0x1.4160a2p+0f, 0x1.f72e2ap-28f},
    {0x1.44e086p+0f, 0x1.8624b4p-30f},
    {0x1.486a2cp+0f, -0x1.47d866p-25f},
    {0x1.4bfdaep+0f, -0x1.593abcp-25f},
    {0x1.4f9b28p+0f, -0x1.2c5a6cp-25f},
    {0x1.5342b6p+0f, -0x1.2c561p-25f},
    {0x1.56f474p+0f, -0x1.295b04p-25f},
    {0x1.5ab07ep+0f, -0x1.5bd5ecp-27f},
    {0x1.5e76f2p+0f, -0x1.4a5bd6p-25f},
    {0x1.6247ecp+0f, -0x1.f8b55p-25f},
    {0x1.662388p+0f, 0x1.2a9112p-27f},
    {0x1.6a09e6p+0f, 0x1.9fcef4p-26f},
    {0x1.6dfb24p+0f, -0x1.cd72e8p-27f},
    {0x1.71f75ep+0f, 0x1.1d8beep-25f},
    {0x1.75feb6p+0f, -0x1.37b306p-25f},
    {0x1.7a1148p+0f, -0x1.829fdp-25f},
    {0x1.7e2f34p+0f, -0x1.261634p-25f},
    {0x1.82589ap+0f, -0x1.accc7cp-26f},
    {0x1.868d9ap+0f, -0x1.2edb44p-26f},
    {0x1.8ace54p+0f, 0x1.15506ep-27f},
    {0x1.8f1aeap+0f, -0x1.baa232p-26f},
    {0x1.93737cp+0f, -0x1.e64744p-25f},
    {0x1.97d82ap+0f, -0x1.0d8d84p-31f},
    {0x1.9c4918p+0f, 0x1.51f848p-27f},
    {0x1.a0c668p+0f, -0x1.2886a6p-26f},
    {0x1.a5503cp+0f, -0x1.b83b54p-25f},
    {0x1.a9e6b6p+0f, -0x1.50c048p-25f},
    {0x1.ae89fap+0f, -0x1.a94b14p-26f},
    {0x1.b33a2cp+0f, -0x1.ec3a82p-26f},
    {0x1.b7f77p+0f, -0x1.a09438p-25f},
    {0x1.bcc1eap+0f, -0x1.f687c6p-25f},
    {0x1.c199bep+0f, -0x1.3d56b2p-27f},
    {0x1.c67f12p+0f, 0x1.cafa2ap-25f},
    {0x1.cb720ep+0f, -0x1.8837ccp-27f},
    {0x1.d072d4p+0f, 0x1.40f13p-25f},
    {0x1.d5818ep+0f, -0x1.822dbcp-27f},
    {0x1.da9e6p+0f, 0x1.ed9942p-27f},
    {0x1.dfc974p+0f, -0x1.908c94p-25f},
    {0x1.e502eep+0f, 0x1.e2cffep-26f},
    {0x1.ea4afap+0f, 0x1.52486cp-27f},
    {0x1.efa1bep+0f, 0x1.cc2b44p-25f},
    {0x1.f50766p+0f, -0x1.246ebp-26f},
    {0x1.fa7c18p+0f, 0x1.9e90d8p-28f}};

// exp(x) of a float-float x <= 0 by the table-driven method of Tang (ACM TOMS
// 15, 1989), written in float-float: x = (64 e + j) ln2/64 + r with
// |r| <= ln2/128 (three-part Cody-Waite reduction, ln2/64 = L1 + L2 + L3 with
// a 9-bit L1 so that k L1 is exact for |k| < 2^15), exp(x) = 2^e 2^(j/64)
// exp(r), exp(r) = 1 + r + r^2/2 + r^3/6 + [r^4/24 + r^5/120 + r^6/720] (the
// bracket in float; the omitted r^7/5040 is below 3e-20).  Relative error
// about 2^-46 while 2^e stays a normal float (x > -87); the result is 0 for
// x < about -87.3 (those entries are below 2^-126 of the row maximum here).
__device__ __forceinline__ FF ff_exp(FF x) {
  constexpr float kInvLn2_64 = 0x1.715476p+6f;  // 64 / ln 2
  constexpr float L1 = 0x1.63p-7f;
  constexpr float L2 = -0x1.bd0106p-19f;
  constexpr float L3 = 0x1.cf79acp-46f;
  constexpr float C6h = 0x1.555556p-3f, C6l = -0x1.555556p-28f;  // 1/6
  const float kf = rintf(x.hi * kInvLn2_64);
  const int k = (int)kf;
  const int e = k >> 6, j = k & 63;
  if (e < -125) return FF{0.f, 0.f};
  // r = x - k (L1 + L2 + L3)
  const float t1 = fmaf(-kf, L1, x.hi);  // exact: k L1 has at most 24 bits
  const float p2 = kf * L2;
  const float e2 = fmaf(kf, L2, -p2);
  FF r = ff_two_sum(t1, -p2);
  // x.lo can be far above ulp(r.hi) once |x| is large: add it exactly too,
  // so that every term left for the low word is below ulp(r.hi)
  const FF s0 = ff_two_sum(r.hi, x.lo);
  r = ff_fast_two_sum(s0.hi, s0.lo + ((r.lo - e2) - kf * L3));
  const FF r2 = ff_mul(r, r);
  const FF r3 = ff_mul(r2, r);
  const float rh = r.hi;
  const float tail = (rh * rh) * (rh * rh) * (1.f / 24.f + rh * (1.f / 120.f + rh * (1.f / 720.f)));
  FF s = ff_add(ff_mul(r3, FF{C6h, C6l}), FF{tail, 0.f});
  s = ff_add(s, ff_scale2(r2, 0.5f));
  s = ff_add(s, r);
  s = ff_add(FF{1.f, 0.f}, s);
  const float2 tj = __ldg(kExp2Tab64 + j);
  const FF v = ff_mul(s, FF{tj.x, tj.y});
  return ff_scale2(v, __int_as_float((e + 127) << 23));
}

}  // namespace ibsn
