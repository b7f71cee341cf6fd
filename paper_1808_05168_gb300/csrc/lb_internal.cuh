// lb_internal.cuh -- types and device helpers shared by the library's translation units.
//
// Populations of lattice i live at f + lat[i].f_off as (A, B) pairs, [link][z][x][species]
// (state_index; the two species of a link and site adjacent, then x).  The stored value is the
// post-collision population minus the background b^S_l(z) = w_l rho_bar c^S_0(z) in
// LB_PREC_DEV32 mode, and the plain post-collision population in LB_PREC_FP64 mode (where the
// background is zero).
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include "lb.h"

namespace lbk {

// D2Q9 links of Fig. 1 (c_0 = 0, c_1 = (1,0), c_2 = (0,1), c_3 = (-1,0), c_4 = (0,-1),
// c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1)).
#define LB_CX(l) ((l) == 1 || (l) == 5 || (l) == 8 ? 1 : ((l) == 3 || (l) == 6 || (l) == 7 ? -1 : 0))
#define LB_CZ(l) ((l) == 2 || (l) == 5 || (l) == 6 ? 1 : ((l) == 4 || (l) == 7 || (l) == 8 ? -1 : 0))
#define LB_OPP(l) ((l) == 0 ? 0 : ((l) <= 4 ? (((l) + 1) % 4) + 1 : (((l) - 3) % 4) + 5))

// Device-level flag bits (subset of the public flags that kernels look at).
// DF_UNIT: the rates of moments 3..8 are all exactly 1 (the step kernels then skip those moments).
enum : int { DF_ASTAR = 1, DF_WALL_FIXED = 2, DF_NOISE_LOC = 4, DF_NOISE = 8, DF_UNIT = 16 };

// Noise variants of the step kernel.
enum : int { NOISE_OFF = 0, NOISE_HOM = 1, NOISE_LOC = 2 };

// Per-lattice constants in the working precision.
template <class real>
struct LatticeDev {
  int Lx, Lz;
  int64_t f_off;     // element offset of the population block
  int64_t site_off;  // site offset into per-site arrays (sampled fields)
  int row_off;       // offset into the per-row table
  int flags;         // DF_* bits
  uint32_t key0, key1, lattice_id, pad;
  // Philox site counter of column x, row z: z * site_Lx + (x + site_x0) mod site_Lx; the
  // identity (0, Lx) unless the lattice is an x-slab window of a wider one (lb_set_site_map)
  int site_x0, site_Lx;
  real lam[9];       // relaxation rate per moment (Eq. MRT)
  real omh[9];       // 1 - lambda_a / 2 (second-order forcing)
  real G;            // coupling (Eq. aNI)
  real g3;           // grad_c0 / 3: gradient force density per unit rho (Eq. ne-acc)
  real k9, k36;      // streaming shift of the background on links with c_z = -1 for
                     // species A, per weight class (w = 1/9, 1/36); zero in FP64 mode
  real rho_bar_off;  // rho_bar in FP64 mode, 0 in deviation mode
  real sig_mom;      // hom noise amplitude of moments 1, 2 (Eq. noise-bin-expl)
  real sig[9];       // hom noise amplitudes of moments 3..8 (Eq. noise-bin-expl-high); the
                     // reference densities of both species are rho_bar / 2 (c_bar0 = 1/2)
  real pref_mom;     // loc noise: sqrt((2 - l_d) l_d kT)
  real pref[9];      // loc noise: sqrt(3 (2 - l_a) l_a N_a kT)
  // Eq. MRT divided by 36 N_a, as used by the step kernels: m*_a / (36 N_a) = kA[a] m_a +
  // kB[a] q_a + kC[a] s_a + kN[a] n_a, with q_a, s_a the equilibrium and forcing moments without
  // their constant factors (q_3 = rho |U|^2, s_3 = U.F, s_4 = U_x F_x - U_z F_z) and n_a a
  // standard normal (kN: hom amplitudes; for loc, times sqrt of the local density); 1/36 is the
  // weight of the diagonal links in the inverse transform
  real kA[9], kB[9], kC[9], kN[9];
};

// Per-row constants of the background (zero in FP64 mode), rows 0..Lz-1.
template <class real>
struct __align__(4 * sizeof(real)) RowConst {  // aligned: the first four load as one vector
  real bgA, bgB;    // rho_bar c^S_0(z)
  real dbgA, dbgB;  // background part of sum_l w_l c_lz rho^S(z + c_lz), wall ghosts included
  real nbA, nbB;    // background part of sum_l w_l |c_l|^2 rho^S(z + c_lz), ghosts included
  real c0;          // c_0(z)
  real ghost_cA;    // fixed-wall ghost: c^A of the wall next to this row (0 if not a wall row)
};

// A work item: columns [x0, x0 + blockDim.x) of rows [z0, z1) of one lattice.
struct WorkItem {
  int lattice;
  int x0;
  int z0, z1;
};

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)),
// the key advanced by the Weyl increments (W0, W1) before every round but the first.
// ------------------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    const U4 n = {hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    c = n;
  }
  return c;
}

// The four Philox4x32-10 calls of one site, counters (c0, c1, c2, call) for call = 0..3, in
// lockstep: the round keys are formed once for all four, and the products that do not yet
// depend on the last counter word (both in round 1, M0 x in round 2, M1 x in round 3) are
// formed once.  out[call] is bit-identical to philox({c0, c1, c2, call}, k0, k1).
__device__ __forceinline__ void philox_site(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1,
                                            U4 out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  // round 1: (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ call ^ k1, lo(M0 c0))
  uint64_t p = (uint64_t)M0 * c0;
  const uint32_t y3 = (uint32_t)p, t1 = (uint32_t)(p >> 32) ^ k1;
  p = (uint64_t)M1 * c2;
  const uint32_t y1 = (uint32_t)p, y0 = (uint32_t)(p >> 32) ^ c1 ^ k0;
  // round 2: M0 y0 is common; M1 y2 depends on the call
  k0 += W0;
  k1 += W1;
  p = (uint64_t)M0 * y0;
  const uint32_t z3 = (uint32_t)p, z2 = (uint32_t)(p >> 32) ^ y3 ^ k1;
  uint32_t s0[4], s1[4], s2[4], s3[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t q = (uint64_t)M1 * (t1 ^ (uint32_t)i);
    s0[i] = (uint32_t)(q >> 32) ^ y1 ^ k0;
    s1[i] = (uint32_t)q;
  }
  // round 3: M1 z2 is common; M0 s0 depends on the call
  k0 += W0;
  k1 += W1;
  p = (uint64_t)M1 * z2;
  const uint32_t r1 = (uint32_t)p, r0x = (uint32_t)(p >> 32) ^ k0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t q = (uint64_t)M0 * s0[i];
    const uint32_t n0 = r0x ^ s1[i], n2 = (uint32_t)(q >> 32) ^ z3 ^ k1, n3 = (uint32_t)q;
    s0[i] = n0;
    s1[i] = r1;
    s2[i] = n2;
    s3[i] = n3;
  }
  // rounds 4..10
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    k0 += W0;
    k1 += W1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t a = (uint64_t)M0 * s0[i], b = (uint64_t)M1 * s2[i];
      const uint32_t n0 = (uint32_t)(b >> 32) ^ s1[i] ^ k0, n1 = (uint32_t)b;
      const uint32_t n2 = (uint32_t)(a >> 32) ^ s3[i] ^ k1, n3 = (uint32_t)a;
      s0[i] = n0;
      s1[i] = n1;
      s2[i] = n2;
      s3[i] = n3;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = U4{s0[i], s1[i], s2[i], s3[i]};
}

// Uniform in (0, 1) from the low 23 bits, u = (2 (k mod 2^23) + 1) 2^-24, exact in float and
// double: the bits form x = 1 + (k mod 2^23) 2^-23 in [1, 2) and u = x - (1 - 2^-24) exactly.
__device__ __forceinline__ float unit_interval_bits(uint32_t k) { return __uint_as_float(0x3F800000u | (k & 0x7FFFFFu)); }
template <class real>
__device__ __forceinline__ real uniform01(uint32_t k);
template <>
__device__ __forceinline__ float uniform01<float>(uint32_t k) {
  return unit_interval_bits(k) - 0.999999940395355224609375f;
}
template <>
__device__ __forceinline__ double uniform01<double>(uint32_t k) {
  return __longlong_as_double((long long)(0x3FF0000000000000ull | ((unsigned long long)(k & 0x7FFFFFu) << 29))) -
         0.999999940395355224609375;
}

// Box-Muller: (r cos 2 pi u2, r sin 2 pi u2) with r = sqrt(-2 ln u1).
template <class real>
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, real& n0, real& n1);
template <>
__device__ __forceinline__ void box_muller<float>(uint32_t a, uint32_t b, float& n0, float& n1) {
  const float u1 = uniform01<float>(a), u2 = uniform01<float>(b);
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  n0 = r * c;
  n1 = r * s;
}
template <>
__device__ __forceinline__ void box_muller<double>(uint32_t a, uint32_t b, double& n0, double& n1) {
  const double u1 = uniform01<double>(a), u2 = uniform01<double>(b);
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  n0 = r * c;
  n1 = r * s;
}

// ---- normals of the step kernels ----------------------------------------------------------
// The hardware approximations in their flush-to-zero forms: their arguments here are never
// subnormal (u1 >= 2^-24, t > 2^-24, phi a multiple of 2^-44), so the results are those of the
// plain forms without their subnormal handling.
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void sincos_ftz(float x, float& s, float& c) {
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// 1 / rho of a site's total density: the hardware reciprocal in single precision (at most 1 ulp
// from the exact value; rho is near rho_bar = 1, never subnormal), refined by Newton steps in
// double.
__device__ __forceinline__ float site_reciprocal(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double site_reciprocal(double x) {
  // two Newton steps y <- y + y (1 - x y) from the single-precision seed (relative error 2^-23
  // -> 2^-46 -> the last bit); x is near 1
  double y = (double)site_reciprocal((float)x);
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}

// Tables of the double-precision Box-Muller (the table-driven method of P. T. P. Tang for the
// logarithm and for sine/cosine): cs[j] = (cos, sin)(2 pi j / 1024), ln[j] = (-2 ln y_j, 1 / y_j)
// with y_j = 3/4 + j/256, j = 0 .. 192, and the exponent's share ex[k] = (-2 n ln2_hi,
// -2 n ln2_lo) for n = k - 24, k = 0 .. 24 (ln 2 = ln2_hi + ln2_lo, ln2_hi rounded to 24 bits, so
// the first product is exact).  The single-precision path needs none.
template <class real>
struct BmTables {};
template <>
struct BmTables<double> {
  double2 cs[1024];
  double2 ln[193];
  double2 ex[25];
};
constexpr double kLn2Hi = 0.693147182464599609375, kLn2Lo = -1.904654299957768e-09;

// All threads of the block fill the tables (from the correctly rounded library functions); the
// caller synchronises the block before use.
template <class real>
__device__ __forceinline__ void fill_bm_tables(BmTables<real>* T) {
  if constexpr (sizeof(real) == 8) {
    for (int j = threadIdx.x; j < 1024; j += blockDim.x) {
      double sn, cs;
      sincospi((double)j / 512.0, &sn, &cs);
      T->cs[j] = make_double2(cs, sn);
    }
    for (int j = threadIdx.x; j < 193; j += blockDim.x) {
      const double y = 0.75 + (double)j / 256.0;
      T->ln[j] = make_double2(-2.0 * log(y), 1.0 / y);  // -2 ln y_j (an exact scaling), 1 / y_j
    }
    for (int k = threadIdx.x; k < 25; k += blockDim.x) {
      const double n = (double)(k - 24);
      T->ex[k] = make_double2(n * (-2.0 * kLn2Hi), n * (-2.0 * kLn2Lo));
    }
  }
}

// Box-Muller pair of the working precision, (r cos 2 pi u2, r sin 2 pi u2) with r = sqrt(-2 ln u1).
// FP32: t = -2 ln u1 from the hardware base-2 logarithm, whose absolute error (~2^-22) the square
// root would magnify where t is small; there (v = 1 - u1 < 2^-6, v exact) the series
// -ln(1 - v) = v + v^2/2 + v^3/3 + ... is used instead (next term below 1e-6 of t).  The radius
// is t / sqrt(t) through the reciprocal square root, and the angle is reduced to (-pi, pi) for
// the fast sine/cosine: cos 2 pi u2 = -cos phi and sin 2 pi u2 = -sin phi with
// phi = 2 pi u2 - pi.  Absolute error below 3e-6 on a normal.
// FP64, table-driven: u = m 2^-24 with m = 2 (k mod 2^23) + 1.  ln u1 = (e - 24) ln 2 + ln y with
// m = 2^e y, y in [3/4, 3/2); ln y = ln y_j + ln(1 + t), y_j the table point nearest y and
// t = y (1 / y_j) - 1 (one fused multiply-add; exact where y_j = 1, i.e. wherever u1 is near 1
// and -2 ln u1 small), |t| <= 2^-9 / (3/4), from its series to t^6; (e - 24) times the two parts
// of -2 ln 2 comes from a table.  The angle 2 pi m 2^-24 is
// the table angle 2 pi (m >> 14) / 1024 plus d = 2 pi (m mod 2^14) 2^-24 < 6.2e-3, whose sine and
// cosine come from their series (to d^5 and d^6) and the addition theorems.  Within a few units
// in the last place of the library functions.
template <class real>
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, real& n0, real& n1, const BmTables<real>* T);
template <>
__device__ __forceinline__ void normal_pair<float>(uint32_t a, uint32_t b, float& n0, float& n1,
                                                   const BmTables<float>*) {
  const float u1 = uniform01<float>(a);
  const float v = 1.0f - u1;
  const float t_log = -1.38629436111989061f * lg2_ftz(u1);
  const float t_ser = v * fmaf(v, fmaf(v, 0.666666666666666667f, 1.0f), 2.0f);
  const float t = v < 0.015625f ? t_ser : t_log;
  const float r = t * rsqrt_ftz(t);
  // phi = 2 pi u2 - pi = 2 pi x2 - 3 pi + 2 pi 2^-24 with x2 = u2 + 1 - 2^-24 built from the bits
  const float phi = fmaf(6.28318530717959f, unit_interval_bits(b), -9.42477758729298f);
  float s, c;
  sincos_ftz(phi, s, c);
  n0 = -r * c;
  n1 = -r * s;
}
template <>
__device__ __forceinline__ void normal_pair<double>(uint32_t a, uint32_t b, double& n0, double& n1,
                                                    const BmTables<double>* T) {
  const uint32_t m1 = 2u * (a & 0x7FFFFFu) + 1u;
  const unsigned long long bits = (unsigned long long)__double_as_longlong((double)m1);
  int e = (int)(bits >> 52) - 1023;
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  int j;
  double y;
  if (mant >= (1ull << 51)) {  // y0 = m1 / 2^e in [3/2, 2): y = y0 / 2 in [3/4, 1)
    e += 1;
    y = __longlong_as_double((long long)(0x3FE0000000000000ull | mant));
    j = (int)(((mant - (1ull << 51)) + (1ull << 44)) >> 45);
  } else {  // y in [1, 3/2)
    y = __longlong_as_double((long long)(0x3FF0000000000000ull | mant));
    j = 64 + (int)((mant + (1ull << 43)) >> 44);
  }
  const double2 L = T->ln[j];
  const double t = fma(y, L.y, -1.0);
  // -2 ln u1 directly: every term and coefficient scaled by -2, a power of two, so the result is
  // bit for bit -2 times the logarithm formed term by term
  const double p2 =
      fma(t, fma(t, fma(t, fma(t, fma(t, 1.0 / 3.0, -0.4), 0.5), -2.0 / 3.0), 1.0), -2.0);  // -2 p(t)
  const double2 E = T->ex[e];  // e - 24 in -24 .. 0
  const double m2lnu = E.x + (L.x + fma(t, p2, E.y));
  const double r = sqrt(m2lnu);
  // angle
  const uint32_t m2 = 2u * (b & 0x7FFFFFu) + 1u;
  const double2 CS = T->cs[m2 >> 14];
  const double d = (double)(m2 & 0x3FFFu) * (6.283185307179586476925286766559 * 5.9604644775390625e-08);
  const double d2 = d * d;
  const double sd = fma(d * d2, fma(d2, 1.0 / 120.0, -1.0 / 6.0), d);
  const double cm1 = d2 * fma(d2, fma(d2, -1.0 / 720.0, 1.0 / 24.0), -0.5);  // cos d - 1
  const double cs = fma(-CS.y, sd, fma(CS.x, cm1, CS.x));
  const double sn = fma(CS.x, sd, fma(CS.y, cm1, CS.y));
  n0 = r * cs;
  n1 = r * sn;
}

// Two Box-Muller pairs at once, (a0, b0) and (a1, b1): normal_pair's arithmetic with its FP32
// steps in packed two-lane instructions; n0 = (n0 of the first pair, n0 of the second), n1
// likewise.  FP64: two normal_pair calls.
template <class real>
__device__ __forceinline__ void normal_pair2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, real& n00,
                                             real& n01, real& n10, real& n11, const BmTables<real>* T) {
  normal_pair<real>(a0, b0, n00, n01, T);
  normal_pair<real>(a1, b1, n10, n11, T);
}
template <>
__device__ __forceinline__ void normal_pair2<float>(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, float& n00,
                                                    float& n01, float& n10, float& n11, const BmTables<float>*) {
  const float2 x1 = make_float2(unit_interval_bits(a0), unit_interval_bits(a1));
  const float2 u1 = __fadd2_rn(x1, make_float2(-0.999999940395355224609375f, -0.999999940395355224609375f));
  const float2 v = __ffma2_rn(u1, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
  const float2 tl = __fmul2_rn(make_float2(-1.38629436111989061f, -1.38629436111989061f),
                               make_float2(lg2_ftz(u1.x), lg2_ftz(u1.y)));
  const float2 ts = __fmul2_rn(
      v, __ffma2_rn(v, __ffma2_rn(v, make_float2(0.666666666666666667f, 0.666666666666666667f), make_float2(1.0f, 1.0f)),
                    make_float2(2.0f, 2.0f)));
  const float2 t = make_float2(v.x < 0.015625f ? ts.x : tl.x, v.y < 0.015625f ? ts.y : tl.y);
  const float2 r = __fmul2_rn(t, make_float2(rsqrt_ftz(t.x), rsqrt_ftz(t.y)));
  const float2 phi = __ffma2_rn(make_float2(6.28318530717959f, 6.28318530717959f),
                                make_float2(unit_interval_bits(b0), unit_interval_bits(b1)),
                                make_float2(-9.42477758729298f, -9.42477758729298f));
  float s0, c0, s1, c1;
  sincos_ftz(phi.x, s0, c0);
  sincos_ftz(phi.y, s1, c1);
  n00 = -r.x * c0;
  n01 = -r.x * s0;
  n10 = -r.y * c1;
  n11 = -r.y * s1;
}


template <class real>
__device__ __forceinline__ real sqrt_pos(real v);
template <>
__device__ __forceinline__ float sqrt_pos<float>(float v) { return sqrtf(v); }
template <>
__device__ __forceinline__ double sqrt_pos<double>(double v) { return sqrt(v); }

// Host-side launch helpers implemented in lb_step.cu / lb_diag.cu.
template <class real>
struct StepArgs {
  const LatticeDev<real>* lat;
  const RowConst<real>* rows;
  const WorkItem* items;
  int n_items;
  const real* src;
  real* dst;
  const int64_t* d_t;  // device step counter; the step index is *d_t + t_offset
  int t_offset;
  real* fields;        // sampled fields [4][Lz][Lx] per lattice (sample steps only)
  real* pfield;        // sampled pressure [Lz][Lx] per lattice, minus the row background in
                       // deviation mode (sample steps only)
  double* partials;    // per item: pressure deviation sum, mass deviation A, B
  int* err;            // set to 1 by a device-side wait that gave up
  // bulk path (FP32 state): 3-d tensor maps [x][z][link] of the (A, B) pairs as 8-byte elements,
  // per state buffer and lattice, for runs of one and of two links (index (buffer n_lat +
  // lattice) 2 + run length - 1), or null; src_buf: the state buffer src points to
  const CUtensorMap* tmaps;
  int n_lat;
  int src_buf;
};

// The stored state of a lattice: [link l][row z][column x][species s], so the populations of both
// species of one (link, site) are adjacent and one 8-byte (FP32) or 16-byte (FP64) access moves
// the pair.  The element index of f^s_l(x, z):
__host__ __device__ __forceinline__ int64_t state_index(int s, int l, int z, int x, int Lx, int64_t LzLx) {
  return ((int64_t)l * LzLx + (int64_t)z * Lx + x) * 2 + s;
}

// The input row slot of the bulk path, in (A, B) pairs: the 9 link rows grouped in the six runs of
// consecutive links with equal c_z, (0 1) (2) (3) (4) (5 6) (7 8).  Run j holds [link of the
// run][BW columns] at a 128-byte aligned base: the layout one tensor copy writes (a box of BW
// columns, one row, the run's links).  PS: bytes per pair.
__host__ __device__ constexpr int run_of(int l) { return l < 2 ? 0 : (l < 5 ? l - 1 : (l < 7 ? 4 : 5)); }
__host__ __device__ constexpr int run_l0(int j) { return j == 0 ? 0 : (j <= 3 ? j + 1 : (j == 4 ? 5 : 7)); }
__host__ __device__ constexpr int run_n(int j) { return (j == 0 || j >= 4) ? 2 : 1; }
template <int BW, int PS>
struct SlotLayout {
  static constexpr int ALIGN = 128 / PS;  // pairs per 128 bytes
  __host__ __device__ static constexpr int run_size(int j) { return ((run_n(j) * BW + ALIGN - 1) / ALIGN) * ALIGN; }
  __host__ __device__ static constexpr int base(int j) { return j == 0 ? 0 : base(j - 1) + run_size(j - 1); }
  // pair offset of link row l in the slot
  __host__ __device__ static constexpr int plane(int l) { return base(run_of(l)) + (l - run_l0(run_of(l))) * BW; }
  static constexpr int slot = base(6);  // pairs per slot (a multiple of 128 bytes)
  // base(j) for a run index known only at run time
  __host__ __device__ static int base_of(int j) {
    constexpr int b1 = base(1), b2 = base(2), b3 = base(3), b4 = base(4), b5 = base(5);
    return j == 0 ? 0 : (j == 1 ? b1 : (j == 2 ? b2 : (j == 3 ? b3 : (j == 4 ? b4 : b5))));
  }
};

// bulk: stage rows with bulk copies (tile_x 32, 64, 128 or 256, every lattice's Lx a multiple of
// 16 bytes); otherwise per-thread copies.
template <class real>
cudaError_t launch_step(const StepArgs<real>& a, int tile_x, bool sample, int noise, bool bulk, cudaStream_t s);

// Dynamic shared memory of the step kernels for a tile width, and the one-time attribute set-up
// that allows it (called before any launch or capture).
template <class real>
size_t step_smem_bytes(int tile_x);
template <class real>
cudaError_t prepare_step(int max_tile_x);

// The persistent launch's scheduling state (see the persistent kernels): the ticket counter and
// done[] zeroed before each launch, and the dependency lists of the items (CSR).
struct PersistArgs {
  unsigned long long* counter;
  unsigned* done;
  const int* nbr_off;
  const int* nbr;
  int* err;
  int limit_ms;
  int trial;  // autotuner's trial mode: every step reads src and writes dst (the state is untouched)
};

template <class real>
cudaError_t launch_step_persistent(const StepArgs<real>& a, int tile_x, int nsteps, int noise, bool bulk,
                                   const PersistArgs& p, int grid, cudaStream_t s);

template <class real>
int persistent_grid(int tile_x, int noise, bool bulk);

cudaError_t launch_advance(int64_t* d_t, int64_t k, cudaStream_t s);

// Diagnostics (lb_diag.cu)
struct DiagLattice {
  int Lx, Lz;
  int64_t site_off;    // offset in sites of this lattice in fields / spectra
  int row_off;         // offset of row 0 in the per-row tables (profiles)
  int64_t r_off;       // offset (doubles) of the real-space correlations [4][Lz][Lz]
  int64_t c_off;       // offset (doubles) of the mode correlations [4][modes][Lz][Lz][re, im]
  int item_begin, item_end;
  double P_bg_mean;    // spatial mean of the background pressure (FP64 mode: 0)
  double mass_bg[2];   // background mass per species (FP64 mode: 0)
  double n_sites;
};

struct DiagStats {  // per lattice, updated by the finalize kernel
  double P_last, P_sum, P_comp;
  double massA_last, massB_last;
  int nonfinite;
  int pad;
};

// Transform tasks of one sample: one block per (lattice, field * Lz + z0) group of rows and per
// (lattice, field * Lx + q_x0) strip of columns (sf_row_group, sf_col_strip below).
struct SfPlan {
  const DiagLattice* lat;
  const int2* row_tasks;
  const int2* col_tasks;
  int n_row_tasks, n_col_tasks;
  int threads;                 // threads per transform block
  int cap;                     // complex points one block holds, 16 per thread
  size_t smem_rows, smem_cols;  // dynamic shared memory of the two passes
  // z-profiles of the four fields: the q_x = 0 bin of each row transform is the row sum
  double* prof_sum;
  double* prof_comp;
  int n_rows;
};

// The row transforms of a sample in tmp: the fields are real, so only q_x = 0 .. Lx/2 is kept,
// H = Lx/2 + 1 values per row, row (field, z) of a lattice at 4 site_off + (field Lz + z) H.
__host__ __device__ __forceinline__ int sf_half(int Lx) { return Lx / 2 + 1; }

// Sizes of the sample-step transforms.  A block of `threads` threads holds cap = 16 threads
// complex points in shared memory: two real rows of x form one complex sequence, and a column
// strip is a set of adjacent q_x.  cap covers the longest sequence of the batch.
inline int sf_threads(int max_Lx, int max_Lz) {
  const int m = max_Lx > max_Lz ? max_Lx : max_Lz;
  return m > 4096 ? m / 16 : 256;
}
// Real rows z0 .. z0 + R - 1 of one row-pass block (R even unless it is all of Lz).
__host__ __device__ __forceinline__ int sf_row_group(int Lx, int Lz, int cap) {
  const int r = 2 * (cap / Lx);
  return r < Lz ? r : Lz;
}
// q_x columns of one column-pass block.
__host__ __device__ __forceinline__ int sf_col_strip(int Lx, int Lz, int cap) {
  const int c = cap / Lz, H = sf_half(Lx);
  return c < H ? c : H;
}
// Shared-memory stride of one sequence of n points: one pad point after every 16 and one per
// sequence, so that strided and transposing accesses spread over the banks.
__host__ __device__ __forceinline__ int sf_seq_stride(int n) { return n + (n >> 4) + 1; }

// What the utility kernels need to rebuild the background w_l rho_bar c^S_0(z) in double.
struct BgParams {
  int Lx, Lz;
  int dev;
  double rho_bar, grad_c0;
};

template <class real>
cudaError_t prepare_sf(size_t smem_rows, size_t smem_cols);

template <class real>
cudaError_t launch_sf(const SfPlan& p, const real* fields, void* tmp, double* acc_sum, double* acc_comp,
                      cudaStream_t s);

// Two-point correlations of one sample (Sec. III.A-B, Appendix A), in tiles of CORR_TILE x
// CORR_TILE rows (z, z'): real_tasks = (lattice, field, z tile, z' tile) add
// (1/Lx) sum_x dphi(x, z) dphi(x, z') to R; mode_tasks = (lattice, field * n_modes + m, z tile,
// z' tile) add dphi(q_m, z)^* dphi(q_m, z') (unitary partial transform in x) to C, from the row
// transforms the structure-factor pass leaves in tmp.
constexpr int CORR_TILE = 16;
struct CorrPlan {
  const DiagLattice* lat;
  const int4* real_tasks;
  int n_real_tasks;
  const int4* mode_tasks;
  int n_mode_tasks;
  const int* modes;
  int n_modes;
};
template <class real>
cudaError_t launch_corr(const CorrPlan& p, const real* fields, const void* tmp, double* R, double* C, cudaStream_t s);

// z-profiles (Sec. III.C): the row pass of launch_sf adds the row means of delta rho, delta c, Ux
// and Uz to the per-row compensated sums [5][n_rows]; this adds those of the sampled pressure
// (deviation), slot 4; row_lat[r] is the lattice of global row r.
template <class real>
cudaError_t launch_profiles(const DiagLattice* lat, const int* row_lat, int n_rows, const real* fields,
                            const real* pfield, double* prof_sum, double* prof_comp, cudaStream_t s);

cudaError_t launch_finalize(const DiagLattice* d_lat, int n_lat, const double* partials, DiagStats* stats,
                            cudaStream_t s);

template <class real>
cudaError_t launch_mass(const real* f, const BgParams& bp, double* out2, cudaStream_t s);
template <class real>
cudaError_t launch_to_absolute(const real* f, const BgParams& bp, double* out, cudaStream_t s);
template <class real>
cudaError_t launch_from_absolute(const double* in, const BgParams& bp, real* f, cudaStream_t s);
template <class real>
cudaError_t launch_init_rest(real* f, const BgParams& bp, cudaStream_t s);
// Columns x_first .. x_first + n - 1 of all 18 planes of a stored state f (Lx x Lz) to or from a
// packed buffer [18][Lz][n] (x-slab halo exchange).
template <class real>
cudaError_t launch_columns(real* f, int Lx, int Lz, int x_first, int n, real* buf, bool to_buf, cudaStream_t s);

// Power spectrum of one real double-precision field (Lx, Lz powers of two, 2..8192), with a
// caller-provided scratch of Lx * Lz complex doubles; prepare once per device before use.
cudaError_t prepare_power_spectrum();
cudaError_t launch_power_spectrum(const double* field, int Lx, int Lz, double* out, void* tmp, cudaStream_t s);

// Host-side checks shared by the two spectrum entry points (lb_api.cu): LB_ERR_BAD_PARAM unless
// Lx and Lz are powers of two in 2..8192 and field and out are device (or managed) memory of the
// current device; LB_OK otherwise.
int power_spectrum_args_ok(const double* field, int Lx, int Lz, const double* out);
// prepare_power_spectrum once per device, with that device current (LB_OK or LB_ERR_CUDA).
int prepare_power_spectrum_current_device();

// Measured fused multiply-add rate of the current device (FP64 or FP32 scalar FMA, 2 flops each),
// best of five timed launches after a warm-up (lb_diag.cu).
cudaError_t measure_fma_rate(bool fp64, double* flops_per_s);

template <class real>
cudaError_t launch_debug_normals(const uint32_t* words, int64_t n_pairs, double* out, cudaStream_t s);

// Test hook of the bounded waits of the persistent launch: `blocks` co-resident blocks each set
// done[b] and wait until done[list[0 .. expected)] are set.
cudaError_t launch_barrier_probe(int blocks, int expected, int spin_limit, unsigned* done, const int* list, int* err,
                                 cudaStream_t s);

}  // namespace lbk
