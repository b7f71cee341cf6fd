// lb_step_impl.cuh -- the fused per-step kernel of the fluctuating two-species D2Q9 MRT method
// (Eq. LB with Eq. MRT), one launch per step for every lattice of a batch, or one cooperative
// launch for a run of steps whose work items wait only for their neighbours' previous step.
//
// The state is stored as (A, B) pairs, [link][z][x][species] (state_index), so each population
// pair moves as one 8-byte (FP32) or 16-byte (FP64) access.
//
// Work decomposition: a block of TX threads owns TX consecutive columns x of one lattice and
// marches up rows z0..z1-1 of that lattice.  The 9 population pairs arriving at each site
// (Eq. LB; mid-way bounce-back at the walls of Sec. II.A) are staged in shared memory, several
// rows ahead of the row being collided, so that every stored value is read once per step from
// HBM and no population is held in registers across rows.  Two staging paths compute the same
// numbers bit for bit:
//  - bulk (rows 16-byte aligned, TX = 32, 64, 128 or 256): for each of the 9 link rows one lane
//    issues a bulk asynchronous copy of the row window [x0 - PAD, x0 + TX + PAD) (PAD = 2
//    columns; wrapped periodically at the lattice's x edges) into a ring of NSI row
//    slots, or, away from the x edges, one 3-d tensor copy per run of links with equal c_z,
//    completion tracked by one mbarrier per slot; a one-warp block (TX = 32) marches without
//    waiting on other warps;
//  - generic (any Lx, any tile): every thread stages its own 9 pairs with per-thread
//    asynchronous copies.
// Both store each post-collision pair with one streaming store.
// The non-ideal force (Eq. aNI) needs the densities of the 8 neighbours at the same time
// level: the densities of rows z-1, z, z+1 live in a 4-slot shared-memory ring (one barrier per
// row); the halo columns are read by the edge threads.  The wall ghost rows follow Sec. II.A.
//
// Arithmetic per site: densities and momenta, forces (Eqs. aNI, ne-acc, a* of its footnote),
// barycentric velocity (Eq. bar), moments of Table I in their structured +- form, relaxation
// toward m^eq with second-order forcing (1 - lambda_a/2) S_a, FDT noise from Philox4x32-10
// (Eqs. noise-bin-expl, noise-bin-expl-high), and the inverse transform
// f_l = w_l sum_a T_al m*_a / N_a.
#pragma once

#include <cstdio>

#include "lb_internal.cuh"

namespace lbk {

namespace {

constexpr int NS = 4;   // generic path: rows of staged populations (power of two)
#ifndef LB_BULK_NSI
#define LB_BULK_NSI 3
#endif
#ifndef LB_BULK_BLOCKS_F32
#define LB_BULK_BLOCKS_F32 6  // resident 128-column blocks per SM the float bulk kernels target
#endif
constexpr int NSI = LB_BULK_NSI;  // bulk path: input row slots
constexpr int WAIT_MS = 2000;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---- (A, B) pairs ------------------------------------------------------------------
// The two species go through identical arithmetic, so every per-species quantity of a site is
// carried as a pair (lane x: species A, lane y: species B).  FP32: the packed two-lane
// instructions of sm_100 and later, one instruction for both species; FP64: two scalar
// operations.
template <class real>
struct PairOf;
template <>
struct PairOf<float> {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};
template <class real>
using Pr = typename PairOf<real>::type;

__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pr(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 pr(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 pr(double a) { return make_double2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// ---- per-thread asynchronous copies of one (A, B) pair (generic path) ---------------
__device__ __forceinline__ void cp_async(float2* dst_smem, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double2* dst_smem, const double2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- bulk copies and mbarriers (bulk path) ------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// One box of a 3-d tensor map (coordinates x, z, link) into shared memory (128-byte aligned),
// completion counted on the mbarrier.
__device__ __forceinline__ void tensor_g2s(void* dst_smem, const CUtensorMap* map, int x, int z, int l, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst_smem)),
      "l"(map), "r"(x), "r"(z), "r"(l), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src_smem, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src_smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ring_slot(int z) { return (z + 4) & 3; }

// Generic path: stage the 9 population pairs arriving at (x, z) (Eq. LB) into dst[l * W]: link l
// comes from (x - c_lx, z - c_lz); a link whose source row lies beyond a wall takes the reflected
// pair f*_opp(l)(x, z).  f: the lattice's state as pairs, [link][z][x].
template <class P>
__device__ __forceinline__ void stage_column(const P* __restrict__ f, int LzLx, int Lx, int Lz, int z, int x, P* dst,
                                             int W) {
  const int xm = (x == 0) ? Lx - 1 : x - 1;
  const int xp = (x + 1 == Lx) ? 0 : x + 1;
  const bool below = z > 0, above = z < Lz - 1;
  const int r0 = z * Lx, rdn = r0 - Lx, rup = r0 + Lx;
  cp_async(dst + 0 * W, f + 0 * LzLx + r0 + x);
  cp_async(dst + 1 * W, f + 1 * LzLx + r0 + xm);
  cp_async(dst + 3 * W, f + 3 * LzLx + r0 + xp);
  cp_async(dst + 2 * W, below ? f + 2 * LzLx + rdn + x : f + 4 * LzLx + r0 + x);
  cp_async(dst + 4 * W, above ? f + 4 * LzLx + rup + x : f + 2 * LzLx + r0 + x);
  cp_async(dst + 5 * W, below ? f + 5 * LzLx + rdn + xm : f + 7 * LzLx + r0 + x);
  cp_async(dst + 6 * W, below ? f + 6 * LzLx + rdn + xp : f + 8 * LzLx + r0 + x);
  cp_async(dst + 7 * W, above ? f + 7 * LzLx + rup + xp : f + 5 * LzLx + r0 + x);
  cp_async(dst + 8 * W, above ? f + 8 * LzLx + rup + xm : f + 6 * LzLx + r0 + x);
}

// The 9 populations of both species of one site as deviations from the background of its row.
// In deviation mode the background difference b_l(z - c_lz) - b_l(z) = -w_l rho_bar c_lz
// d_z c^S_0 belongs on every non-reflected link with c_lz != 0 (k9, k36: its size on the
// 1/9- and 1/36-weight links of species A, the opposite for B; zero in FP64 mode).  In interior
// rows these shifts sum to zero and change no moment but m_2 (see interior_m2_shift), so they are
// applied to the moments there; in the two wall rows, where the reflected links carry none, per
// link.
template <class real>
__device__ __forceinline__ void deviations(Pr<real> v[9], bool below, bool above, real k9, real k36) {
  if (!(below && above)) {
    const Pr<real> q9 = pr(k9, -k9), q36 = pr(k36, -k36), z = pr(real(0));
    const Pr<real> b9 = below ? q9 : z, b36 = below ? q36 : z;
    const Pr<real> a9 = above ? q9 : z, a36 = above ? q36 : z;
    v[2] = sub2(v[2], b9);
    v[4] = add2(v[4], a9);
    v[5] = sub2(v[5], b36);
    v[6] = sub2(v[6], b36);
    v[7] = add2(v[7], a36);
    v[8] = add2(v[8], a36);
  }
}

// Interior rows: the shifts (-q9 on link 2, +q9 on 4, -q36 on 5 and 6, +q36 on 7 and 8; q = k for
// species A, -k for B) have zero sum and zero moments except m_2 = -2 q9 - 4 q36.
template <class real>
__device__ __forceinline__ Pr<real> interior_m2_shift(real k9, real k36) {
  const real q = 2 * k9 + 4 * k36;
  return pr(-q, q);
}

// Generic path: stage column c of a slot holds the pairs pulled to that site.
template <class real>
__device__ __forceinline__ void read_generic(const Pr<real>* st, int W, int c, bool below, bool above, real k9,
                                             real k36, Pr<real> v[9]) {
  const Pr<real>* d = st + c;
#pragma unroll
  for (int l = 0; l < 9; ++l) v[l] = d[l * W];
  deviations(v, below, above, k9, k36);
}

// Bulk path: link row l of a slot (SlotLayout) holds the source row window of link l, so link l
// of the site at window column j sits at column j - c_lx (at j on reflected links, whose row
// holds the opposite link's own row).
template <class real, int SW>
__device__ __forceinline__ void read_bulk(const Pr<real>* st, int j, bool below, bool above, real k9, real k36,
                                          Pr<real> v[9]) {
  using LAY = SlotLayout<SW, (int)sizeof(Pr<real>)>;
  constexpr int o[9] = {LAY::plane(0), LAY::plane(1), LAY::plane(2), LAY::plane(3), LAY::plane(4),
                        LAY::plane(5), LAY::plane(6), LAY::plane(7), LAY::plane(8)};
  const Pr<real>* a = st + j;
  const int j5 = below ? -1 : 0, j6 = below ? 1 : 0, j7 = above ? 1 : 0, j8 = above ? -1 : 0;
  const int dx[9] = {0, -1, 0, 1, 0, j5, j6, j7, j8};
#pragma unroll
  for (int l = 0; l < 9; ++l) v[l] = a[o[l] + dx[l]];
  deviations(v, below, above, k9, k36);
}

template <class real>
__device__ __forceinline__ Pr<real> sum9(const Pr<real> v[9]) {
  return add2(add2(add2(add2(v[0], v[1]), add2(v[2], v[3])), add2(add2(v[4], v[5]), add2(v[6], v[7]))), v[8]);
}

// Moments m_1..m_8 of Table I of both species, in the structured form.
template <class real>
struct Mom {
  Pr<real> m1, m2, m3, m4, m5, m6, m7, m8;
};

template <class real>
__device__ __forceinline__ Mom<real> moments(const Pr<real> v[9]) {
  const Pr<real> a57 = sub2(v[5], v[7]), a68 = sub2(v[6], v[8]);
  const Pr<real> d13 = sub2(v[1], v[3]), d24 = sub2(v[2], v[4]);
  const Pr<real> s13 = add2(v[1], v[3]), s24 = add2(v[2], v[4]);
  const Pr<real> e = add2(s13, s24);
  const Pr<real> s57 = add2(v[5], v[7]), s68 = add2(v[6], v[8]);
  const Pr<real> dg = add2(s57, s68);
  const Pr<real> am = sub2(a57, a68), ap = add2(a57, a68);
  Mom<real> m;
  m.m1 = add2(d13, am);
  m.m2 = add2(d24, ap);
  m.m3 = fma2(pr(real(-2)), v[0], fma2(pr(real(4)), dg, e));
  m.m4 = sub2(s13, s24);
  m.m5 = sub2(s57, s68);
  m.m6 = sub2(add2(am, am), d13);
  m.m7 = sub2(add2(ap, ap), d24);
  m.m8 = fma2(pr(real(2)), v[0], fma2(pr(real(-4)), e, mul2(pr(real(8)), dg)));
  return m;
}

// Constants of one lattice the site update needs, in registers (unused ones are never loaded).
template <class real>
struct SiteK {
  real G, g3, rho_bar_off;
  real kA[9], kB[9], kC[9], kN[9];  // folded collision coefficients, as in LatticeDev
  uint32_t key0, key1, lid;
};

template <class real, int NOISE>
__device__ __forceinline__ SiteK<real> site_constants(const LatticeDev<real>& L) {
  SiteK<real> K;
  K.G = L.G;
  K.g3 = L.g3;
  K.rho_bar_off = L.rho_bar_off;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    K.kA[a] = L.kA[a];
    K.kB[a] = L.kB[a];
    K.kC[a] = L.kC[a];
    K.kN[a] = L.kN[a];
  }
  K.key0 = L.key0;
  K.key1 = L.key1;
  K.lid = L.lattice_id;
  return K;
}

// Compile-time flag for the two variants of the site update.
template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

// Collision of both species in moment space (Eq. MRT) with second-order forcing and noise, and
// the inverse transform f_l = w_l sum_a T_al m*_a / N_a.  Relaxation, forcing and noise factors
// and 1/N_a are folded into the per-lattice coefficients kA..kN; moments 1-2 share theirs (both
// relax at l_d), as do 6-7 (l_Q).  UNIT: the rates of moments 3..8 are 1, so their
// pre-collision values drop out (kA = 0) and are never formed.  nz[1..8]: the standard normals
// of the moments (pairs); cm, cq: their amplitude factors for moments 1-2 and 3-8 (sign and
// local density; (1, -1) and (1, 1) for hom noise).
template <class real, int NOISE, bool UNIT>
__device__ __forceinline__ void collide_out(const Mom<real>& m, Pr<real> d, Pr<real> rs, real Ux, real Uz,
                                            Pr<real> Fx, Pr<real> Fz, const SiteK<real>& K, const Pr<real> nz[9],
                                            Pr<real> cm, Pr<real> cq, Pr<real>* out, int stride) {
  using P = Pr<real>;
  const P U_x = pr(Ux), U_z = pr(Uz);
  const real UxUx = Ux * Ux, UzUz = Uz * Uz;
  const P r1 = mul2(pr(K.kB[1]), rs);
  P M1 = fma2(pr(K.kC[1]), Fx, fma2(r1, U_x, mul2(pr(K.kA[1]), m.m1)));
  P M2 = fma2(pr(K.kC[1]), Fz, fma2(r1, U_z, mul2(pr(K.kA[1]), m.m2)));
  const P uxF = mul2(U_x, Fx), uzF = mul2(U_z, Fz);
  P M3 = fma2(mul2(pr(K.kB[3]), rs), pr(UxUx + UzUz), mul2(pr(K.kC[3]), add2(uxF, uzF)));
  P M4 = fma2(mul2(pr(K.kB[4]), rs), pr(UxUx - UzUz), mul2(pr(K.kC[4]), sub2(uxF, uzF)));
  P M5 = fma2(mul2(pr(K.kB[5]), rs), pr(Ux * Uz), mul2(pr(K.kC[5]), fma2(U_x, Fz, mul2(U_z, Fx))));
  P M6 = pr(real(0)), M7 = pr(real(0)), M8 = pr(real(0));
  if (!UNIT) {
    M3 = fma2(pr(K.kA[3]), m.m3, M3);
    M4 = fma2(pr(K.kA[4]), m.m4, M4);
    M5 = fma2(pr(K.kA[5]), m.m5, M5);
    M6 = mul2(pr(K.kA[6]), m.m6);
    M7 = mul2(pr(K.kA[6]), m.m7);
    M8 = mul2(pr(K.kA[8]), m.m8);
  }
  if (NOISE != NOISE_OFF) {
    // hom noise: the amplitude factors are constants, so the coefficients need no product
    const bool loc = NOISE == NOISE_LOC;
    const P a1 = loc ? mul2(pr(K.kN[1]), cm) : pr(K.kN[1], -K.kN[1]);
    const P a3 = loc ? mul2(pr(K.kN[3]), cq) : pr(K.kN[3]), a4 = loc ? mul2(pr(K.kN[4]), cq) : pr(K.kN[4]);
    const P a5 = loc ? mul2(pr(K.kN[5]), cq) : pr(K.kN[5]), a6 = loc ? mul2(pr(K.kN[6]), cq) : pr(K.kN[6]);
    const P a8 = loc ? mul2(pr(K.kN[8]), cq) : pr(K.kN[8]);
    M1 = fma2(a1, nz[1], M1);
    M2 = fma2(a1, nz[2], M2);
    M3 = fma2(a3, nz[3], M3);
    M4 = fma2(a4, nz[4], M4);
    M5 = fma2(a5, nz[5], M5);
    if (UNIT) {
      M6 = mul2(a6, nz[6]);
      M7 = mul2(a6, nz[7]);
      M8 = mul2(a8, nz[8]);
    } else {
      M6 = fma2(a6, nz[6], M6);
      M7 = fma2(a6, nz[7], M7);
      M8 = fma2(a8, nz[8], M8);
    }
  }
  // links of opposite velocity pair up as f = u + v and f_opp = u - v (u: the even moments,
  // v: the odd ones).  The coefficients carry the weight 1/36 of the diagonal links (M here is
  // m* / (36 N_a)), so those need no product; the others have weight 4/36 and the rest link 16/36.
  const P dq = mul2(pr(real(1) / 36), d);
  const P base4 = fma2(pr(real(-4)), M8, add2(dq, M3));
  const P base5 = fma2(pr(real(8)), M8, fma2(pr(real(4)), M3, dq));
  const P u13 = mul2(pr(real(4)), add2(base4, M4)), v13 = sub2(M1, M6);
  const P u24 = mul2(pr(real(4)), sub2(base4, M4)), v24 = sub2(M2, M7);
  const P u57 = add2(base5, M5), v57 = fma2(pr(real(2)), add2(M6, M7), add2(M1, M2));
  const P u68 = sub2(base5, M5), v68 = fma2(pr(real(2)), sub2(M6, M7), sub2(M1, M2));
  const P f0 = mul2(pr(real(16)), fma2(pr(real(2)), M8, fma2(pr(real(-2)), M3, dq)));
  const P f[9] = {f0,
                  fma2(pr(real(4)), v13, u13),
                  fma2(pr(real(4)), v24, u24),
                  fma2(pr(real(-4)), v13, u13),
                  fma2(pr(real(-4)), v24, u24),
                  add2(u57, v57),
                  sub2(u68, v68),
                  sub2(u57, v57),
                  add2(u68, v68)};
#pragma unroll
  for (int l = 0; l < 9; ++l) __stcs(out + l * stride, f[l]);  // the pair of link l, streaming
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Everything of one site after its moments are known and the densities of its row and the two
// neighbouring rows sit in the ring: forces, velocity, optional sampling, noise, collision of
// both species and the output.
template <class real, bool SAMPLE, int NOISE, bool UNIT, bool ASTAR>
__device__ __forceinline__ void site_update(const SiteK<real>& K, const RowConst<real>& rc, const Mom<real>& m,
                                            const Pr<real>* ring, int bc, int bu, int bd, uint32_t site,
                                            uint32_t step, real* fl, real* pl, int LzLx, double& acc_p,
                                            double& acc_a, double& acc_b, Pr<real>* out, int ostride, int flags,
                                            const BmTables<real>* bm) {
  using P = Pr<real>;
  const P c9 = pr(real(1) / 9), c36 = pr(real(1) / 36);
  const P d = ring[bc];
  const P w = ring[bc - 1], e = ring[bc + 1], n = ring[bu], nw = ring[bu - 1], ne = ring[bu + 1], s = ring[bd],
          sw = ring[bd - 1], se = ring[bd + 1];
  // sum_l w_l c_l rho^S(r + c_l) of both species, deviations plus the background part (Eq. aNI)
  const P sx = fma2(c9, sub2(e, w), mul2(c36, add2(sub2(ne, nw), sub2(se, sw))));
  const P sz = add2(fma2(c9, sub2(n, s), mul2(c36, sub2(add2(ne, nw), add2(se, sw)))), pr(rc.dbgA, rc.dbgB));
  const P rs = add2(pr(rc.bgA, rc.bgB), d);  // (rho^A, rho^B)
  const real rho = rs.x + rs.y;
  const real inv = site_reciprocal(rho);
  // non-ideal forces: F^A = -G rho^A sum(rho^B), F^B = -G rho^B sum(rho^A)
  const real gA = -K.G * rs.x, gB = -K.G * rs.y;
  const real FnAx = gA * sx.y, FnAz = gA * sz.y, FnBx = gB * sx.x, FnBz = gB * sz.x;
  const real FNx = FnAx + FnBx, FNz = FnAz + FnBz;
  P Fx, Fz;
  if (ASTAR) {
    // a* makes the non-ideal acceleration common: rho^S a^S = (rho^S / rho) F_NI
    const P cs = mul2(rs, pr(inv));
    Fx = mul2(cs, pr(FNx));
    Fz = mul2(cs, pr(FNz));
  } else {
    Fx = pr(FnAx, FnBx);
    Fz = pr(FnAz, FnBz);
  }
  // gradient forcing: rho^A a^A_NE = (0, rho grad_c0 / 3) = -rho^B a^B_NE (Eq. NEcond)
  Fz = fma2(pr(rho), pr(K.g3, -K.g3), Fz);
  if (SAMPLE) {
    // pressure (half trace; kinetic + interaction), minus its background part
    const real kin = (m.m3.x + m.m3.y + 2 * (d.x + d.y)) * (real(1) / 6);
    const P N = fma2(c9, add2(add2(e, w), add2(n, s)), mul2(pr(real(2) / 36), add2(add2(ne, nw), add2(se, sw))));
    const real inter = d.x * (rc.nbB + N.y) + rc.bgA * N.y + d.y * (rc.nbA + N.x) + rc.bgB * N.x;
    const real psite = kin + real(0.25) * K.G * inter;
    pl[0] = psite;
    acc_p += (double)psite;
    acc_a += (double)d.x;
    acc_b += (double)d.y;
  }
  // barycentric velocity, Eq. (bar)
  const real Ux = (m.m1.x + m.m1.y + real(0.5) * FNx) * inv;
  const real Uz = (m.m2.x + m.m2.y + real(0.5) * FNz) * inv;
  if (SAMPLE) {
    fl[0] = d.x + d.y - K.rho_bar_off;
    fl[LzLx] = (d.x - rc.c0 * (d.x + d.y)) * inv;
    fl[2 * LzLx] = Ux;
    fl[3 * LzLx] = Uz;
  }
  P nz[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) nz[k] = pr(real(0));
  P cm = pr(real(1), real(-1)), cq = pr(real(1));  // momentum noise is equal and opposite in A and B
  if (NOISE != NOISE_OFF) {
    U4 w4[4];
    philox_site(site, step, K.lid, K.key0, K.key1, w4);
    real g[14];
    normal_pair2<real>(w4[0].x, w4[0].y, w4[0].z, w4[0].w, g[0], g[1], g[2], g[3], bm);
    normal_pair2<real>(w4[1].x, w4[1].y, w4[1].z, w4[1].w, g[4], g[5], g[6], g[7], bm);
    normal_pair2<real>(w4[2].x, w4[2].y, w4[2].z, w4[2].w, g[8], g[9], g[10], g[11], bm);
    normal_pair<real>(w4[3].x, w4[3].y, g[12], g[13], bm);
    if (NOISE == NOISE_LOC) {
      const real sm = sqrt_pos<real>(rs.x * rs.y * inv);
      cm = pr(sm, -sm);
      cq = pr(sqrt_pos<real>(rs.x), sqrt_pos<real>(rs.y));
    }
    // normals 0-1: momentum (one draw for both species); 2-7: moments 3..8 of A; 8-13: of B
    nz[1] = pr(g[0]);
    nz[2] = pr(g[1]);
#pragma unroll
    for (int k = 3; k < 9; ++k) nz[k] = pr(g[k - 1], g[k + 5]);
  }
  collide_out<real, NOISE, UNIT>(m, d, rs, Ux, Uz, Fx, Fz, K, nz, cm, cq, out, ostride);
}

__device__ __forceinline__ void block_partials(double acc_p, double acc_a, double acc_b, double* red, double* out) {
  acc_p = warp_sum(acc_p);
  acc_a = warp_sum(acc_a);
  acc_b = warp_sum(acc_b);
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    red[3 * wid + 0] = acc_p;
    red[3 * wid + 1] = acc_a;
    red[3 * wid + 2] = acc_b;
  }
  __syncthreads();
  if (tid == 0) {
    double p = 0, ma = 0, mb = 0;
    for (int w = 0; w < nw; ++w) {
      p += red[3 * w];
      ma += red[3 * w + 1];
      mb += red[3 * w + 2];
    }
    out[0] = p;
    out[1] = ma;
    out[2] = mb;
  }
}

}  // namespace

// ======================================================================================
// Shared-memory layouts.
// ======================================================================================
// Generic: reduction scratch, lattice constants, density ring (4 rows of TX + 2 pairs), stage
// (NS rows x 9 links x (TX + 2) pairs).
template <class real>
struct BmBytes {
  static constexpr size_t value = sizeof(real) == 8 ? sizeof(BmTables<double>) : 0;
};

template <class real>
struct Smem {
  static constexpr size_t red = 0;
  static constexpr size_t lat = 8 * 3 * sizeof(double);
  static constexpr size_t ring = lat + ((sizeof(LatticeDev<real>) + 15) / 16) * 16;
  __host__ __device__ static size_t stage(int tx) { return ring + (size_t)8 * (tx + 2) * sizeof(real); }
  __host__ __device__ static size_t bm(int tx) {
    return ((stage(tx) + (size_t)NS * 9 * (tx + 2) * sizeof(Pr<real>) + 15) / 16) * 16;
  }
  __host__ __device__ static size_t bytes(int tx) { return bm(tx) + BmBytes<real>::value; }
};

// Bulk: as generic, then input slots (NSI slots of SlotLayout, 128-byte aligned: the dynamic
// shared memory is declared 128-byte aligned), NSI mbarriers and an abort flag.  Both end with
// the double-precision Box-Muller tables (FP64 kernels only).
template <class real, int TX>
struct SmemBulk {
  // halo columns on each side: the densities of the columns next to the strip pull from two
  // columns out (16 or 32 bytes of pairs, so every copy stays 16-byte aligned)
  static constexpr int PAD = 2;
  static constexpr int SW = TX + 2 * PAD;
  using LAY = SlotLayout<SW, (int)sizeof(Pr<real>)>;
  static constexpr size_t red = 0;
  static constexpr size_t lat = 8 * 3 * sizeof(double);
  static constexpr size_t ring = lat + ((sizeof(LatticeDev<real>) + 15) / 16) * 16;
  static constexpr size_t in = ((ring + 8 * (TX + 2) * sizeof(real) + 127) / 128) * 128;
  static constexpr size_t bars = in + (size_t)NSI * LAY::slot * sizeof(Pr<real>);
  static constexpr size_t abort_flag = bars + NSI * sizeof(uint64_t);
  static constexpr size_t tmap = abort_flag + 8;  // the item's tensor maps (pointer), or null
  // per-link and per-run copy descriptors (int4 each), filled once per launch by bulk_init
  static constexpr size_t ptab = ((tmap + 8 + 15) / 16) * 16;
  static constexpr size_t rtab = ptab + 9 * 16;
  static constexpr size_t bm = rtab + 6 * 16;  // 16-byte entries
  static constexpr size_t bytes = bm + BmBytes<real>::value;
  static_assert(in % 128 == 0 && bars % 8 == 0 && tmap % 8 == 0 && ptab % 16 == 0 && bm % 16 == 0,
                "shared-memory regions must stay aligned");
};

// ======================================================================================
// Generic path.
// ======================================================================================
template <class real, bool SAMPLE, int NOISE>
__device__ __forceinline__ void process_item(const StepArgs<real>& a, const real* __restrict__ src,
                                             real* __restrict__ dst, int item_index, uint32_t step,
                                             unsigned char* smem) {
  double* red = reinterpret_cast<double*>(smem + Smem<real>::red);
  const BmTables<real>* bm = reinterpret_cast<const BmTables<real>*>(smem + Smem<real>::bm(blockDim.x));
  LatticeDev<real>* Ls = reinterpret_cast<LatticeDev<real>*>(smem + Smem<real>::lat);
  const int TX = blockDim.x, W = TX + 2;
  Pr<real>* ring = reinterpret_cast<Pr<real>*>(smem + Smem<real>::ring);
  Pr<real>* stage = reinterpret_cast<Pr<real>*>(smem + Smem<real>::stage(TX));

  const WorkItem it = a.items[item_index];
  __syncthreads();  // shared memory may still be read for the previous item
  {
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(a.lat + it.lattice);
    uint32_t* d32 = reinterpret_cast<uint32_t*>(Ls);
    for (int i = threadIdx.x; i < (int)(sizeof(LatticeDev<real>) / 4); i += TX) d32[i] = s32[i];
  }
  __syncthreads();
  const LatticeDev<real>& L = *Ls;
  const int Lx = L.Lx, Lz = L.Lz, LzLx = Lx * Lz;
  const int tid = threadIdx.x;
  const int nact = min(TX, Lx - it.x0);
  const bool active = tid < nact;
  const int x = it.x0 + (active ? tid : 0);
  const int xl = (it.x0 == 0) ? Lx - 1 : it.x0 - 1;
  const int xr = (it.x0 + nact == Lx) ? 0 : it.x0 + nact;
  const bool do_left = tid == 0, do_right = tid == nact - 1;
  const Pr<real>* f = reinterpret_cast<const Pr<real>*>(src + L.f_off);  // [link][z][x] pairs
  Pr<real>* g = reinterpret_cast<Pr<real>*>(dst + L.f_off);
  const real k9 = L.k9, k36 = L.k36;
  const int flags = L.flags;
  const RowConst<real>* rows = a.rows + L.row_off;
  const int z0 = it.z0, z1 = it.z1;
  // noise counter of this thread's site: z * L.site_Lx + (x + L.site_x0) mod L.site_Lx (the
  // lattice's own site index z Lx + x unless it is an x-slab window of a wider lattice), carried
  // from row to row
  uint32_t site = (uint32_t)(z0 * L.site_Lx + (x + L.site_x0) % L.site_Lx);

  auto stage_row = [&](int r) {
    if (r >= 0 && r < Lz && r <= z1) {
      Pr<real>* sb = stage + (r & (NS - 1)) * 9 * W;
      if (active) stage_column(f, LzLx, Lx, Lz, r, x, sb + tid + 1, W);
      if (do_left) stage_column(f, LzLx, Lx, Lz, r, xl, sb, W);
      if (do_right) stage_column(f, LzLx, Lx, Lz, r, xr, sb + nact + 1, W);
    }
    cp_commit();
  };
  auto rho_at = [&](int r, int c) {
    const Pr<real>* sb = stage + (r & (NS - 1)) * 9 * W;
    Pr<real> v[9];
    read_generic(sb, W, c, r > 0, r < Lz - 1, k9, k36, v);
    return sum9<real>(v);
  };
  auto put_rho = [&](int r) {
    const int b = ring_slot(r) * W;
    if (active) ring[b + tid + 1] = rho_at(r, tid + 1);
    if (do_left) ring[b] = rho_at(r, 0);
    if (do_right) ring[b + nact + 1] = rho_at(r, nact + 1);
  };
  // wall ghost row zg from the adjacent fluid row za (Sec. II.A)
  auto ghost_row = [&](int zg, int za) {
    const int bg = ring_slot(zg) * W, ba = ring_slot(za) * W;
    const bool fixed = flags & DF_WALL_FIXED;
    const real cw = rows[za].ghost_cA;
    auto copy1 = [&](int i) {
      const Pr<real> a = ring[ba + i];
      if (fixed) {
        const real t = a.x + a.y;
        ring[bg + i] = pr(t * cw, t * (1 - cw));
      } else {
        ring[bg + i] = a;
      }
    };
    if (active) copy1(tid + 1);
    if (do_left) copy1(0);
    if (do_right) copy1(nact + 1);
  };

  // prologue: rows z0-1 .. z0+NS-2 in flight, rows z0-1 and z0 landed
  for (int r = z0 - 1; r <= z0 + NS - 2; ++r) stage_row(r);
  cp_wait<NS - 2>();
  if (z0 > 0) put_rho(z0 - 1);
  put_rho(z0);
  if (z0 == 0) ghost_row(-1, 0);

  const SiteK<real> K = site_constants<real, NOISE>(L);
  double acc_p = 0.0, acc_a = 0.0, acc_b = 0.0;

  for (int z = z0; z < z1; ++z) {
    cp_wait<NS - 3>();  // row z+1 landed
    if (z + 1 < Lz) put_rho(z + 1);
    else ghost_row(Lz, Lz - 1);
    __syncthreads();
    stage_row(z + NS - 1);  // into the slot of row z-1, read by every thread before the barrier
    if (active) {
      const int bc = ring_slot(z) * W + tid + 1, bu = ring_slot(z + 1) * W + tid + 1,
                bd = ring_slot(z - 1) * W + tid + 1;
      const Pr<real>* sb = stage + (z & (NS - 1)) * 9 * W;
      const bool below = z > 0, above = z < Lz - 1;
      const int r0 = z * Lx + x;
      // the variants are inlined; the branches are uniform over the block (one lattice per item)
      auto site_at = [&](auto unit, auto astar) {
        Pr<real> v[9];
        read_generic(sb, W, tid + 1, below, above, k9, k36, v);
        Mom<real> m = moments<real>(v);
        if (below && above) m.m2 = add2(m.m2, interior_m2_shift(k9, k36));
        site_update<real, SAMPLE, NOISE, decltype(unit)::value, decltype(astar)::value>(
            K, rows[z], m, ring, bc, bu, bd, site, step, a.fields + 4 * L.site_off + r0, a.pfield + L.site_off + r0,
            LzLx, acc_p, acc_a, acc_b, g + r0, LzLx, flags, bm);
      };
      if (flags & DF_UNIT) {
        if (flags & DF_ASTAR) site_at(BoolC<true>(), BoolC<true>());
        else site_at(BoolC<true>(), BoolC<false>());
      } else {
        if (flags & DF_ASTAR) site_at(BoolC<false>(), BoolC<true>());
        else site_at(BoolC<false>(), BoolC<false>());
      }
    }
    site += (uint32_t)L.site_Lx;
  }
  cp_wait<0>();  // nothing may land in shared memory after the item
  if (SAMPLE) block_partials(acc_p, acc_a, acc_b, red, a.partials + 3 * item_index);
}

// ======================================================================================
// Bulk path (rows 16-byte aligned, TX = 32, 64, 128 or 256).
// ======================================================================================
template <class real, int TX>
__device__ __forceinline__ void bulk_init(unsigned char* smem) {
  using SM = SmemBulk<real, TX>;
  using LAY = typename SM::LAY;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SM::bars);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSI; ++i) mbar_init(bars + i, 1);
    *reinterpret_cast<volatile int*>(smem + SM::abort_flag) = 0;
    mbar_fence_init();
  }
  // link l: (slot offset, c_z, source link, source link on a reflected row); run j: (slot
  // offset, first link, first link when reflected, run length + 4 (c_z + 1))
  const int t = threadIdx.x;
  if (t < 9) {
    const int j = run_of(t);
    reinterpret_cast<int4*>(smem + SM::ptab)[t] =
        make_int4(LAY::base_of(j) + (t - run_l0(j)) * SM::SW, LB_CZ(t), t, LB_OPP(t));
  } else if (t < 15) {
    const int j = t - 9, l0 = run_l0(j);
    reinterpret_cast<int4*>(smem + SM::rtab)[j] =
        make_int4(LAY::base_of(j), l0, LB_OPP(l0), run_n(j) + 4 * (LB_CZ(l0) + 1));
  }
  __syncthreads();
}

// ph: expected parity bit per input slot, carried across items by the caller.  Returns false if
// a wait gave up (the block then stops; a.err is set).
template <class real, int TX, bool SAMPLE, int NOISE>
__device__ __forceinline__ bool process_item_bulk(const StepArgs<real>& a, const real* __restrict__ src,
                                                  real* __restrict__ dst, int item_index, uint32_t step,
                                                  unsigned char* smem, uint32_t& ph, int src_buf) {
  using SM = SmemBulk<real, TX>;
  using LAY = typename SM::LAY;
  constexpr int PAD = SM::PAD, SW = SM::SW, W = TX + 2;
  double* red = reinterpret_cast<double*>(smem + SM::red);
  const BmTables<real>* bm = reinterpret_cast<const BmTables<real>*>(smem + SM::bm);
  LatticeDev<real>* Ls = reinterpret_cast<LatticeDev<real>*>(smem + SM::lat);
  Pr<real>* ring = reinterpret_cast<Pr<real>*>(smem + SM::ring);
  Pr<real>* instage = reinterpret_cast<Pr<real>*>(smem + SM::in);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SM::bars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SM::abort_flag);

  const CUtensorMap* const* tmap_s = reinterpret_cast<const CUtensorMap* const*>(smem + SM::tmap);
  const int4* ptab = reinterpret_cast<const int4*>(smem + SM::ptab);
  const int4* rtab = reinterpret_cast<const int4*>(smem + SM::rtab);

  const WorkItem it = a.items[item_index];
  __syncthreads();  // shared memory may still be read for the previous item
  {
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(a.lat + it.lattice);
    uint32_t* d32 = reinterpret_cast<uint32_t*>(Ls);
    for (int i = threadIdx.x; i < (int)(sizeof(LatticeDev<real>) / 4); i += TX) d32[i] = s32[i];
    // the tensor maps of this lattice in the source buffer (kept in shared memory, not
    // registers); null if the input slots were not 128-byte aligned after all
    if (threadIdx.x == 0)
      *const_cast<const CUtensorMap**>(tmap_s) = a.tmaps && (smem_u32(instage) & 127u) == 0
                                                     ? a.tmaps + ((size_t)src_buf * a.n_lat + it.lattice) * 2
                                                     : nullptr;
  }
  __syncthreads();
  const LatticeDev<real>& L = *Ls;
  const int Lx = L.Lx, Lz = L.Lz, LzLx = Lx * Lz;
  const int tid = threadIdx.x;
  const int x0 = it.x0;
  const int nact = min(TX, Lx - x0);
  const bool active = tid < nact;
  const int x = x0 + (active ? tid : 0);
  const bool do_left = tid == 0, do_right = tid == nact - 1;
  const Pr<real>* f = reinterpret_cast<const Pr<real>*>(src + L.f_off);  // [link][z][x] pairs
  Pr<real>* g = reinterpret_cast<Pr<real>*>(dst + L.f_off);
  const real k9 = L.k9, k36 = L.k36;
  const int flags = L.flags;
  const RowConst<real>* rows = a.rows + L.row_off;
  const int z0 = it.z0, z1 = it.z1;
  // noise counter of this thread's site: z * L.site_Lx + (x + L.site_x0) mod L.site_Lx (the
  // lattice's own site index z Lx + x unless it is an x-slab window of a wider lattice), carried
  // from row to row
  uint32_t site = (uint32_t)(z0 * L.site_Lx + (x + L.site_x0) % L.site_Lx);
  const unsigned row_bytes = 9u * (unsigned)(nact + 2 * PAD) * (unsigned)sizeof(Pr<real>);

  // copy k of row r (link row k, or run k on the tensor path; its source row, reflected at the
  // walls) is issued by lane k / NW of warp k % NW, so that every warp issues about the same
  // number of copies
  constexpr int NW = TX / 32;
  const int my_plane = (tid & 31) * NW + (tid >> 5);
  // row r goes to input slot r mod NSI; the callers carry the slots along
  auto stage_row = [&](int r, int slot) {
    if (r < 0 || r >= Lz || r > z1) return;
    uint64_t* bar = bars + slot;
    Pr<real>* sbase = instage + slot * LAY::slot;
    if (tid == 0) mbar_expect_tx(bar, row_bytes);
    const unsigned sz = (unsigned)sizeof(Pr<real>);
    // interior strips (no periodic wrap) with tensor maps: one 3-d tensor copy per run of links;
    // otherwise one 1-d bulk copy (or up to three at the x edges) per link row
    if (TX + 2 * PAD <= 256 && a.tmaps != nullptr && x0 > 0 && x0 + nact < Lx) {
      if (my_plane < 6) {
        const CUtensorMap* maps = *tmap_s;
        const int4 e = rtab[my_plane];
        const int n = e.w & 3;
        int sr = r - ((e.w >> 2) - 1), ls = e.y;
        if (sr < 0 || sr >= Lz) {
          sr = r;
          ls = e.z;
        }
        Pr<real>* d = sbase + e.x;
        if (maps) {
          tensor_g2s(d, maps + (n - 1), x0 - PAD, sr, ls, bar);
        } else {  // the same box as 1-d copies, one per link row
          for (int q = 0; q < n; ++q)
            bulk_g2s(d + q * SW, f + (size_t)(ls + q) * LzLx + (size_t)sr * Lx + x0 - PAD, (unsigned)SW * sz, bar);
        }
      }
    } else if (my_plane < 9) {
      const int4 e = ptab[my_plane];
      int sr = r - e.y, p = e.z;
      if (sr < 0 || sr >= Lz) {
        sr = r;
        p = e.w;
      }
      const Pr<real>* rowp = f + (size_t)p * LzLx + (size_t)sr * Lx;
      Pr<real>* d = sbase + e.x;
      if (x0 > 0 && x0 + nact < Lx) {
        bulk_g2s(d, rowp + x0 - PAD, (unsigned)(nact + 2 * PAD) * sz, bar);
      } else {
        bulk_g2s(d, rowp + (x0 == 0 ? Lx - PAD : x0 - PAD), PAD * sz, bar);
        if (x0 + nact < Lx) {
          bulk_g2s(d + PAD, rowp + x0, (unsigned)(nact + PAD) * sz, bar);
        } else {
          bulk_g2s(d + PAD, rowp + x0, (unsigned)nact * sz, bar);
          bulk_g2s(d + PAD + nact, rowp, PAD * sz, bar);
        }
      }
    }
  };
  auto wait_row = [&](int slot) {
    const unsigned par = (ph >> slot) & 1u;
    if (!mbar_try_wait(bars + slot, par)) {
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(bars + slot, par)) {
        if (*abort_flag) break;
        if (global_ns() - t0 > (uint64_t)WAIT_MS * 1000000ull) {
          *abort_flag = 1;
          atomicExch(a.err, 1);
          break;
        }
      }
    }
    ph ^= 1u << slot;
  };
  auto rho_at = [&](int r, int slot, int j) {
    const Pr<real>* sb = instage + slot * LAY::slot;
    Pr<real> v[9];
    read_bulk<real, SW>(sb, j, r > 0, r < Lz - 1, k9, k36, v);
    return sum9<real>(v);
  };
  auto put_rho = [&](int r, int slot) {
    wait_row(slot);
    const int b = ring_slot(r) * W;
    if (active) ring[b + tid + 1] = rho_at(r, slot, tid + PAD);
    if (do_left) ring[b] = rho_at(r, slot, PAD - 1);
    if (do_right) ring[b + nact + 1] = rho_at(r, slot, nact + PAD);
  };
  auto ghost_row = [&](int zg, int za) {
    const int bg = ring_slot(zg) * W, ba = ring_slot(za) * W;
    const bool fixed = flags & DF_WALL_FIXED;
    const real cw = rows[za].ghost_cA;
    auto copy1 = [&](int i) {
      const Pr<real> a = ring[ba + i];
      if (fixed) {
        const real t = a.x + a.y;
        ring[bg + i] = pr(t * cw, t * (1 - cw));
      } else {
        ring[bg + i] = a;
      }
    };
    if (active) copy1(tid + 1);
    if (do_left) copy1(0);
    if (do_right) copy1(nact + 1);
  };
  // prologue: rows z0-1 .. z0+NSI-2 in flight
  auto slot_of = [](int r) { return (int)((unsigned)(r + NSI) % NSI); };  // r >= -1
  for (int r = z0 - 1; r <= z0 + NSI - 2; ++r) stage_row(r, slot_of(r));
  if (z0 > 0) put_rho(z0 - 1, slot_of(z0 - 1));
  put_rho(z0, slot_of(z0));
  if (z0 == 0) ghost_row(-1, 0);
  int sp = slot_of(z0 - 1), sc = slot_of(z0), sn = slot_of(z0 + 1);  // slots of rows z-1, z, z+1

  const SiteK<real> K = site_constants<real, NOISE>(L);
  double acc_p = 0.0, acc_a = 0.0, acc_b = 0.0;
  bool ok = true;

  for (int z = z0; z < z1; ++z) {
    if (z + 1 < Lz) put_rho(z + 1, sn);
    else ghost_row(Lz, Lz - 1);
    __syncthreads();
    if (*abort_flag) {
      ok = false;
      break;
    }
    stage_row(z + NSI - 1, sp);  // row z+NSI-1 shares the slot of row z-1, read by all before the barrier
    if (active) {
      const int bc = ring_slot(z) * W + tid + 1, bu = ring_slot(z + 1) * W + tid + 1,
                bd = ring_slot(z - 1) * W + tid + 1;
      const Pr<real>* sb = instage + sc * LAY::slot;
      const bool below = z > 0, above = z < Lz - 1;
      const int r0 = z * Lx + x;
      // the variants are inlined; the branches are uniform over the block (one lattice per item,
      // one row at a time): unit rates, a*, and interior rows (no wall within one link)
      auto site_at = [&](auto unit, auto astar, auto inner) {
        constexpr bool IN = decltype(inner)::value;
        Pr<real> v[9];
        read_bulk<real, SW>(sb, tid + PAD, IN || below, IN || above, k9, k36, v);
        Mom<real> m = moments<real>(v);
        if (IN) m.m2 = add2(m.m2, interior_m2_shift(k9, k36));
        site_update<real, SAMPLE, NOISE, decltype(unit)::value, decltype(astar)::value>(
            K, rows[z], m, ring, bc, bu, bd, site, step, a.fields + 4 * L.site_off + r0, a.pfield + L.site_off + r0,
            LzLx, acc_p, acc_a, acc_b, g + r0, LzLx, flags, bm);
      };
      auto rates = [&](auto inner) {
        if (flags & DF_UNIT) {
          if (flags & DF_ASTAR) site_at(BoolC<true>(), BoolC<true>(), inner);
          else site_at(BoolC<true>(), BoolC<false>(), inner);
        } else {
          if (flags & DF_ASTAR) site_at(BoolC<false>(), BoolC<true>(), inner);
          else site_at(BoolC<false>(), BoolC<false>(), inner);
        }
      };
      if (below && above) rates(BoolC<true>());
      else rates(BoolC<false>());
    }
    sp = sc;
    sc = sn;
    sn = sn + 1 == NSI ? 0 : sn + 1;
    site += (uint32_t)L.site_Lx;
  }
  if (!ok) {
    // drain the input rows still in flight (bounded), then stop
    if (tid == 0) {
      for (int i = 0; i < NSI; ++i) {
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(bars + i, (ph >> i) & 1u) && global_ns() - t0 < 100000000ull) {
        }
      }
    }
    __syncthreads();
    return false;
  }
  if (SAMPLE) block_partials(acc_p, acc_a, acc_b, red, a.partials + 3 * item_index);
  return true;
}

// ======================================================================================
// Kernels.
// ======================================================================================
// The FP64 noise tables of the block (before its first item; none in FP32 or without noise).
template <class real, int NOISE>
__device__ __forceinline__ void prepare_bm(unsigned char* p) {
  if constexpr (sizeof(real) == 8 && NOISE != NOISE_OFF) {
    fill_bm_tables<real>(reinterpret_cast<BmTables<real>*>(p));
    __syncthreads();
  }
}

template <class real>
struct MinBlocks {
  static constexpr int value = sizeof(real) == 4 ? 2 : 1;
};

template <class real, bool SAMPLE, int NOISE>
__global__ void __launch_bounds__(256, MinBlocks<real>::value) step_kernel(StepArgs<real> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t step = (uint32_t)(*a.d_t + a.t_offset);
  prepare_bm<real, NOISE>(smem + Smem<real>::bm(blockDim.x));
  process_item<real, SAMPLE, NOISE>(a, a.src, a.dst, blockIdx.x, step, smem);
}

template <class real>
struct BulkBlocks {  // 128-thread blocks per SM the bulk kernels are compiled for
  static constexpr int value = sizeof(real) == 4 ? LB_BULK_BLOCKS_F32 : 2;
};
// The persistent kernel runs plain steps only (a sample step is an ordinary launch after it), so
// it targets the blocks per SM of the step kernels.
template <class real>
struct PersistentBlocks {
  static constexpr int value = BulkBlocks<real>::value;
};

template <class real, int TX, bool SAMPLE, int NOISE>
__global__ void __launch_bounds__(TX, BulkBlocks<real>::value * 128 / TX) step_kernel_bulk(StepArgs<real> a) {
  static_assert(TX == 32 || TX == 64 || TX == 128 || TX == 256, "bulk tiles are 32, 64, 128 or 256 columns");
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t step = (uint32_t)(*a.d_t + a.t_offset);
  bulk_init<real, TX>(smem);
  prepare_bm<real, NOISE>(smem + SmemBulk<real, TX>::bm);
  uint32_t ph = 0;
  process_item_bulk<real, TX, SAMPLE, NOISE>(a, a.src, a.dst, blockIdx.x, step, smem, ph, a.src_buf);
}

// ---- the persistent launch: items handed out in order, per-item dependencies -------------
// Tickets t = 0, 1, ... come from one counter (PersistArgs::counter, zero at launch): ticket t is
// item t mod n_items of step t / n_items of the launch, so the items of a step go to whichever
// block is free, longest first, and blocks roll on into the next step without a grid-wide
// barrier.  done[i] counts the steps of the launch that item i has completed.  Item i may run
// step k once every item whose region lies within the rows and columns it reads (its own and
// the two-row / four-column halo of its streaming, density and aligned staging windows:
// nbr[nbr_off[i] .. nbr_off[i + 1]), itself included) has completed step k - 1: then everything
// it reads is written, and no one still reads the region it overwrites.  The relation is
// symmetric and the tickets an item waits on were all handed out before its own, so with every
// block resident (cooperative launch) each wait ends; it is bounded all the same.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until done[list[q]] >= need for all q (pausing 32 ns .. 1 us between polls);
// false, for the whole block, if the wait gave up after limit_ms (err is then set) or another
// block reported an error.  The data behind the flags are then read through bulk copies (the
// async proxy), hence the proxy fence.
static __device__ bool wait_items(const unsigned* done, const int* list, int cnt, unsigned need, int* err, int limit_ms) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint64_t t0 = global_ns(), lim = (uint64_t)limit_ms * 1000000ull;
    for (int q = 0; q < cnt && ok; ++q) {
      unsigned pause = 32;
      while (ld_acquire(done + list[q]) < need) {
        if (*(volatile int*)err) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > lim) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(pause);
        if (pause < 1024) pause <<= 1;
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return ok_s != 0;
}

// Every thread of the block has issued its stores of the item; thread 0 makes them visible and
// then sets done[i] = value.
__device__ __forceinline__ void publish_item(unsigned* done, int i, unsigned value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(done + i, value);
  }
}

// The next ticket of the block (thread 0 draws it; block-uniform result).  The item's own first
// barrier orders every read of the shared copy before thread 0 replaces it.
__device__ __forceinline__ unsigned long long next_ticket(unsigned long long* counter) {
  __shared__ unsigned long long t_s;
  if (threadIdx.x == 0) t_s = atomicAdd(counter, 1ull);
  __syncthreads();
  return t_s;
}

// nsteps plain steps in one cooperative launch.
template <class real, int NOISE>
__global__ void __launch_bounds__(256, MinBlocks<real>::value)
    persistent_kernel(StepArgs<real> a, int nsteps, PersistArgs p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t t0 = *a.d_t + a.t_offset;
  prepare_bm<real, NOISE>(smem + Smem<real>::bm(blockDim.x));
  const unsigned long long n = (unsigned)a.n_items, total = (unsigned long long)nsteps * n;
  for (unsigned long long t; (t = next_ticket(p.counter)) < total;) {
    const int k = (int)(t / n), i = (int)(t - (unsigned long long)k * n);
    if (k > 0 && !wait_items(p.done, p.nbr + p.nbr_off[i], p.nbr_off[i + 1] - p.nbr_off[i], (unsigned)k, p.err,
                             p.limit_ms))
      return;
    const bool odd = (k & 1) && !p.trial;
    const real* src = odd ? a.dst : a.src;
    real* dst = odd ? const_cast<real*>(a.src) : a.dst;
    process_item<real, false, NOISE>(a, src, dst, i, (uint32_t)(t0 + k), smem);
    publish_item(p.done, i, (unsigned)(k + 1));
  }
}

template <class real, int TX, int NOISE>
__global__ void __launch_bounds__(TX, PersistentBlocks<real>::value * 128 / TX)
    persistent_kernel_bulk(StepArgs<real> a, int nsteps, PersistArgs p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t t0 = *a.d_t + a.t_offset;
  bulk_init<real, TX>(smem);
  prepare_bm<real, NOISE>(smem + SmemBulk<real, TX>::bm);
  uint32_t ph = 0;
  const unsigned long long n = (unsigned)a.n_items, total = (unsigned long long)nsteps * n;
  for (unsigned long long t; (t = next_ticket(p.counter)) < total;) {
    const int k = (int)(t / n), i = (int)(t - (unsigned long long)k * n);
    if (k > 0 && !wait_items(p.done, p.nbr + p.nbr_off[i], p.nbr_off[i + 1] - p.nbr_off[i], (unsigned)k, p.err,
                             p.limit_ms))
      return;
    const bool odd = (k & 1) && !p.trial;
    const real* src = odd ? a.dst : a.src;
    real* dst = odd ? const_cast<real*>(a.src) : a.dst;
    if (!process_item_bulk<real, TX, false, NOISE>(a, src, dst, i, (uint32_t)(t0 + k), smem, ph,
                                                   a.src_buf ^ (odd ? 1 : 0)))
      return;  // the blocks that wait on this item give up (bounded)
    publish_item(p.done, i, (unsigned)(k + 1));
  }
}

// ======================================================================================
// Host side.
// ======================================================================================
template <class real>
size_t step_smem_bytes(int tile_x) {
  return Smem<real>::bytes(tile_x);
}

// ---- kernel families ------------------------------------------------------------------
// The kernels come in families that are compiled in translation units of their own (so that the
// build runs in parallel): TX = 0 is the generic path (any tile width), TX = 32, 64, 128 the bulk
// path of that width.  A family prepares its kernels' shared-memory limits, launches one step
// and hands out its persistent kernel; the dispatch below only sees these declarations.
template <class real, int TX>
cudaError_t family_prepare(int max_tile_x);
template <class real, int TX>
void family_launch(const StepArgs<real>& a, int tile_x, bool sample, int noise, cudaStream_t s);
template <class real, int TX>
const void* family_persistent(int tile_x, int noise, size_t* smem);

#ifdef LB_STEP_FAMILY_DEFS
static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class real, int TX>
struct Family {
  static size_t smem(int tile_x) { return TX == 0 ? Smem<real>::bytes(tile_x) : SmemBulk<real, TX == 0 ? 32 : TX>::bytes; }
  template <bool SAMPLE, int NOISE>
  static const void* step_fn() {
    if constexpr (TX == 0) return (const void*)step_kernel<real, SAMPLE, NOISE>;
    else return (const void*)step_kernel_bulk<real, TX, SAMPLE, NOISE>;
  }
  template <int NOISE>
  static const void* persistent_fn() {
    if constexpr (TX == 0) return (const void*)persistent_kernel<real, NOISE>;
    else return (const void*)persistent_kernel_bulk<real, TX, NOISE>;
  }
  template <bool SAMPLE, int NOISE>
  static void launch(const StepArgs<real>& a, int tile_x, cudaStream_t s) {
    if constexpr (TX == 0) step_kernel<real, SAMPLE, NOISE><<<a.n_items, tile_x, smem(tile_x), s>>>(a);
    else step_kernel_bulk<real, TX, SAMPLE, NOISE><<<a.n_items, TX, smem(TX), s>>>(a);
  }
};

template <class real, int TX>
cudaError_t family_prepare(int max_tile_x) {
  using F = Family<real, TX>;
  const size_t b = F::smem(max_tile_x);
  const void* fns[] = {F::template step_fn<true, NOISE_OFF>(),  F::template step_fn<true, NOISE_HOM>(),
                       F::template step_fn<true, NOISE_LOC>(),  F::template step_fn<false, NOISE_OFF>(),
                       F::template step_fn<false, NOISE_HOM>(), F::template step_fn<false, NOISE_LOC>(),
                       F::template persistent_fn<NOISE_OFF>(),  F::template persistent_fn<NOISE_HOM>(),
                       F::template persistent_fn<NOISE_LOC>()};
  for (const void* fn : fns) {
    cudaError_t e = set_smem(fn, b);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class real, int TX>
void family_launch(const StepArgs<real>& a, int tile_x, bool sample, int noise, cudaStream_t s) {
  using F = Family<real, TX>;
  if (sample) {
    if (noise == NOISE_HOM) F::template launch<true, NOISE_HOM>(a, tile_x, s);
    else if (noise == NOISE_LOC) F::template launch<true, NOISE_LOC>(a, tile_x, s);
    else F::template launch<true, NOISE_OFF>(a, tile_x, s);
  } else {
    if (noise == NOISE_HOM) F::template launch<false, NOISE_HOM>(a, tile_x, s);
    else if (noise == NOISE_LOC) F::template launch<false, NOISE_LOC>(a, tile_x, s);
    else F::template launch<false, NOISE_OFF>(a, tile_x, s);
  }
}

template <class real, int TX>
const void* family_persistent(int tile_x, int noise, size_t* smem) {
  using F = Family<real, TX>;
  *smem = F::smem(tile_x);
  if (noise == NOISE_HOM) return F::template persistent_fn<NOISE_HOM>();
  if (noise == NOISE_LOC) return F::template persistent_fn<NOISE_LOC>();
  return F::template persistent_fn<NOISE_OFF>();
}

#define LB_STEP_FAMILY_INST(real, TX)                                                                            \
  template cudaError_t family_prepare<real, TX>(int);                                                            \
  template void family_launch<real, TX>(const StepArgs<real>&, int, bool, int, cudaStream_t);                    \
  template const void* family_persistent<real, TX>(int, int, size_t*);
#endif  // LB_STEP_FAMILY_DEFS

template <class real>
cudaError_t prepare_step(int max_tile_x) {
  cudaError_t e = family_prepare<real, 0>(max_tile_x);
  if (e == cudaSuccess) e = family_prepare<real, 32>(32);
  if (e == cudaSuccess) e = family_prepare<real, 64>(64);
  if (e == cudaSuccess) e = family_prepare<real, 128>(128);
  if (e == cudaSuccess) e = family_prepare<real, 256>(256);
  return e;
}

template <class real>
cudaError_t launch_step(const StepArgs<real>& a, int tile_x, bool sample, int noise, bool bulk, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  if (bulk && tile_x == 32) family_launch<real, 32>(a, tile_x, sample, noise, s);
  else if (bulk && tile_x == 64) family_launch<real, 64>(a, tile_x, sample, noise, s);
  else if (bulk && tile_x == 128) family_launch<real, 128>(a, tile_x, sample, noise, s);
  else if (bulk && tile_x == 256) family_launch<real, 256>(a, tile_x, sample, noise, s);
  else family_launch<real, 0>(a, tile_x, sample, noise, s);
  return cudaGetLastError();
}

template <class real>
static const void* persistent_fn(int tile_x, int noise, bool bulk, size_t* smem) {
  if (bulk && tile_x == 32) return family_persistent<real, 32>(tile_x, noise, smem);
  if (bulk && tile_x == 64) return family_persistent<real, 64>(tile_x, noise, smem);
  if (bulk && tile_x == 128) return family_persistent<real, 128>(tile_x, noise, smem);
  if (bulk && tile_x == 256) return family_persistent<real, 256>(tile_x, noise, smem);
  return family_persistent<real, 0>(tile_x, noise, smem);
}

template <class real>
int persistent_grid(int tile_x, int noise, bool bulk) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = 0;
  const void* fn = persistent_fn<real>(tile_x, noise, bulk, &smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, tile_x, smem) != cudaSuccess) return 0;
  return per * sms;
}

template <class real>
cudaError_t launch_step_persistent(const StepArgs<real>& a, int tile_x, int nsteps, int noise, bool bulk,
                                   const PersistArgs& p, int grid, cudaStream_t s) {
  StepArgs<real> aa = a;
  int ns = nsteps;
  PersistArgs pp = p;
  void* args[] = {&aa, &ns, &pp};
  size_t smem = 0;
  const void* fn = persistent_fn<real>(tile_x, noise, bulk, &smem);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tile_x), args, smem, s);
}

// The normals of the step kernels for given Philox word pairs (test hook): thread j forms pairs
// 2j and 2j + 1 together as the step kernels do, a trailing odd pair alone.
template <class real>
__global__ void debug_normals_kernel(const uint32_t* __restrict__ words, int64_t n_pairs, double* __restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  prepare_bm<real, NOISE_HOM>(smem);
  const BmTables<real>* bm = reinterpret_cast<const BmTables<real>*>(smem);
  const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i + 1 < n_pairs) {
    real n[4];
    normal_pair2<real>(words[2 * i], words[2 * i + 1], words[2 * i + 2], words[2 * i + 3], n[0], n[1], n[2], n[3],
                       bm);
    for (int k = 0; k < 4; ++k) out[2 * i + k] = (double)n[k];
  } else if (i < n_pairs) {
    real n0, n1;
    normal_pair<real>(words[2 * i], words[2 * i + 1], n0, n1, bm);
    out[2 * i] = (double)n0;
    out[2 * i + 1] = (double)n1;
  }
}

template <class real>
cudaError_t launch_debug_normals(const uint32_t* words, int64_t n_pairs, double* out, cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  const int64_t blocks = ((n_pairs + 1) / 2 + 255) / 256;
  const size_t smem = BmBytes<real>::value;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(debug_normals_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  debug_normals_kernel<real><<<(unsigned)blocks, 256, smem, s>>>(words, n_pairs, out);
  return cudaGetLastError();
}

#ifdef LB_STEP_COMMON_DEFS
// Kernels and helpers that do not depend on the precision (compiled once).
__global__ void advance_kernel(int64_t* d_t, int64_t k) { *d_t += k; }

// Block b marks itself done and waits (bounded) until blocks list[0 .. expected) are.
__global__ void barrier_probe_kernel(unsigned* done, const int* list, int* err, int expected, int limit_ms) {
  publish_item(done, blockIdx.x, 1u);
  wait_items(done, list, expected, 1u, err, limit_ms);
}

cudaError_t launch_advance(int64_t* d_t, int64_t k, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(d_t, k);
  return cudaGetLastError();
}

cudaError_t launch_barrier_probe(int blocks, int expected, int limit_ms, unsigned* done, const int* list, int* err,
                                 cudaStream_t s) {
  void* args[] = {&done, &list, &err, &expected, &limit_ms};
  return cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(blocks), dim3(32), args, 0, s);
}

#endif

}  // namespace lbk
