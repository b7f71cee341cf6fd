// lb_step.cu -- the fused per-step kernel of the fluctuating two-species D2Q9 MRT method
// (Eq. LB with Eq. MRT), one launch per step for every lattice of a batch, or one
// cooperative launch with a bounded grid barrier between steps.
//
// Work decomposition: a block of TX threads owns TX consecutive columns x of one lattice
// and marches up rows z0..z1-1 of that lattice.  Each thread pulls the 18 populations of its
// own site (Eq. LB, mid-way bounce-back at the walls of Sec. II.A), so every stored value
// is read once per step from HBM with coalesced loads.  The non-ideal force (Eq. aNI) needs
// the densities of the 8 neighbours at the same time level: each thread keeps the pulled
// row z+1 in registers while it collides row z, and the densities of rows z-1, z, z+1 live
// in a 4-slot shared-memory ring (one __syncthreads per row).  The two halo columns are
// pulled by the edge threads.  The wall ghost rows follow Sec. II.A.
//
// Arithmetic per site: densities and momenta from the pulled populations, forces
// (Eqs. aNI, ne-acc, a* of its footnote), barycentric velocity (Eq. bar), moments of
// Table I in their structured +- form, relaxation toward m^eq with second-order forcing
// (1 - lambda_a/2) S_a, FDT noise from Philox4x32-10 (Eqs. noise-bin-expl,
// noise-bin-expl-high), and the inverse transform f_l = w_l sum_a T_al m*_a / N_a.
#include <cstdio>

#include "lb_internal.cuh"

namespace lbk {

namespace {

__device__ __forceinline__ int ring_slot(int z) { return (z + 4) & 3; }

// Pull the 18 populations arriving at (x, z) (Eq. LB): link l comes from (x - c_lx, z - c_lz);
// a link whose source row lies beyond a wall is the reflected population f*_opp(l)(x, z).
// In deviation mode the background difference b_l(z - c_lz) - b_l(z) = -w_l rho_bar c_lz
// d_z c^S_0 is added on non-reflected links with c_lz != 0 (zero on reflected links).
template <class real>
__device__ __forceinline__ void pull_site(const real* __restrict__ f, int LzLx, int Lx, int Lz, int z, int x, int xm,
                                          int xp, real k9, real k36, real v[18], real& dA, real& dB) {
  const bool below = z > 0;
  const bool above = z < Lz - 1;
  const int r0 = z * Lx, rdn = r0 - Lx, rup = r0 + Lx;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const real* fs = f + s * 9 * LzLx;
    const real q9 = s == 0 ? k9 : -k9, q36 = s == 0 ? k36 : -k36;
    real* w = v + 9 * s;
    w[0] = fs[0 * LzLx + r0 + x];
    w[1] = fs[1 * LzLx + r0 + xm];
    w[3] = fs[3 * LzLx + r0 + xp];
    w[2] = below ? fs[2 * LzLx + rdn + x] - q9 : fs[4 * LzLx + r0 + x];
    w[4] = above ? fs[4 * LzLx + rup + x] + q9 : fs[2 * LzLx + r0 + x];
    w[5] = below ? fs[5 * LzLx + rdn + xm] - q36 : fs[7 * LzLx + r0 + x];
    w[6] = below ? fs[6 * LzLx + rdn + xp] - q36 : fs[8 * LzLx + r0 + x];
    w[7] = above ? fs[7 * LzLx + rup + xp] + q36 : fs[5 * LzLx + r0 + x];
    w[8] = above ? fs[8 * LzLx + rup + xm] + q36 : fs[6 * LzLx + r0 + x];
  }
  dA = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
  dB = ((v[9] + v[10]) + (v[11] + v[12])) + ((v[13] + v[14]) + (v[15] + v[16])) + v[17];
}

// Density deviations only (halo columns and the row below an item's first row).
template <class real>
__device__ __forceinline__ void pull_rho(const real* __restrict__ f, int LzLx, int Lx, int Lz, int z, int x, real k9,
                                         real k36, real& dA, real& dB) {
  const int xm = (x == 0) ? Lx - 1 : x - 1;
  const int xp = (x + 1 == Lx) ? 0 : x + 1;
  real v[18];
  pull_site(f, LzLx, Lx, Lz, z, x, xm, xp, k9, k36, v, dA, dB);
}

template <class real>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One collision of species S in moment space (Eq. MRT) with second-order forcing and noise;
// v: the 9 pulled deviations; d: their sum; rs: the full density rho^S; (Fx, Fz): rho^S a^S.
// Writes the 9 post-collision deviations back into v.
template <class real>
__device__ __forceinline__ void collide_species(real v[9], real d, real rs, real Ux, real Uz, real Fx, real Fz,
                                                const real lam[9], const real omh[9], const real xi[9]) {
  // moments of Table I in the structured form
  const real a57 = v[5] - v[7], a68 = v[6] - v[8];
  const real d13 = v[1] - v[3], d24 = v[2] - v[4];
  const real e = (v[1] + v[3]) + (v[2] + v[4]);
  const real dg = (v[5] + v[7]) + (v[6] + v[8]);
  const real m1 = d13 + a57 - a68;
  const real m2 = d24 + a57 + a68;
  const real m3 = -2 * v[0] + e + 4 * dg;
  const real m4 = (v[1] + v[3]) - (v[2] + v[4]);
  const real m5 = (v[5] + v[7]) - (v[6] + v[8]);
  const real m6 = -d13 + 2 * (a57 - a68);
  const real m7 = -d24 + 2 * (a57 + a68);
  const real m8 = 2 * v[0] - 4 * e + 8 * dg;
  const real UxUx = Ux * Ux, UzUz = Uz * Uz;
  // relaxation toward m^eq(rho^S, U) of Table I, forcing moments S_a, noise xi_a
  const real s1 = m1 + lam[1] * (rs * Ux - m1) + omh[1] * Fx + xi[1];
  const real s2 = m2 + lam[2] * (rs * Uz - m2) + omh[2] * Fz + xi[2];
  const real s3 = m3 + lam[3] * (3 * rs * (UxUx + UzUz) - m3) + omh[3] * (6 * (Ux * Fx + Uz * Fz)) + xi[3];
  const real s4 = m4 + lam[4] * (rs * (UxUx - UzUz) - m4) + omh[4] * (2 * (Ux * Fx - Uz * Fz)) + xi[4];
  const real s5 = m5 + lam[5] * (rs * Ux * Uz - m5) + omh[5] * (Ux * Fz + Uz * Fx) + xi[5];
  const real s6 = m6 - lam[6] * m6 + xi[6];
  const real s7 = m7 - lam[7] * m7 + xi[7];
  const real s8 = m8 - lam[8] * m8 + xi[8];
  // divide by N_a = (1, 1/3, 1/3, 4, 4/9, 1/9, 2/3, 2/3, 16)
  const real M0 = d, M1 = 3 * s1, M2 = 3 * s2, M3 = real(0.25) * s3, M4 = real(2.25) * s4, M5 = 9 * s5,
             M6 = real(1.5) * s6, M7 = real(1.5) * s7, M8 = real(0.0625) * s8;
  // f_l = w_l sum_a T_al M_a
  const real c9 = real(1) / 9, c36 = real(1) / 36;
  const real base4 = M0 + M3 - 4 * M8;
  const real base5 = M0 + 4 * M3 + 8 * M8;
  v[0] = real(4) / 9 * (M0 - 2 * M3 + 2 * M8);
  v[1] = c9 * (base4 + M1 + M4 - M6);
  v[3] = c9 * (base4 - M1 + M4 + M6);
  v[2] = c9 * (base4 + M2 - M4 - M7);
  v[4] = c9 * (base4 - M2 - M4 + M7);
  const real p12 = M1 + M2, p1m2 = M1 - M2, q67 = 2 * (M6 + M7), q6m7 = 2 * (M6 - M7);
  v[5] = c36 * (base5 + p12 + M5 + q67);
  v[7] = c36 * (base5 - p12 + M5 - q67);
  v[6] = c36 * (base5 - p1m2 - M5 - q6m7);
  v[8] = c36 * (base5 + p1m2 - M5 + q6m7);
}

}  // namespace

// Advance one work item by one step.  ring: 2 x 4 x (TX + 2) reals of shared memory.
template <class real, bool SAMPLE, bool NOISE>
__device__ __forceinline__ void process_item(const StepArgs<real>& a, const real* __restrict__ src, real* __restrict__ dst,
                                             int item_index, uint32_t step, real* ringA, real* ringB,
                                             double* red) {
  const WorkItem it = a.items[item_index];
  const LatticeDev<real>& L = a.lat[it.lattice];
  const int Lx = L.Lx, Lz = L.Lz, LzLx = Lx * Lz;
  const int tid = threadIdx.x, TX = blockDim.x, W = TX + 2;
  const int nact = min(TX, Lx - it.x0);
  const bool active = tid < nact;
  const int x = it.x0 + (active ? tid : 0);
  const int xm = (x == 0) ? Lx - 1 : x - 1;
  const int xp = (x + 1 == Lx) ? 0 : x + 1;
  const int xl = (it.x0 == 0) ? Lx - 1 : it.x0 - 1;
  const int xr = (it.x0 + nact == Lx) ? 0 : it.x0 + nact;
  const bool do_left = tid == 0, do_right = tid == nact - 1;
  const real* f = src + L.f_off;
  real* g = dst + L.f_off;
  const real k9 = L.k9, k36 = L.k36;
  const int flags = L.flags;
  const RowConst<real>* rows = a.rows + L.row_off;

  __syncthreads();  // the ring may still be read for the previous item

  // densities of row z (own column and halo columns) into the ring
  auto put_rho = [&](int z, real dA, real dB) {
    const int b = ring_slot(z) * W;
    if (active) {
      ringA[b + tid + 1] = dA;
      ringB[b + tid + 1] = dB;
    }
    if (do_left) {
      real hA, hB;
      pull_rho(f, LzLx, Lx, Lz, z, xl, k9, k36, hA, hB);
      ringA[b] = hA;
      ringB[b] = hB;
    }
    if (do_right) {
      real hA, hB;
      pull_rho(f, LzLx, Lx, Lz, z, xr, k9, k36, hA, hB);
      ringA[b + nact + 1] = hA;
      ringB[b + nact + 1] = hB;
    }
  };
  // wall ghost row zg from the adjacent fluid row za (Sec. II.A)
  auto ghost_row = [&](int zg, int za) {
    const int bg = ring_slot(zg) * W, ba = ring_slot(za) * W;
    const bool fixed = flags & DF_WALL_FIXED;
    const real cw = rows[za].ghost_cA;
    auto copy1 = [&](int i) {
      const real A = ringA[ba + i], B = ringB[ba + i];
      if (fixed) {
        const real t = A + B;
        ringA[bg + i] = t * cw;
        ringB[bg + i] = t * (1 - cw);
      } else {
        ringA[bg + i] = A;
        ringB[bg + i] = B;
      }
    };
    if (active) copy1(tid + 1);
    if (do_left) copy1(0);
    if (do_right) copy1(nact + 1);
  };

  real cur[18], dA = 0, dB = 0;
  if (active) pull_site(f, LzLx, Lx, Lz, it.z0, x, xm, xp, k9, k36, cur, dA, dB);
  put_rho(it.z0, dA, dB);
  if (it.z0 > 0) {
    real pA = 0, pB = 0;
    if (active) pull_rho(f, LzLx, Lx, Lz, it.z0 - 1, x, k9, k36, pA, pB);
    put_rho(it.z0 - 1, pA, pB);
  } else {
    ghost_row(-1, 0);
  }

  double acc_p = 0.0, acc_a = 0.0, acc_b = 0.0;
  const real G = L.G;

  for (int z = it.z0; z < it.z1; ++z) {
    real nxt[18], nA = 0, nB = 0;
    if (z + 1 < Lz) {
      if (active) pull_site(f, LzLx, Lx, Lz, z + 1, x, xm, xp, k9, k36, nxt, nA, nB);
      put_rho(z + 1, nA, nB);
    } else {
      ghost_row(Lz, Lz - 1);
    }
    __syncthreads();

    if (active) {
      const RowConst<real> rc = rows[z];
      const int bc = ring_slot(z) * W + tid + 1, bu = ring_slot(z + 1) * W + tid + 1,
                bd = ring_slot(z - 1) * W + tid + 1;
      const real Aw = ringA[bc - 1], Ae = ringA[bc + 1], An = ringA[bu], Anw = ringA[bu - 1], Ane = ringA[bu + 1],
                 As = ringA[bd], Asw = ringA[bd - 1], Ase = ringA[bd + 1];
      const real Bw = ringB[bc - 1], Be = ringB[bc + 1], Bn = ringB[bu], Bnw = ringB[bu - 1], Bne = ringB[bu + 1],
                 Bs = ringB[bd], Bsw = ringB[bd - 1], Bse = ringB[bd + 1];
      const real c9 = real(1) / 9, c36 = real(1) / 36;
      // sum_l w_l c_l rho^S(r + c_l), deviations plus the background part (Eq. aNI)
      const real sAx = c9 * (Ae - Aw) + c36 * ((Ane - Anw) + (Ase - Asw));
      const real sAz = c9 * (An - As) + c36 * ((Ane + Anw) - (Ase + Asw)) + rc.dbgA;
      const real sBx = c9 * (Be - Bw) + c36 * ((Bne - Bnw) + (Bse - Bsw));
      const real sBz = c9 * (Bn - Bs) + c36 * ((Bne + Bnw) - (Bse + Bsw)) + rc.dbgB;
      const real rhoA = rc.bgA + dA, rhoB = rc.bgB + dB, rho = rhoA + rhoB;
      const real inv = real(1) / rho;
      // non-ideal force densities rho^S a^S_NI and their sum
      const real FnAx = -G * rhoA * sBx, FnAz = -G * rhoA * sBz;
      const real FnBx = -G * rhoB * sAx, FnBz = -G * rhoB * sAz;
      const real FNx = FnAx + FnBx, FNz = FnAz + FnBz;
      real FAx, FAz, FBx, FBz;
      if (flags & DF_ASTAR) {
        // a* makes the non-ideal acceleration common: rho^S a^S = (rho^S / rho) F_NI
        const real cA = rhoA * inv, cB = rhoB * inv;
        FAx = cA * FNx; FAz = cA * FNz;
        FBx = cB * FNx; FBz = cB * FNz;
      } else {
        FAx = FnAx; FAz = FnAz;
        FBx = FnBx; FBz = FnBz;
      }
      // gradient forcing: rho^A a^A_NE = (0, rho grad_c0 / 3) = -rho^B a^B_NE (Eq. NEcond)
      const real ne = rho * L.g3;
      FAz += ne;
      FBz -= ne;
      // barycentric velocity, Eq. (bar)
      const real jAx = (cur[1] - cur[3]) + (cur[5] - cur[6]) + (cur[8] - cur[7]);
      const real jAz = (cur[2] - cur[4]) + (cur[5] + cur[6]) - (cur[7] + cur[8]);
      const real jBx = (cur[10] - cur[12]) + (cur[14] - cur[15]) + (cur[17] - cur[16]);
      const real jBz = (cur[11] - cur[13]) + (cur[14] + cur[15]) - (cur[16] + cur[17]);
      const real Ux = (jAx + jBx + real(0.5) * FNx) * inv;
      const real Uz = (jAz + jBz + real(0.5) * FNz) * inv;

      if (SAMPLE) {
        real* fl = a.fields + 4 * (L.site_off) + z * Lx + x;
        fl[0] = dA + dB - L.rho_bar_off;
        fl[LzLx] = (dA - rc.c0 * (dA + dB)) * inv;
        fl[2 * LzLx] = Ux;
        fl[3 * LzLx] = Uz;
        // pressure (half trace; kinetic + interaction), minus its background part
        const real m3A = -2 * cur[0] + (cur[1] + cur[2] + cur[3] + cur[4]) +
                         4 * (cur[5] + cur[6] + cur[7] + cur[8]);
        const real m3B = -2 * cur[9] + (cur[10] + cur[11] + cur[12] + cur[13]) +
                         4 * (cur[14] + cur[15] + cur[16] + cur[17]);
        const real kin = (m3A + m3B + 2 * (dA + dB)) * (real(1) / 6);
        const real NA = c9 * (Ae + Aw + An + As) + real(2) / 36 * (Ane + Anw + Ase + Asw);
        const real NB = c9 * (Be + Bw + Bn + Bs) + real(2) / 36 * (Bne + Bnw + Bse + Bsw);
        const real inter = dA * (rc.nbB + NB) + rc.bgA * NB + dB * (rc.nbA + NA) + rc.bgB * NA;
        acc_p += (double)(kin + real(0.25) * G * inter);
        acc_a += (double)dA;
        acc_b += (double)dB;
      }

      real xiA[9], xiB[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) { xiA[k] = 0; xiB[k] = 0; }
      if (NOISE) {
        const uint32_t site = (uint32_t)(z * Lx + x);
        real n[14];
        const U4 r0 = philox(U4{site, step, L.lattice_id, 0u}, L.key0, L.key1);
        box_muller<real>(r0.x, r0.y, n[0], n[1]);
        box_muller<real>(r0.z, r0.w, n[2], n[3]);
        const U4 r1 = philox(U4{site, step, L.lattice_id, 1u}, L.key0, L.key1);
        box_muller<real>(r1.x, r1.y, n[4], n[5]);
        box_muller<real>(r1.z, r1.w, n[6], n[7]);
        const U4 r2 = philox(U4{site, step, L.lattice_id, 2u}, L.key0, L.key1);
        box_muller<real>(r2.x, r2.y, n[8], n[9]);
        box_muller<real>(r2.z, r2.w, n[10], n[11]);
        const U4 r3 = philox(U4{site, step, L.lattice_id, 3u}, L.key0, L.key1);
        box_muller<real>(r3.x, r3.y, n[12], n[13]);
        real smom, sA[9], sB[9];
        if (flags & DF_NOISE_LOC) {
          smom = L.pref_mom * rsqrt_pos<real>(rhoA * rhoB * inv);
          const real qA = rsqrt_pos<real>(rhoA), qB = rsqrt_pos<real>(rhoB);
#pragma unroll
          for (int k = 3; k < 9; ++k) { sA[k] = L.pref[k] * qA; sB[k] = L.pref[k] * qB; }
        } else {
          smom = L.sig_mom;
#pragma unroll
          for (int k = 3; k < 9; ++k) { sA[k] = L.sig[0][k]; sB[k] = L.sig[1][k]; }
        }
        xiA[1] = smom * n[0];
        xiA[2] = smom * n[1];
        xiB[1] = -xiA[1];
        xiB[2] = -xiA[2];
#pragma unroll
        for (int k = 3; k < 9; ++k) {
          xiA[k] = sA[k] * n[k - 1];
          xiB[k] = sB[k] * n[k + 5];
        }
      }
      collide_species<real>(cur, dA, rhoA, Ux, Uz, FAx, FAz, L.lam, L.omh, xiA);
      collide_species<real>(cur + 9, dB, rhoB, Ux, Uz, FBx, FBz, L.lam, L.omh, xiB);
      const int r0 = z * Lx + x;
#pragma unroll
      for (int k = 0; k < 18; ++k) g[k * LzLx + r0] = cur[k];
    }
#pragma unroll
    for (int k = 0; k < 18; ++k) cur[k] = nxt[k];
    dA = nA;
    dB = nB;
  }

  if (SAMPLE) {
    acc_p = warp_sum<real>(acc_p);
    acc_a = warp_sum<real>(acc_a);
    acc_b = warp_sum<real>(acc_b);
    const int wid = tid >> 5, lane = tid & 31, nw = (TX + 31) >> 5;
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
      a.partials[3 * item_index + 0] = p;
      a.partials[3 * item_index + 1] = ma;
      a.partials[3 * item_index + 2] = mb;
    }
  }
}

template <class real>
__host__ __device__ constexpr size_t ring_bytes(int tile_x) {
  return (size_t)2 * 4 * (tile_x + 2) * sizeof(real) + 8 * 3 * sizeof(double) + 64;
}

template <class real, bool SAMPLE, bool NOISE>
__global__ void __launch_bounds__(256) step_kernel(StepArgs<real> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);
  real* ringA = reinterpret_cast<real*>(smem + 8 * 3 * sizeof(double));
  real* ringB = ringA + 4 * (blockDim.x + 2);
  const uint32_t step = (uint32_t)(*a.d_t + a.t_offset);
  process_item<real, SAMPLE, NOISE>(a, a.src, a.dst, blockIdx.x, step, ringA, ringB, red);
}

// ---- bounded grid barrier for the persistent launch --------------------------------
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0]: arrivals, bar[1]: generation.  Returns false if the wait gave up after limit_ms
// (err is then set) or another block reported an error.
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks, int limit_ms) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    int ok = 1;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns(), lim = (uint64_t)limit_ms * 1000000ull;
      while (*vgen == gen) {
        if (global_ns() - t0 > lim) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
      __threadfence();
    }
    ok_s = ok && (*(volatile int*)err == 0);
  }
  __syncthreads();
  return ok_s != 0;
}

template <class real, bool NOISE>
__global__ void __launch_bounds__(256) persistent_kernel(StepArgs<real> a, int nsteps, int sample_last,
                                                         unsigned* bar, int* err, int limit_ms) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);
  real* ringA = reinterpret_cast<real*>(smem + 8 * 3 * sizeof(double));
  real* ringB = ringA + 4 * (blockDim.x + 2);
  const int64_t t0 = *a.d_t + a.t_offset;
  for (int k = 0; k < nsteps; ++k) {
    const real* src = (k & 1) ? a.dst : a.src;
    real* dst = (k & 1) ? const_cast<real*>(a.src) : a.dst;
    const uint32_t step = (uint32_t)(t0 + k);
    const bool sample = sample_last && k == nsteps - 1;
    for (int i = blockIdx.x; i < a.n_items; i += gridDim.x) {
      if (sample) process_item<real, true, NOISE>(a, src, dst, i, step, ringA, ringB, red);
      else process_item<real, false, NOISE>(a, src, dst, i, step, ringA, ringB, red);
    }
    if (k + 1 < nsteps) {
      if (!grid_barrier(bar, err, gridDim.x, limit_ms)) return;
    }
  }
}

__global__ void advance_kernel(int64_t* d_t, int64_t k) { *d_t += k; }

__global__ void barrier_probe_kernel(unsigned* bar, int* err, unsigned expected, int limit_ms) {
  grid_barrier(bar, err, expected, limit_ms);
}

template <class real>
cudaError_t launch_step(const StepArgs<real>& a, int tile_x, bool sample, bool noise, cudaStream_t s) {
  const size_t smem = ring_bytes<real>(tile_x);
  if (a.n_items <= 0) return cudaSuccess;
  if (sample) {
    if (noise) step_kernel<real, true, true><<<a.n_items, tile_x, smem, s>>>(a);
    else step_kernel<real, true, false><<<a.n_items, tile_x, smem, s>>>(a);
  } else {
    if (noise) step_kernel<real, false, true><<<a.n_items, tile_x, smem, s>>>(a);
    else step_kernel<real, false, false><<<a.n_items, tile_x, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <class real>
int persistent_grid(int tile_x, bool sample, bool noise) {
  (void)sample;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ring_bytes<real>(tile_x);
  cudaError_t e = noise ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persistent_kernel<real, true>, tile_x, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persistent_kernel<real, false>, tile_x, smem);
  if (e != cudaSuccess) return 0;
  return per * sms;
}

template <class real>
cudaError_t launch_step_persistent(const StepArgs<real>& a, int tile_x, int nsteps, bool sample_last, bool noise,
                                   unsigned* barrier, int* err, int grid, int limit_ms, cudaStream_t s) {
  const size_t smem = ring_bytes<real>(tile_x);
  StepArgs<real> aa = a;
  int ns = nsteps, sl = sample_last ? 1 : 0;
  void* args[] = {&aa, &ns, &sl, &barrier, &err, &limit_ms};
  const void* fn = noise ? (const void*)persistent_kernel<real, true> : (const void*)persistent_kernel<real, false>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(tile_x), args, smem, s);
}

cudaError_t launch_advance(int64_t* d_t, int64_t k, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(d_t, k);
  return cudaGetLastError();
}

cudaError_t launch_barrier_probe(int blocks, int expected, int limit_ms, unsigned* barrier, int* err,
                                 cudaStream_t s) {
  unsigned ex = (unsigned)expected;
  void* args[] = {&barrier, &err, &ex, &limit_ms};
  return cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(blocks), dim3(32), args, 0, s);
}

template cudaError_t launch_step<float>(const StepArgs<float>&, int, bool, bool, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs<double>&, int, bool, bool, cudaStream_t);
template int persistent_grid<float>(int, bool, bool);
template int persistent_grid<double>(int, bool, bool);
template cudaError_t launch_step_persistent<float>(const StepArgs<float>&, int, int, bool, bool, unsigned*, int*, int,
                                                   int, cudaStream_t);
template cudaError_t launch_step_persistent<double>(const StepArgs<double>&, int, int, bool, bool, unsigned*, int*,
                                                    int, int, cudaStream_t);

}  // namespace lbk
