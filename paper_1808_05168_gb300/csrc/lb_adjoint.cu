// lb_adjoint.cu -- reverse-mode (adjoint) sweep of the fluctuating LB step for the gradient of
// the time-averaged mean-pressure shift
//     L = (1/T) sum_{t<T} Pbar(t) |_{kT}  -  (1/T) sum_{t<T} Pbar(t) |_{kT = 0}
// with respect to (G, lambda_s, lambda_d), on a fixed noise stream, both runs from the rest
// state.  Pbar(t) is the spatial mean of the mechanical pressure (Sec. III.C) of the
// pre-collision state of step t.
//
// One step k maps the stored state f*_{k-1} to f*_k (Eq. LB with Eq. MRT).  Its adjoint maps
// fbar*_k (the loss's sensitivity to f*_k) to fbar*_{k-1} and adds the step's share of the
// parameter gradient, in three passes:
//   1. densities: rho^S of the pre-collision state at every site (needed by the neighbours),
//      computed by the previous adjoint step's gather/push, or on their own at the top of a
//      checkpoint segment;
//   2. local: at every site, the forward quantities are recomputed and the transposed Jacobian
//      of the site update is applied to fbar*_k(r) (plus the pressure term of the loss); this
//      gives the sensitivity to the 18 pulled populations through the site's own moments and
//      densities, the sensitivity to the two neighbour sums sum_l w_l c_l rho^S(r + c_l) of
//      Eq. (aNI), and the parameter contributions;
//   3. gather/push: each site collects what its neighbours' forces and pressures owe to its
//      densities (wall ghosts copy the adjacent row, Sec. II.A), adds it to every pulled
//      population of the species, and pushes the result back along the streaming map (the
//      transpose of the pull with mid-way bounce-back is a one-to-one scatter).
// The forward states are recomputed segment by segment from checkpoints (every C steps) into a
// ring of C states, so memory is O(T/C + C) states.
//
// Supported: every lattice of a batch at once, each with its own loss and gradient; the a*
// correction on or off, wall ghosts copying the adjacent row or taking the fixed wall
// composition, hom or loc noise; both precisions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "lb_adjoint.cuh"

namespace lbk {

namespace {

// v_l = sum_a T_al m_a (the transpose of the moment transform), Table I.
template <class real>
__device__ __forceinline__ void transpose_moments(const real m[9], real v[9]) {
  const real b4 = m[0] + m[3] - 4 * m[8], b5 = m[0] + 4 * m[3] + 8 * m[8];
  v[0] = m[0] - 2 * m[3] + 2 * m[8];
  v[1] = b4 + m[1] + m[4] - m[6];
  v[2] = b4 + m[2] - m[4] - m[7];
  v[3] = b4 - m[1] + m[4] + m[6];
  v[4] = b4 - m[2] - m[4] + m[7];
  v[5] = b5 + m[1] + m[2] + m[5] + 2 * m[6] + 2 * m[7];
  v[6] = b5 - m[1] + m[2] - m[5] - 2 * m[6] + 2 * m[7];
  v[7] = b5 - m[1] - m[2] + m[5] - 2 * m[6] - 2 * m[7];
  v[8] = b5 + m[1] - m[2] - m[5] + 2 * m[6] - 2 * m[7];
}

// m_a = sum_l T_al v_l, Table I (all nine moments).
template <class real>
__device__ __forceinline__ void all_moments(const real v[9], real m[9]) {
  const real a57 = v[5] - v[7], a68 = v[6] - v[8], d13 = v[1] - v[3], d24 = v[2] - v[4];
  const real s13 = v[1] + v[3], s24 = v[2] + v[4], s57 = v[5] + v[7], s68 = v[6] + v[8];
  const real e = s13 + s24, dg = s57 + s68;
  m[0] = v[0] + e + dg;
  m[1] = d13 + a57 - a68;
  m[2] = d24 + a57 + a68;
  m[3] = -2 * v[0] + e + 4 * dg;
  m[4] = s13 - s24;
  m[5] = s57 - s68;
  m[6] = -d13 + 2 * (a57 - a68);
  m[7] = -d24 + 2 * (a57 + a68);
  m[8] = 2 * v[0] - 4 * e + 8 * dg;
}

// The lattice velocities enter through LB_CX / LB_CZ / LB_OPP in fully unrolled loops: as
// compile-time constants, the products with c = 0 and c = +-1 cost no FP64 instruction.

// Deviations of the 9 populations of species s pulled at (x, z) (Eq. LB; reflected at the walls;
// the background streaming shift on non-reflected links), as in the forward kernel.
template <class real>
__device__ __forceinline__ void pull9(const real* __restrict__ f, int Lx, int Lz, int x, int z, double k9, double k36,
                                      int s, double v[9]) {
  const int LzLx = Lx * Lz;
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int zs = z - LB_CZ(l);
    const int xs = LB_CX(l) == 0 ? x : (x - LB_CX(l) + Lx) % Lx;
    double val;
    if (zs >= 0 && zs < Lz) {
      val = (double)f[state_index(s, l, zs, xs, Lx, LzLx)];
      if (LB_CZ(l) != 0) {  // the background shift -c_lz w_l rho_bar d_z c_0 (k9, k36: species A)
        const double q = l <= 4 ? k9 : k36;
        const double sh = LB_CZ(l) > 0 ? -q : q;
        val += s == 0 ? sh : -sh;
      }
    } else {
      val = (double)f[state_index(s, LB_OPP(l), z, x, Lx, LzLx)];
    }
    v[l] = val;
  }
}

// Both species: v[9 s + l].
template <class real>
__device__ __forceinline__ void pull18(const real* __restrict__ f, int Lx, int Lz, int x, int z, double k9, double k36,
                                       double v[18]) {
  pull9(f, Lx, Lz, x, z, k9, k36, 0, v);
  pull9(f, Lx, Lz, x, z, k9, k36, 1, v + 9);
}

// Absolute pre-collision densities of site i = z Lx + x of state f, into rho[i] and rho[N + i].
template <class real>
__device__ __forceinline__ void site_densities(const real* __restrict__ f, const LatticeDev<real>& L,
                                               const RowConst<real>* rows, int i, int x, int z, double* rho) {
  const int N = L.Lx * L.Lz;
  double v[18];
  pull18(f, L.Lx, L.Lz, x, z, (double)L.k9, (double)L.k36, v);
  double a = 0, b = 0;
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    a += v[l];
    b += v[9 + l];
  }
  rho[i] = (double)rows[z].bgA + a;
  rho[N + i] = (double)rows[z].bgB + b;
}

// The lattice of this block (AdjMap) and the block's first site within it.
__device__ __forceinline__ int adj_lattice(const AdjMap& map) { return map.lat_of[blockIdx.x]; }
__device__ __forceinline__ int adj_site(const AdjMap& map, int li) {
  return (blockIdx.x - map.first[li]) * blockDim.x + threadIdx.x;
}

// Absolute pre-collision densities of every site of every lattice.
template <class real>
__global__ void adj_rho_kernel(const real* __restrict__ f, const LatticeDev<real>* lat, const RowConst<real>* rows,
                               const AdjMap map, double* __restrict__ rho) {
  const int li = adj_lattice(map);
  const LatticeDev<real> L = lat[li];
  const int N = L.Lx * L.Lz;
  const int i = adj_site(map, li);
  if (i >= N) return;
  site_densities(f + L.f_off, L, rows + L.row_off, i, i % L.Lx, i / L.Lx, rho + 2 * L.site_off);
}

// Density of species s at (x, z), beyond a wall the ghost of Sec. II.A: a copy of the adjacent
// row, or (fixed) that row's total density split by the wall composition cw of that row.
template <class real>
__device__ __forceinline__ double rho_at(const double* rho, const RowConst<real>* rows, bool fixed, int Lx, int Lz,
                                         int s, int x, int z) {
  x = (x + Lx) % Lx;
  if (z >= 0 && z < Lz) return rho[s * Lx * Lz + z * Lx + x];
  const int za = z < 0 ? 0 : Lz - 1;
  if (!fixed) return rho[s * Lx * Lz + za * Lx + x];
  const double cw = (double)rows[za].ghost_cA, t = rho[za * Lx + x] + rho[Lx * Lz + za * Lx + x];
  return s == 0 ? cw * t : (1 - cw) * t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The fourteen normals of a site.  FP32: exactly those of the forward FP32 kernel.  FP64: the
// library Box-Muller; the forward FP64 kernel's table-driven normals agree with it to a few units
// in the last place, far below what the gradient resolves.
template <class real>
__device__ __forceinline__ void normals14(uint32_t site, uint32_t step, const LatticeDev<real>& L, real n[14]);
template <>
__device__ __forceinline__ void normals14<double>(uint32_t site, uint32_t step, const LatticeDev<double>& L,
                                                  double n[14]) {
  U4 w[4];
  philox_site(site, step, L.lattice_id, L.key0, L.key1, w);
  box_muller<double>(w[0].x, w[0].y, n[0], n[1]);
  box_muller<double>(w[0].z, w[0].w, n[2], n[3]);
  box_muller<double>(w[1].x, w[1].y, n[4], n[5]);
  box_muller<double>(w[1].z, w[1].w, n[6], n[7]);
  box_muller<double>(w[2].x, w[2].y, n[8], n[9]);
  box_muller<double>(w[2].z, w[2].w, n[10], n[11]);
  box_muller<double>(w[3].x, w[3].y, n[12], n[13]);
}
template <>
__device__ __forceinline__ void normals14<float>(uint32_t site, uint32_t step, const LatticeDev<float>& L, float n[14]) {
  U4 w[4];
  philox_site(site, step, L.lattice_id, L.key0, L.key1, w);
  const uint32_t k[16] = {w[0].x, w[0].y, w[0].z, w[0].w, w[1].x, w[1].y, w[1].z, w[1].w,
                          w[2].x, w[2].y, w[2].z, w[2].w, w[3].x, w[3].y, w[3].z, w[3].w};
#pragma unroll
  for (int p = 0; p < 7; ++p) normal_pair<float>(k[2 * p], k[2 * p + 1], n[2 * p], n[2 * p + 1], nullptr);
}

// The local part of the transposed step at every site of every lattice (see the file comment).
// alpha = sign w_loss: weight of the site's pressure in the loss.  Outputs, per lattice at its
// site offset: fl[18][N] (local sensitivity of the pulled
// populations), sb[4][N] (sensitivity of sum_l w_l c_l rho^A, rho^B (r + c_l): x, z for A then
// B), and per block the three parameter partials (G, lambda_s, lambda_d), added to the block's own
// slot of `partials` (zeroed before the sweep; one fixed summation order, step after step).
// The state may be single precision (FP32 deviations); the transposed step is evaluated in double
// precision throughout, since the loss is a small difference of two runs' pressures.
template <class real, bool NOISE, bool OPTS>
__global__ void adj_local_kernel(const real* __restrict__ f, const double* __restrict__ fbar,
                                 const LatticeDev<real>* lat, const RowConst<real>* rows,
                                 const AdjConst* __restrict__ kcs, const AdjMap map, const double* __restrict__ rho,
                                 uint32_t step, double sign, double* __restrict__ fl, double* __restrict__ sb,
                                 double* __restrict__ partials) {
  using real_s = real;
  const int li = adj_lattice(map);
  const LatticeDev<real_s> L = lat[li];
  const AdjConst& kc = kcs[li];
  const double alpha = sign * kc.w_loss;  // weight of this site's pressure in the loss
  const int Lx = L.Lx, Lz = L.Lz, N = Lx * Lz;
  const int i = adj_site(map, li);
  // this lattice's part of the batch's buffers
  f += L.f_off;
  rows += L.row_off;
  fbar += 18 * L.site_off;
  rho += 2 * L.site_off;
  fl += 18 * L.site_off;
  sb += 4 * L.site_off;
  double gG = 0, gS = 0, gD = 0;
  // the default options (a* on, copy-rule ghosts, hom noise) are compiled without the branches
  const bool astar = !OPTS || (L.flags & DF_ASTAR), fixed = OPTS && (L.flags & DF_WALL_FIXED),
             loc = OPTS && NOISE && (L.flags & DF_NOISE_LOC);
  if (i < N) {
    const int x = i % Lx, z = i / Lx;
    double v[18];
    pull18(f, Lx, Lz, x, z, (double)L.k9, (double)L.k36, v);
    double mA[9], mB[9];
    all_moments(v, mA);
    all_moments(v + 9, mB);
    const double rA = rho[i], rB = rho[N + i];
    const double rho_t = rA + rB, inv = double(1) / rho_t;
    // neighbour sums (Eq. aNI) and the pressure's neighbour sums, copy-rule ghosts
    double sAx = 0, sAz = 0, sBx = 0, sBz = 0, NA = 0, NB = 0;
#pragma unroll
    for (int l = 1; l < 9; ++l) {
      constexpr double w9 = double(1) / 9, w36 = double(1) / 36;
      const double w = l <= 4 ? w9 : w36, wc2 = l <= 4 ? w9 : 2 * w36;  // w_l, w_l |c_l|^2
      const double a = rho_at(rho, rows, fixed, Lx, Lz, 0, x + LB_CX(l), z + LB_CZ(l));
      const double b = rho_at(rho, rows, fixed, Lx, Lz, 1, x + LB_CX(l), z + LB_CZ(l));
      if (LB_CX(l) != 0) {
        sAx += (LB_CX(l) * w) * a;
        sBx += (LB_CX(l) * w) * b;
      }
      if (LB_CZ(l) != 0) {
        sAz += (LB_CZ(l) * w) * a;
        sBz += (LB_CZ(l) * w) * b;
      }
      NA += wc2 * a;
      NB += wc2 * b;
    }
    const double G = L.G;
    const double FNx = -G * (rA * sBx + rB * sAx), FNz = -G * (rA * sBz + rB * sAz);
    const double cA = rA * inv, cB = rB * inv;
    const double ne = rho_t * L.g3;
    // the species' forces: with a*, F^S = (rho^S / rho) F_N; without, F^A = -G rho^A s^B and
    // F^B = -G rho^B s^A; plus the gradient forcing +- (0, rho g3)
    const double FA[2] = {astar ? cA * FNx : -G * rA * sBx, (astar ? cA * FNz : -G * rA * sBz) + ne};
    const double FB[2] = {astar ? cB * FNx : -G * rB * sAx, (astar ? cB * FNz : -G * rB * sAz) - ne};
    const double Px = mA[1] + mB[1] + double(0.5) * FNx, Pz = mA[2] + mB[2] + double(0.5) * FNz;
    const double Ux = Px * inv, Uz = Pz * inv;
    const double ld = L.lam[1], le = L.lam[3], ls = L.lam[4], lq = L.lam[6], leps = L.lam[8];
    const double lam[9] = {double(1), ld, ld, le, ls, ls, lq, lq, leps};

    double n[14];
    if (NOISE) {
      real_s nn[14];
      normals14<real_s>((uint32_t)i, step, L, nn);
#pragma unroll
      for (int q = 0; q < 14; ++q) n[q] = (double)nn[q];
    }

    // adjoints accumulated over both species
    double Ubx = 0, Ubz = 0, FNbx = 0, FNbz = 0, rhob_t = 0, invb = 0;
    double rhob[2] = {0, 0};
    double mb[2][9];
    double lamb_d = 0, lamb_s = 0;
    double sbarA[9], sbarB[9];
    double Fb[2][2];  // sensitivities of the species' forces (without a*)
    for (int s = 0; s < 2; ++s) {
      const double* m = s == 0 ? mA : mB;
      const double rs = s == 0 ? rA : rB;
      const double* F = s == 0 ? FA : FB;
      double g[9];
#pragma unroll
      for (int l = 0; l < 9; ++l) {
        const double w = l == 0 ? double(4) / 9 : (l <= 4 ? double(1) / 9 : double(1) / 36);
        g[l] = w * fbar[(s * 9 + l) * N + i];
      }
      double sbar[9];
      all_moments(g, sbar);  // sbar_a = (1/N_a) sum_l T_al w_l fbar_l, before the 1/N_a
      const double invN[9] = {1, 3, 3, double(0.25), double(2.25), 9, double(1.5), double(1.5), double(0.0625)};
#pragma unroll
      for (int a = 0; a < 9; ++a) sbar[a] *= invN[a];
      for (int a = 0; a < 9; ++a) (s == 0 ? sbarA : sbarB)[a] = sbar[a];
      // s_0 = rho^S
      rhob[s] += sbar[0];
      // equilibrium moments and forcing sources
      const double UxUx = Ux * Ux, UzUz = Uz * Uz;
      const double meq[6] = {0, rs * Ux, rs * Uz, 3 * rs * (UxUx + UzUz), rs * (UxUx - UzUz), rs * Ux * Uz};
      const double src[6] = {0, F[0], F[1], 6 * (Ux * F[0] + Uz * F[1]), 2 * (Ux * F[0] - Uz * F[1]),
                           Ux * F[1] + Uz * F[0]};
      double mbar[9];
      mbar[0] = 0;
      double meqb[6], srcb[6];
      for (int a = 1; a < 9; ++a) mbar[a] = kc.oml[a] * sbar[a];
      for (int a = 1; a < 6; ++a) {
        meqb[a] = lam[a] * sbar[a];
        srcb[a] = kc.ohl[a] * sbar[a];
        const double dl = sbar[a] * (meq[a] - m[a] - double(0.5) * src[a]);
        if (a <= 2) lamb_d += dl;
        else if (a >= 4) lamb_s += dl;
      }
      // meq -> rho^S, U
      rhob[s] += meqb[1] * Ux + meqb[2] * Uz + 3 * meqb[3] * (UxUx + UzUz) + meqb[4] * (UxUx - UzUz) +
                 meqb[5] * Ux * Uz;
      Ubx += meqb[1] * rs + 6 * meqb[3] * rs * Ux + 2 * meqb[4] * rs * Ux + meqb[5] * rs * Uz;
      Ubz += meqb[2] * rs + 6 * meqb[3] * rs * Uz - 2 * meqb[4] * rs * Uz + meqb[5] * rs * Ux;
      // sources -> F^S, U
      const double Fbx = srcb[1] + 6 * srcb[3] * Ux + 2 * srcb[4] * Ux + srcb[5] * Uz;
      const double Fbz = srcb[2] + 6 * srcb[3] * Uz - 2 * srcb[4] * Uz + srcb[5] * Ux;
      Ubx += 6 * srcb[3] * F[0] + 2 * srcb[4] * F[0] + srcb[5] * F[1];
      Ubz += 6 * srcb[3] * F[1] - 2 * srcb[4] * F[1] + srcb[5] * F[0];
      if (astar) {  // F^S = (rho^S / rho) F_N +- (0, rho g3)
        const double cS = s == 0 ? cA : cB;
        FNbx += cS * Fbx;
        FNbz += cS * Fbz;
        const double cSb = Fbx * FNx + Fbz * FNz;
        rhob[s] += cSb * inv;
        invb += cSb * rs;
      } else {
        Fb[s][0] = Fbx;
        Fb[s][1] = Fbz;
      }
      rhob_t += (s == 0 ? 1 : -1) * L.g3 * Fbz;
      for (int a = 0; a < 9; ++a) mb[s][a] = mbar[a];
    }
    // U = (j^A + j^B + F_N / 2) / rho
    const double Pbx = Ubx * inv, Pbz = Ubz * inv;
    invb += Ubx * Px + Ubz * Pz;
    mb[0][1] += Pbx;
    mb[0][2] += Pbz;
    mb[1][1] += Pbx;
    mb[1][2] += Pbz;
    FNbx += double(0.5) * Pbx;
    FNbz += double(0.5) * Pbz;
    // F_N = -G (rho^A s^B + rho^B s^A)
    gG += (double)(-(FNbx * (rA * sBx + rB * sAx) + FNbz * (rA * sBz + rB * sAz)));
    rhob[0] += -G * (FNbx * sBx + FNbz * sBz);
    rhob[1] += -G * (FNbx * sAx + FNbz * sAz);
    double eAx = 0, eAz = 0, eBx = 0, eBz = 0;  // the species' own forces (without a*)
    if (!astar) {
      gG += -(Fb[0][0] * rA * sBx + Fb[0][1] * rA * sBz + Fb[1][0] * rB * sAx + Fb[1][1] * rB * sAz);
      rhob[0] += -G * (Fb[0][0] * sBx + Fb[0][1] * sBz);
      rhob[1] += -G * (Fb[1][0] * sAx + Fb[1][1] * sAz);
      eAx = -G * rB * Fb[1][0];
      eAz = -G * rB * Fb[1][1];
      eBx = -G * rA * Fb[0][0];
      eBz = -G * rA * Fb[0][1];
    }
    sb[0 * N + i] = -G * rB * FNbx + eAx;  // sensitivity of s^A (x, z)
    sb[1 * N + i] = -G * rB * FNbz + eAz;
    sb[2 * N + i] = -G * rA * FNbx + eBx;  // sensitivity of s^B (x, z)
    sb[3 * N + i] = -G * rA * FNbz + eBz;
    // the loss's pressure at this site: (1/2) sum |c|^2 f + (G/4) [rho^A N^B + rho^B N^A]
    rhob[0] += alpha * double(0.25) * G * NB;
    rhob[1] += alpha * double(0.25) * G * NA;
    gG += (double)(alpha * double(0.25) * (rA * NB + rB * NA));
    // inv = 1 / rho, rho = rho^A + rho^B
    rhob_t += -invb * inv * inv;
    rhob[0] += rhob_t;
    rhob[1] += rhob_t;
    // noise amplitudes depend on lambda_d (moments 1, 2) and lambda_s (moments 4, 5); loc noise
    // also on the site's densities: sigma_mom = p_mom sqrt(rho^A rho^B / rho), sigma^S_a = p_a
    // sqrt(rho^S)
    if (NOISE) {
      const double q1 = n[0] * (sbarA[1] - sbarB[1]) + n[1] * (sbarA[2] - sbarB[2]);
      if (loc) {
        const double sm = sqrt(rA * rB * inv), qA = sqrt(rA), qB = sqrt(rB);
        lamb_d += kc.dpm * sm * q1;
        lamb_s += kc.dp4 * (qA * sbarA[4] * n[3] + qB * sbarB[4] * n[9]) +
                  kc.dp5 * (qA * sbarA[5] * n[4] + qB * sbarB[5] * n[10]);
        // d sm / d rho^A = (rho^B / rho)^2 / (2 sm), d sm / d rho^B = (rho^A / rho)^2 / (2 sm)
        const double hm = kc.pm * q1 * inv * inv / (2 * sm);
        double tA = 0, tB = 0;
#pragma unroll
        for (int a = 3; a < 9; ++a) {
          tA += kc.pa[a] * sbarA[a] * n[a - 1];
          tB += kc.pa[a] * sbarB[a] * n[a + 5];
        }
        rhob[0] += hm * rB * rB + tA / (2 * qA);
        rhob[1] += hm * rA * rA + tB / (2 * qB);
      } else {
        lamb_d += kc.dsm * q1;
        lamb_s += kc.d4 * (sbarA[4] * n[3] + sbarB[4] * n[9]) + kc.d5 * (sbarA[5] * n[4] + sbarB[5] * n[10]);
      }
    }
    gS += (double)lamb_s;
    gD += (double)lamb_d;
    // back to the pulled populations: moments (transposed), density (every link), kinetic pressure
    for (int s = 0; s < 2; ++s) {
      double o[9];
      mb[s][0] = rhob[s];
      transpose_moments(mb[s], o);
      const double k1 = alpha * double(0.5), k2 = alpha;  // alpha |c_l|^2 / 2 on the axis, diagonal links
#pragma unroll
      for (int l = 0; l < 9; ++l) fl[(s * 9 + l) * N + i] = l == 0 ? o[l] : o[l] + (l <= 4 ? k1 : k2);
    }
  }
  // block partials of the parameter gradient
  __shared__ double red[3][32];
  gG = warp_sum(gG);
  gS = warp_sum(gS);
  gD = warp_sum(gD);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = gG;
    red[1][wid] = gS;
    red[2][wid] = gD;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
    }
    partials[3 * blockIdx.x + 0] += a;
    partials[3 * blockIdx.x + 1] += b;
    partials[3 * blockIdx.x + 2] += c;
  }
}

// Gather the neighbour-owed density sensitivities and push along the transposed streaming map.
// With f_next (the state before f_prev) given, also the densities of f_next into rho_next, for the
// next adjoint step (one launch instead of two).  Two threads per site, one per species (blocks of
// 2 kAdjBlock threads over the lattice's adjoint blocks): the species' work is independent but
// for the fixed-composition ghosts, which mix both.
template <class real>
__global__ void adj_gather_push_kernel(const LatticeDev<real>* lat, const RowConst<real>* rows,
                                       const AdjConst* __restrict__ kcs, const AdjMap map,
                                       const double* __restrict__ rho, const double* __restrict__ fl,
                                       const double* __restrict__ sb, double sign, double* __restrict__ fbar_prev,
                                       const real* __restrict__ f_next, double* __restrict__ rho_next) {
  const int li = adj_lattice(map);
  const LatticeDev<real> L = lat[li];
  const double alpha = sign * kcs[li].w_loss;
  const int Lx = L.Lx, Lz = L.Lz, N = Lx * Lz;
  const int t = adj_site(map, li), i = t >> 1, sp = t & 1;  // site, species
  if (i >= N) return;
  rows += L.row_off;
  rho += 2 * L.site_off;
  fl += 18 * L.site_off;
  sb += 4 * L.site_off;
  fbar_prev += 18 * L.site_off;
  if (f_next) f_next += L.f_off;
  rho_next += 2 * L.site_off;
  const int x = i % Lx, z = i / Lx;
  if (f_next) {  // this species' density of f_next at the site
    double v[9];
    pull9(f_next, Lx, Lz, x, z, (double)L.k9, (double)L.k36, sp, v);
    double a = 0;
#pragma unroll
    for (int l = 0; l < 9; ++l) a += v[l];
    rho_next[sp * N + i] = (double)(sp == 0 ? rows[z].bgA : rows[z].bgB) + a;
  }
  const double q = alpha * 0.25 * (double)L.G;
  const bool fixed = L.flags & DF_WALL_FIXED;
  double rb = 0;
#pragma unroll
  for (int l = 1; l < 9; ++l) {
    constexpr double w9 = 1.0 / 9, w36 = 1.0 / 36;
    const double w = l <= 4 ? w9 : w36, wc2 = l <= 4 ? w9 : 2 * w36;  // w_l, w_l |c_l|^2
    // what the site j = (x - c_lx, zs) owes the density of species s its link l reaches: through
    // its neighbour sums of s (sb[2 s], sb[2 s + 1]) and its pressure, which pairs s with the
    // other species' density there
    auto owed = [&](int zs, int s) {
      const int j = zs * Lx + (LB_CX(l) == 0 ? x : (x - LB_CX(l) + Lx) % Lx);
      const double* sx = sb + (2 * s) * N;
      const double* sz = sb + (2 * s + 1) * N;
      double ts = 0;
      if (LB_CX(l) != 0) ts = LB_CX(l) * sx[j];
      if (LB_CZ(l) != 0) ts = LB_CX(l) != 0 ? ts + LB_CZ(l) * sz[j] : LB_CZ(l) * sz[j];
      return w * ts + (wc2 * q) * rho[(1 - s) * N + j];
    };
    const int zs = z - LB_CZ(l);
    if (zs >= 0 && zs < Lz) rb += owed(zs, sp);
    // the wall ghost next to this row: a copy of this row's densities, or (fixed) this row's total
    // density split by the wall composition
    if ((z == 0 && LB_CZ(l) == -1) || (z == Lz - 1 && LB_CZ(l) == 1)) {
      if (fixed) {
        const double cw = (double)rows[z].ghost_cA;
        rb += cw * owed(z, 0) + (1 - cw) * owed(z, 1);
      } else {
        rb += owed(z, sp);
      }
    }
  }
  const int64_t LzLx = N;
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const double val = fl[(sp * 9 + l) * N + i] + rb;
    const int zs = z - LB_CZ(l);
    if (zs >= 0 && zs < Lz) {
      const int xs = LB_CX(l) == 0 ? x : (x - LB_CX(l) + Lx) % Lx;
      fbar_prev[(sp * 9 + l) * LzLx + zs * Lx + xs] = val;
    } else {
      fbar_prev[(sp * 9 + LB_OPP(l)) * LzLx + z * Lx + x] = val;
    }
  }
}

// grads[3 i + k] = sum over the blocks b of lattice i of partials[3 b + k]: one warp per lattice
// (block i), lanes strided over the blocks, then a fixed butterfly (deterministic).
__global__ void adj_sum_partials(const double* partials, const AdjMap map, double* grads) {
  const int li = blockIdx.x;
  const int b0 = map.first[li], n = map.first[li + 1] - b0;
  partials += 3 * (size_t)b0;
  double* grad = grads + 3 * li;
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < n; k += 32) {
    a += partials[3 * k];
    b += partials[3 * k + 1];
    c += partials[3 * k + 2];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (threadIdx.x == 0) {
    grad[0] = a;
    grad[1] = b;
    grad[2] = c;
  }
}

}  // namespace

template <class real>
cudaError_t launch_adjoint_step(const real* f_prev, const real* f_next, const double* fbar, double* fbar_prev,
                                const LatticeDev<real>* lat, const RowConst<real>* rows, const AdjConst* kcs,
                                bool options, const AdjMap& map, uint32_t step, bool noise, double sign,
                                bool rho_ready, double* rho, double* rho_next, double* fl, double* sb,
                                double* partials, cudaStream_t s) {
  const int nb = map.n_blocks;
  if (!rho_ready) adj_rho_kernel<real><<<nb, kAdjBlock, 0, s>>>(f_prev, lat, rows, map, rho);
  auto local = [&](auto noise_c, auto opts_c) {
    adj_local_kernel<real, decltype(noise_c)::value, decltype(opts_c)::value>
        <<<nb, kAdjBlock, 0, s>>>(f_prev, fbar, lat, rows, kcs, map, rho, step, sign, fl, sb, partials);
  };
  using T = std::true_type;
  using F = std::false_type;
  if (noise) options ? local(T(), T()) : local(T(), F());
  else options ? local(F(), T()) : local(F(), F());
  adj_gather_push_kernel<real>
      <<<nb, 2 * kAdjBlock, 0, s>>>(lat, rows, kcs, map, rho, fl, sb, sign, fbar_prev, f_next, rho_next);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gradient(const double* partials, const AdjMap& map, double* grads, cudaStream_t s) {
  adj_sum_partials<<<map.n_lat, 32, 0, s>>>(partials, map, grads);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint_step<float>(const float*, const float*, const double*, double*,
                                                const LatticeDev<float>*, const RowConst<float>*, const AdjConst*,
                                                bool, const AdjMap&, uint32_t, bool, double, bool, double*, double*,
                                                double*, double*, double*, cudaStream_t);
template cudaError_t launch_adjoint_step<double>(const double*, const double*, const double*, double*,
                                                 const LatticeDev<double>*, const RowConst<double>*, const AdjConst*,
                                                 bool, const AdjMap&, uint32_t, bool, double, bool, double*, double*,
                                                 double*, double*, double*, cudaStream_t);

}  // namespace lbk
