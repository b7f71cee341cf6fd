/*
 * lb_oracle.cpp -- the oracle: a plain, slow, double-precision CPU implementation of the
 * two-species fluctuating D2Q9 MRT lattice Boltzmann step of Belardinelli, Sbragaglia,
 * Benzi & Ciliberto, "Lattice Boltzmann simulations of non-equilibrium fluctuations in a
 * non-ideal binary mixture" (arXiv:1808.05168), with its diagnostics.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header, table or constant
 * generator with the CUDA library; both sides implement the Philox4x32-10 generator from
 * its published definition (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random numbers:
 * as easy as 1, 2, 3").
 *
 * Everything is written for clarity, not speed: dense 9x9 moment transforms, whole-lattice
 * arrays for every intermediate, a separable O(n^2) discrete Fourier transform.  The loops over
 * the rows of the lattice carry OpenMP pragmas: the same source compiled with -fopenmp runs them
 * on several host cores.  Every site is then still computed by the same operations in the same
 * order, and every sum across sites (mean pressure, mass, loss, profiles, correlations) stays in
 * one thread, so both builds give identical results.
 *
 * Readings where the paper is silent:
 *  - forcing moments: the second-order (Guo-type) source; its moments S_a are taken
 *    with the factor (1 - lambda_a/2), so F_{1,2} = (1 - lambda_d/2) rho^S a^S (Sec. II,
 *    "First order moments");
 *  - the a* correction of the footnote to Eq. (ne-acc) is on unless disabled;
 *  - hom noise uses rho^A_ref = rho_bar c_bar0, rho^B_ref = rho_bar (1 - c_bar0);
 *  - the noise stream: Philox4x32-10, key = (seed_lo, seed_hi), counter = (site, step,
 *    lattice_id, call), u = (2 (k mod 2^23) + 1) 2^-24, Box-Muller pairs;
 *  - walls: mid-way bounce-back; the wall-ghost densities for the non-ideal force copy
 *    the adjacent fluid row (Sec. II.A), or take a fixed wall composition if asked;
 *  - diagnostics are taken on the pre-collision state after streaming.
 * No routine here is parity-unpinned except where a function's comment says so.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ------------------------------------------------------------------------------------
// Forward-mode dual numbers, used to differentiate the whole run with respect to
// (G, lambda_s, lambda_d) for the gradient reference.  Plain double is the other scalar.
// ------------------------------------------------------------------------------------
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0) { for (int i = 0; i < K; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < K; ++i) d[i] = 0; }
};
template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v + b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v - b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a) { Dual<K> r(-a.v); for (int i = 0; i < K; ++i) r.d[i] = -a.d[i]; return r; }
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v * b.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) { Dual<K> r(a.v / b.v); for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> Dual<K>& operator+=(Dual<K>& a, const Dual<K>& b) { a = a + b; return a; }
template <int K> Dual<K> dsqrt(const Dual<K>& a) {
  Dual<K> r(std::sqrt(a.v));
  for (int i = 0; i < K; ++i) r.d[i] = (r.v > 0) ? a.d[i] / (2.0 * r.v) : 0.0;
  return r;
}
inline double dsqrt(double a) { return std::sqrt(a); }
inline double value_of(double a) { return a; }
template <int K> double value_of(const Dual<K>& a) { return a.v; }

typedef Dual<3> D3;

// ------------------------------------------------------------------------------------
// D2Q9 lattice of Fig. 1: c_0 = 0, c_1 = (1,0) = -c_3, c_2 = (0,1) = -c_4,
// c_5 = (1,1) = -c_7, c_6 = (-1,1) = -c_8; w_0 = 4/9, w_1..4 = 1/9, w_5..8 = 1/36.
// ------------------------------------------------------------------------------------
const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int CZ[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

double link_weight(int l) {
  if (l == 0) return 4.0 / 9.0;
  if (l <= 4) return 1.0 / 9.0;
  return 1.0 / 36.0;
}

// The nine polynomials T_a(c) of Table I (tab:mom), evaluated at a link velocity.
double moment_polynomial(int a, int cx, int cz) {
  const double x = cx, z = cz, c2 = x * x + z * z;
  switch (a) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return z;
    case 3: return 3.0 * c2 - 2.0;
    case 4: return x * x - z * z;
    case 5: return x * z;
    case 6: return (3.0 * c2 - 4.0) * x;
    case 7: return (3.0 * c2 - 4.0) * z;
    default: return 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
  }
}

struct Basis {
  double T[9][9];  // T[a][l] = T_a(c_l)                            (Table I)
  double N[9];     // N_a = sum_l w_l T_al^2                        (Eq. modes-discrete)
  double w[9];
  int opp[9];      // c_opp(l) = -c_l
  Basis() {
    for (int l = 0; l < 9; ++l) {
      w[l] = link_weight(l);
      for (int m = 0; m < 9; ++m)
        if (CX[m] == -CX[l] && CZ[m] == -CZ[l]) opp[l] = m;
    }
    for (int a = 0; a < 9; ++a) {
      N[a] = 0.0;
      for (int l = 0; l < 9; ++l) {
        T[a][l] = moment_polynomial(a, CX[l], CZ[l]);
        N[a] += w[l] * T[a][l] * T[a][l];
      }
    }
  }
};
const Basis B;

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box
//   (x0,x1,x2,x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
// with the key bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * (uint64_t)x[0];
    const uint64_t p1 = (uint64_t)M1 * (uint64_t)x[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x[1] ^ k0, y1 = lo1, y2 = hi0 ^ x[3] ^ k1, y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
  }
  for (int i = 0; i < 4; ++i) out[i] = x[i];
}

// Uniform in (0,1) from the low 23 bits: (2 (k mod 2^23) + 1) 2^-24, exact in float and double.
double uniform_of(uint32_t k) { return (double)(2u * (k & 0x7FFFFFu) + 1u) * std::ldexp(1.0, -24); }

// Box-Muller (Sec. II.B draws Gaussian noise; the pairing is the textbook polar form): from the
// words (a, b), u1 = uniform_of(a), u2 = uniform_of(b), r = sqrt(-2 ln u1) and the two standard
// normals n0 = r cos(2 pi u2), n1 = r sin(2 pi u2).
void box_muller(uint32_t a, uint32_t b, double out[2]) {
  const double two_pi = 6.283185307179586476925286766559;
  const double u1 = uniform_of(a), u2 = uniform_of(b);
  const double r = std::sqrt(-2.0 * std::log(u1));
  out[0] = r * std::cos(two_pi * u2);
  out[1] = r * std::sin(two_pi * u2);
}

// Sixteen standard normals for one site and step: Box-Muller on the word pairs (k_{2i}, k_{2i+1})
// of four Philox calls (call = 0..3).
void site_normals(uint64_t seed, uint32_t lattice_id, uint32_t site, uint32_t step, double n[16]) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (uint32_t call = 0; call < 4; ++call) {
    const uint32_t ctr[4] = {site, step, lattice_id, call};
    uint32_t k[4];
    philox4x32_10(ctr, key, k);
    for (int pair = 0; pair < 2; ++pair) box_muller(k[2 * pair], k[2 * pair + 1], n + 4 * call + 2 * pair);
  }
}

// ------------------------------------------------------------------------------------
// The simulation state.  Populations are stored post-collision, f*^S_l(x, z), in the
// array f[((s * 9 + l) * Lz + z) * Lx + x]; s = 0 is species A, s = 1 is species B.
// Rows z = 0..Lz-1 sit at height z_j = j + 1/2 - Lz/2; walls at +-Lz/2 (Sec. II.A).
// ------------------------------------------------------------------------------------
template <class R>
struct Sim {
  int Lx, Lz;
  R lam[9];         // lambda_a per moment: (-, d, d, e, s, s, Q, Q, eps)     (Eq. MRT)
  R G;              // inter-species coupling                                (Eq. aNI)
  double kT;        // thermal energy
  double grad_c0;   // imposed concentration gradient, c_0(z) = 1/2 + z grad_c0
  uint64_t seed;
  uint32_t lattice_id;
  bool astar, wall_fixed, noise_loc;
  // Philox site counter of (x, z) is z * site_Lx + (x + site_x0) mod site_Lx: the identity
  // map by default; a window of a wider lattice keeps that lattice's counters.
  int site_x0 = 0, site_Lx = 0;
  double rho_bar = 1.0, c_bar0 = 0.5;  // reference values (Sec. II.A)
  std::vector<R> f;
  int64_t t = 0;
  // diagnostics
  int64_t discard = 0, every = 0, nsamples = 0;
  std::vector<double> S_acc;  // [4][Lz][Lx]: fields rho, c, Ux, Uz
  double P_sum = 0.0, P_last = 0.0;
  // z-profiles (Sec. III.C): sums over samples of the row means of rho, c, Ux, Uz and P
  std::vector<double> prof_acc;  // [5][Lz]
  // two-point correlations of the fields in corr_mask (bit f for field f): the equal-x real-space
  // correlation (1/Lx) sum_x dphi(x, z) dphi(x, z') (Sec. III.A-B) and, for the q_x mode
  // indices in corr_modes, C(q_x, z, z') = dphi(q_x, z)^* dphi(q_x, z') (Appendix A)
  int corr_mask = 0;
  int64_t corr_nsamples = 0;  // samples since the correlations were (re)enabled
  std::vector<int> corr_modes;
  std::vector<double> R_acc;  // [4][Lz][Lz]
  std::vector<double> C_acc;  // [4][modes][Lz][Lz][re, im]
  // loss accumulation for the gradient reference: sum over steps of the mean pressure
  bool accumulate_loss = false;
  R loss_sum = R(0.0);

  int idx(int s, int l, int z, int x) const { return ((s * 9 + l) * Lz + z) * Lx + x; }
  double z_of(int j) const { return j + 0.5 - 0.5 * Lz; }
  double c0(int j) const { return 0.5 + z_of(j) * grad_c0; }

  void init_rest() {
    f.assign((size_t)2 * 9 * Lz * Lx, R(0.0));
    for (int s = 0; s < 2; ++s)
      for (int l = 0; l < 9; ++l)
        for (int z = 0; z < Lz; ++z)
          for (int x = 0; x < Lx; ++x) {
            const double cs = (s == 0) ? c0(z) : 1.0 - c0(z);
            f[idx(s, l, z, x)] = R(B.w[l] * rho_bar * cs);
          }
    S_acc.assign((size_t)4 * Lz * Lx, 0.0);
    prof_acc.assign((size_t)5 * Lz, 0.0);
  }
};

// Pre-collision quantities of one step, for the whole lattice.
template <class R>
struct Pre {
  std::vector<R> fpre;   // streamed populations f^S_l(x, z, t)       [2][9][Lz][Lx]
  std::vector<R> rho;    // rho^S                                     [2][Lz][Lx]
  std::vector<R> jx, jz; // j^S                                       [2][Lz][Lx]
  std::vector<R> Fx, Fz; // force density rho^S a^S                   [2][Lz][Lx]
  std::vector<R> Ux, Uz; // barycentric velocity U (Eq. bar)          [Lz][Lx]
};

// Density of species s at (x, z), with the wall ghosts of Sec. II.A for z outside 0..Lz-1:
// the ghost row copies the adjacent fluid row, or, with a fixed wall composition, takes
// the adjacent row's total density split by c_0 at the wall.
template <class R>
R rho_ghosted(const Sim<R>& S, const std::vector<R>& rho, int s, int x, int z) {
  const int Lx = S.Lx, Lz = S.Lz;
  x = ((x % Lx) + Lx) % Lx;
  if (z >= 0 && z < Lz) return rho[(s * Lz + z) * Lx + x];
  const int zadj = (z < 0) ? 0 : Lz - 1;
  if (!S.wall_fixed) return rho[(s * Lz + zadj) * Lx + x];
  const double zwall = (z < 0) ? -0.5 * Lz : 0.5 * Lz;
  const double cw = 0.5 + zwall * S.grad_c0;
  const R total = rho[(0 * Lz + zadj) * Lx + x] + rho[(1 * Lz + zadj) * Lx + x];
  return total * ((s == 0) ? cw : 1.0 - cw);
}

template <class R>
void compute_pre(const Sim<R>& S, Pre<R>& P) {
  const int Lx = S.Lx, Lz = S.Lz, n = Lx * Lz;
  P.fpre.assign((size_t)18 * n, R(0.0));
  P.rho.assign((size_t)2 * n, R(0.0));
  P.jx.assign((size_t)2 * n, R(0.0));
  P.jz.assign((size_t)2 * n, R(0.0));
  P.Fx.assign((size_t)2 * n, R(0.0));
  P.Fz.assign((size_t)2 * n, R(0.0));
  P.Ux.assign((size_t)n, R(0.0));
  P.Uz.assign((size_t)n, R(0.0));

  // 1. Streaming, Eq. (LB): f_l(r, t) = f*_l(r - c_l, t - 1); periodic in x; a link whose
  //    source row lies beyond a wall is reflected at the mid-way wall: f_l(r) = f*_opp(l)(r).
#pragma omp parallel for collapse(3) schedule(static)
  for (int s = 0; s < 2; ++s)
    for (int l = 0; l < 9; ++l)
      for (int z = 0; z < Lz; ++z)
        for (int x = 0; x < Lx; ++x) {
          const int zs = z - CZ[l];
          const int xs = ((x - CX[l]) % Lx + Lx) % Lx;
          R v;
          if (zs >= 0 && zs < Lz) v = S.f[S.idx(s, l, zs, xs)];
          else v = S.f[S.idx(s, B.opp[l], z, x)];
          P.fpre[((s * 9 + l) * Lz + z) * Lx + x] = v;
        }

  // 2. rho^S = sum_l f^S_l, j^S = sum_l c_l f^S_l.
#pragma omp parallel for collapse(2) schedule(static)
  for (int s = 0; s < 2; ++s)
    for (int z = 0; z < Lz; ++z)
      for (int x = 0; x < Lx; ++x) {
        R r(0.0), jx(0.0), jz(0.0);
        for (int l = 0; l < 9; ++l) {
          const R v = P.fpre[((s * 9 + l) * Lz + z) * Lx + x];
          r += v;
          jx += v * (double)CX[l];
          jz += v * (double)CZ[l];
        }
        P.rho[(s * Lz + z) * Lx + x] = r;
        P.jx[(s * Lz + z) * Lx + x] = jx;
        P.jz[(s * Lz + z) * Lx + x] = jz;
      }

  // 3. Accelerations.  Eq. (aNI): a^A_NI = -G sum_l w_l c_l rho^B(r + c_l), and A <-> B.
  //    Footnote to Eq. (ne-acc): a^A_* = (1-c)(a^B_NI - a^A_NI), a^B_* = c (a^A_NI - a^B_NI).
  //    Eq. (ne-acc): a^A_NE = (1/3)(0, grad_c0 / c), a^B_NE = (1/3)(0, grad_c0 / (c - 1)).
#pragma omp parallel for schedule(static)
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x) {
      R sA_x(0.0), sA_z(0.0), sB_x(0.0), sB_z(0.0);  // sum_l w_l c_l rho^{A,B}(r + c_l)
      for (int l = 0; l < 9; ++l) {
        const R rA = rho_ghosted(S, P.rho, 0, x + CX[l], z + CZ[l]);
        const R rB = rho_ghosted(S, P.rho, 1, x + CX[l], z + CZ[l]);
        sA_x += rA * (B.w[l] * CX[l]);
        sA_z += rA * (B.w[l] * CZ[l]);
        sB_x += rB * (B.w[l] * CX[l]);
        sB_z += rB * (B.w[l] * CZ[l]);
      }
      const int i = z * Lx + x;
      const R rhoA = P.rho[i], rhoB = P.rho[n + i], rho = rhoA + rhoB;
      const R c = rhoA / rho;
      R aAx = -S.G * sB_x, aAz = -S.G * sB_z;  // a^A_NI
      R aBx = -S.G * sA_x, aBz = -S.G * sA_z;  // a^B_NI
      if (S.astar) {
        const R dAx = (1.0 - c) * (aBx - aAx), dAz = (1.0 - c) * (aBz - aAz);
        const R dBx = c * (aAx - aBx), dBz = c * (aAz - aBz);
        aAx = aAx + dAx; aAz = aAz + dAz;
        aBx = aBx + dBx; aBz = aBz + dBz;
      }
      aAz = aAz + (1.0 / 3.0) * (S.grad_c0 / c);
      aBz = aBz + (1.0 / 3.0) * (S.grad_c0 / (c - 1.0));
      P.Fx[i] = rhoA * aAx;      P.Fz[i] = rhoA * aAz;
      P.Fx[n + i] = rhoB * aBx;  P.Fz[n + i] = rhoB * aBz;
      // 4. Eq. (bar): rho U = j^A + j^B + (1/2) rho a.
      const R rUx = P.jx[i] + P.jx[n + i] + 0.5 * (P.Fx[i] + P.Fx[n + i]);
      const R rUz = P.jz[i] + P.jz[n + i] + 0.5 * (P.Fz[i] + P.Fz[n + i]);
      P.Ux[i] = rUx / rho;
      P.Uz[i] = rUz / rho;
    }
}

// Mechanical pressure at every site: half the trace of the pressure tensor (Sec. III.C),
// kinetic part (1/2) sum_S sum_l |c_l|^2 f^S_l plus the interaction part of the
// inter-species force, (G/4) sum_l w_l |c_l|^2 [rho^A(r) rho^B(r+c_l) + rho^B(r) rho^A(r+c_l)],
// whose value in a uniform state is G rho^A rho^B / 3 (Eq. EQUATIONofSTATE).
template <class R>
void pressure_field(const Sim<R>& S, const Pre<R>& P, std::vector<R>& out) {
  const int Lx = S.Lx, Lz = S.Lz, n = Lx * Lz;
  out.assign((size_t)n, R(0.0));
#pragma omp parallel for schedule(static)
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x) {
      const int i = z * Lx + x;
      R kin(0.0), inter(0.0);
      for (int s = 0; s < 2; ++s)
        for (int l = 0; l < 9; ++l)
          kin += P.fpre[((s * 9 + l) * Lz + z) * Lx + x] * (double)(CX[l] * CX[l] + CZ[l] * CZ[l]);
      for (int l = 0; l < 9; ++l) {
        const double c2 = CX[l] * CX[l] + CZ[l] * CZ[l];
        const R rAn = rho_ghosted(S, P.rho, 0, x + CX[l], z + CZ[l]);
        const R rBn = rho_ghosted(S, P.rho, 1, x + CX[l], z + CZ[l]);
        inter += (B.w[l] * c2) * (P.rho[i] * rBn + P.rho[n + i] * rAn);
      }
      out[i] = 0.5 * kin + (S.G * 0.25) * inter;
    }
}

// The 18 noise moments xi^S_a at one site (Eqs. noise-bin-expl, noise-bin-expl-high):
// xi_0 = 0; xi^A_{1,2} = sigma_d (n_0, n_1), xi^B_{1,2} = -xi^A_{1,2} with
// sigma_d^2 = (2 - lambda_d) lambda_d kT rho^A rho^B / rho; for a = 3..8,
// xi^S_a = sigma^S_a n, (sigma^S_a)^2 = 3 (2 - lambda_a) lambda_a N_a kT rho^S, species A
// drawing n_2..n_7 and species B n_8..n_13.  The densities are the reference values
// (hom) or the local pre-collision ones (loc).
template <class R>
void site_noise(const Sim<R>& S, const R& rhoA_loc, const R& rhoB_loc, uint32_t site, uint32_t step,
                R xi[2][9]) {
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a < 9; ++a) xi[s][a] = R(0.0);
  if (S.kT == 0.0) return;
  double n[16];
  site_normals(S.seed, S.lattice_id, site, step, n);
  R rA, rB;
  if (S.noise_loc) { rA = rhoA_loc; rB = rhoB_loc; }
  else { rA = R(S.rho_bar * S.c_bar0); rB = R(S.rho_bar * (1.0 - S.c_bar0)); }
  const R ld = S.lam[1];
  const R sig_d = dsqrt((2.0 - ld) * ld * S.kT * rA * rB / (rA + rB));
  xi[0][1] = sig_d * n[0];
  xi[0][2] = sig_d * n[1];
  xi[1][1] = -xi[0][1];
  xi[1][2] = -xi[0][2];
  for (int a = 3; a < 9; ++a) {
    const R la = S.lam[a];
    const R sA = dsqrt(3.0 * (2.0 - la) * la * B.N[a] * S.kT * rA);
    const R sB = dsqrt(3.0 * (2.0 - la) * la * B.N[a] * S.kT * rB);
    xi[0][a] = sA * n[a - 1];
    xi[1][a] = sB * n[a + 5];
  }
}

// Separable discrete Fourier power of one real field: |sum_{x,z} phi e^{-2 pi i (kx x/Lx +
// n z/Lz)}|^2 / (Lx Lz), written out as an O(Lx^2) transform per row followed by an O(Lz^2)
// transform per column (Appendix, Eqs. SF1 and integral on the lattice).
void dft2_power(const double* phi, int Lx, int Lz, double* out) {
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> re((size_t)Lz * Lx), im((size_t)Lz * Lx);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < Lz; ++z)
    for (int k = 0; k < Lx; ++k) {
      double sr = 0.0, si = 0.0;
      for (int x = 0; x < Lx; ++x) {
        const double ang = two_pi * (double)(((int64_t)k * x) % Lx) / (double)Lx;
        sr += phi[z * Lx + x] * std::cos(ang);
        si -= phi[z * Lx + x] * std::sin(ang);
      }
      re[z * Lx + k] = sr;
      im[z * Lx + k] = si;
    }
#pragma omp parallel for schedule(static)
  for (int k = 0; k < Lx; ++k)
    for (int q = 0; q < Lz; ++q) {
      double sr = 0.0, si = 0.0;
      for (int z = 0; z < Lz; ++z) {
        const double ang = two_pi * (double)(((int64_t)q * z) % Lz) / (double)Lz;
        const double c = std::cos(ang), s = -std::sin(ang);
        sr += re[z * Lx + k] * c - im[z * Lx + k] * s;
        si += re[z * Lx + k] * s + im[z * Lx + k] * c;
      }
      out[q * Lx + k] = (sr * sr + si * si) / ((double)Lx * (double)Lz);
    }
}

// One sample of the diagnostics on the pre-collision state: structure factors of
// delta rho = rho - rho_bar, delta c = c - c_0(z), U_x, U_z, and the mean pressure.
// The sampled field f (0 delta rho, 1 delta c, 2 Ux, 3 Uz) of Appendix A at every site.
template <class R>
void sampled_field(const Sim<R>& S, const Pre<R>& P, int fld, std::vector<double>& field) {
  const int Lx = S.Lx, Lz = S.Lz, n = Lx * Lz;
  field.assign((size_t)n, 0.0);
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x) {
      const int i = z * Lx + x;
      const double rA = value_of(P.rho[i]), rB = value_of(P.rho[n + i]);
      if (fld == 0) field[i] = rA + rB - S.rho_bar;
      else if (fld == 1) field[i] = rA / (rA + rB) - S.c0(z);
      else if (fld == 2) field[i] = value_of(P.Ux[i]);
      else field[i] = value_of(P.Uz[i]);
    }
}

// Two-point correlations of one sample, written out from their definitions: the real-space
// product averaged over x, and the products of the partial transforms
// dphi(q_x, z) = Lx^(-1/2) sum_x dphi(x, z) exp(-i q_x x) of Eq. (SF1).
template <class R>
void correlate(Sim<R>& S, const Pre<R>& P) {
  const int Lx = S.Lx, Lz = S.Lz;
  const size_t LL = (size_t)Lz * Lz, nm = S.corr_modes.size();
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> field, re((size_t)Lz), im((size_t)Lz);
  S.corr_nsamples += 1;
  for (int fld = 0; fld < 4; ++fld) {
    if (!(S.corr_mask & (1 << fld))) continue;
    sampled_field(S, P, fld, field);
    for (int z = 0; z < Lz; ++z)
      for (int zp = 0; zp < Lz; ++zp) {
        double acc = 0.0;
        for (int x = 0; x < Lx; ++x) acc += field[(size_t)z * Lx + x] * field[(size_t)zp * Lx + x];
        S.R_acc[fld * LL + (size_t)z * Lz + zp] += acc / (double)Lx;
      }
    for (size_t m = 0; m < nm; ++m) {
      const int k = S.corr_modes[m];
      for (int z = 0; z < Lz; ++z) {
        double a = 0.0, b = 0.0;
        for (int x = 0; x < Lx; ++x) {
          const double ang = two_pi * (double)(((int64_t)k * x) % Lx) / (double)Lx;
          a += field[(size_t)z * Lx + x] * std::cos(ang);
          b -= field[(size_t)z * Lx + x] * std::sin(ang);
        }
        re[z] = a / std::sqrt((double)Lx);
        im[z] = b / std::sqrt((double)Lx);
      }
      double* C = S.C_acc.data() + ((size_t)fld * nm + m) * LL * 2;
      for (int z = 0; z < Lz; ++z)
        for (int zp = 0; zp < Lz; ++zp) {
          // conj(X_z) X_z'
          C[2 * ((size_t)z * Lz + zp)] += re[z] * re[zp] + im[z] * im[zp];
          C[2 * ((size_t)z * Lz + zp) + 1] += re[z] * im[zp] - im[z] * re[zp];
        }
    }
  }
}

template <class R>
void sample(Sim<R>& S, const Pre<R>& P) {
  const int Lx = S.Lx, Lz = S.Lz, n = Lx * Lz;
  std::vector<double> field, power((size_t)n);
  for (int fld = 0; fld < 4; ++fld) {
    sampled_field(S, P, fld, field);
    dft2_power(field.data(), Lx, Lz, power.data());
    for (int i = 0; i < n; ++i) S.S_acc[(size_t)fld * n + i] += power[i];
  }
  std::vector<R> p;
  pressure_field(S, P, p);
  double mean = 0.0;
  for (int i = 0; i < n; ++i) mean += value_of(p[i]);
  mean /= (double)n;
  // row means of the absolute fields rho, c, Ux, Uz and of the pressure, one row at a time
  for (int z = 0; z < Lz; ++z) {
    double row[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int x = 0; x < Lx; ++x) {
      const int i = z * Lx + x;
      const double rA = value_of(P.rho[i]), rB = value_of(P.rho[n + i]);
      row[0] += rA + rB;
      row[1] += rA / (rA + rB);
      row[2] += value_of(P.Ux[i]);
      row[3] += value_of(P.Uz[i]);
      row[4] += value_of(p[i]);
    }
    for (int k = 0; k < 5; ++k) S.prof_acc[(size_t)k * Lz + z] += row[k] / (double)Lx;
  }
  if (S.corr_mask) correlate(S, P);
  S.P_last = mean;
  S.P_sum += mean;
  S.nsamples += 1;
}

template <class R>
uint32_t site_counter(const Sim<R>& S, int x, int z) {
  if (S.site_Lx <= 0) return (uint32_t)(z * S.Lx + x);
  return (uint32_t)((int64_t)z * S.site_Lx + (x + S.site_x0) % S.site_Lx);
}

template <class R>
bool is_sample_step(const Sim<R>& S) {
  return S.every > 0 && S.t >= S.discard && (S.t - S.discard) % S.every == 0;
}

// One time step t -> t+1 (Eq. LB with Eq. MRT):
//   m* = m + lambda (m^eq - m) + (1 - lambda/2) S + xi,   f*_l = w_l sum_a T_al m*_a / N_a.
template <class R>
void step(Sim<R>& S) {
  const int Lx = S.Lx, Lz = S.Lz, n = Lx * Lz;
  Pre<R> P;
  compute_pre(S, P);
  if (is_sample_step(S)) sample(S, P);
  if (S.accumulate_loss) {
    std::vector<R> p;
    pressure_field(S, P, p);
    R mean(0.0);
    for (int i = 0; i < n; ++i) mean += p[i];
    S.loss_sum += mean / (double)n;
  }
#pragma omp parallel for schedule(static)
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x) {
      const int i = z * Lx + x;
      const R Ux = P.Ux[i], Uz = P.Uz[i];
      R xi[2][9];
      site_noise(S, P.rho[i], P.rho[n + i], site_counter(S, x, z), (uint32_t)S.t, xi);
      for (int s = 0; s < 2; ++s) {
        R fl[9];
        for (int l = 0; l < 9; ++l) fl[l] = P.fpre[((s * 9 + l) * Lz + z) * Lx + x];
        // moments, Eq. (modes-discrete)
        R m[9];
        for (int a = 0; a < 9; ++a) {
          m[a] = R(0.0);
          for (int l = 0; l < 9; ++l) m[a] += fl[l] * B.T[a][l];
        }
        // equilibrium moments of Table I with rho^S and the barycentric U
        const R rs = P.rho[s * n + i];
        R meq[9];
        meq[0] = rs;
        meq[1] = rs * Ux;
        meq[2] = rs * Uz;
        meq[3] = 3.0 * rs * (Ux * Ux + Uz * Uz);
        meq[4] = rs * (Ux * Ux - Uz * Uz);
        meq[5] = rs * Ux * Uz;
        meq[6] = R(0.0); meq[7] = R(0.0); meq[8] = R(0.0);
        // forcing: moments of the second-order source
        //   g_l = w_l [3 (c_l - U).F + 9 (c_l.U)(c_l.F)],  F = rho^S a^S
        const R Fx = P.Fx[s * n + i], Fz = P.Fz[s * n + i];
        R g[9];
        for (int l = 0; l < 9; ++l) {
          const R cF = Fx * (double)CX[l] + Fz * (double)CZ[l];
          const R cU = Ux * (double)CX[l] + Uz * (double)CZ[l];
          const R UF = Ux * Fx + Uz * Fz;
          g[l] = B.w[l] * (3.0 * (cF - UF) + 9.0 * cU * cF);
        }
        R mstar[9];
        for (int a = 0; a < 9; ++a) {
          R Sa(0.0);
          for (int l = 0; l < 9; ++l) Sa += g[l] * B.T[a][l];
          const R la = S.lam[a];
          mstar[a] = m[a] + la * (meq[a] - m[a]) + (1.0 - 0.5 * la) * Sa + xi[s][a];
        }
        // back to populations
        for (int l = 0; l < 9; ++l) {
          R v(0.0);
          for (int a = 0; a < 9; ++a) v += B.T[a][l] * mstar[a] / B.N[a];
          S.f[S.idx(s, l, z, x)] = B.w[l] * v;
        }
      }
    }
  S.t += 1;
}

template <class R>
void set_params(Sim<R>& S, int Lx, int Lz, R ls, R ld, double le, double lq, double leps, double kT, R G,
                double grad_c0, uint64_t seed, uint32_t lattice_id, int astar, int wall_fixed, int noise_loc) {
  S.Lx = Lx; S.Lz = Lz;
  S.lam[0] = R(1.0);
  S.lam[1] = ld; S.lam[2] = ld;
  S.lam[3] = R(le);
  S.lam[4] = ls; S.lam[5] = ls;
  S.lam[6] = R(lq); S.lam[7] = R(lq);
  S.lam[8] = R(leps);
  S.kT = kT; S.G = G; S.grad_c0 = grad_c0;
  S.seed = seed; S.lattice_id = lattice_id;
  S.astar = astar != 0; S.wall_fixed = wall_fixed != 0; S.noise_loc = noise_loc != 0;
  S.init_rest();
}

}  // namespace

// ======================================================================================
// C interface for the test suite (ctypes).
// ======================================================================================
extern "C" {

typedef Sim<double> olb_sim;

void* olb_create(int Lx, int Lz, double lambda_s, double lambda_d, double lambda_e, double lambda_q,
                 double lambda_eps, double kT, double G, double grad_c0, uint64_t seed, uint32_t lattice_id,
                 int astar, int wall_fixed, int noise_loc) {
  if (Lx < 1 || Lz < 2) return nullptr;
  olb_sim* S = new olb_sim();
  set_params<double>(*S, Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G, grad_c0, seed,
                     lattice_id, astar, wall_fixed, noise_loc);
  return S;
}

void olb_destroy(void* h) { delete (olb_sim*)h; }

void olb_set_sampling(void* h, int64_t discard, int64_t every) {
  olb_sim* S = (olb_sim*)h;
  S->discard = discard;
  S->every = every;
}

void olb_step(void* h, int64_t nsteps) {
  olb_sim* S = (olb_sim*)h;
  for (int64_t k = 0; k < nsteps; ++k) step(*S);
}

int64_t olb_time(void* h) { return ((olb_sim*)h)->t; }

void olb_set_site_map(void* h, int x0, int Lx_global) {
  olb_sim* S = (olb_sim*)h;
  S->site_x0 = x0;
  S->site_Lx = Lx_global;
}
void olb_set_time(void* h, int64_t t) { ((olb_sim*)h)->t = t; }

void olb_get_populations(void* h, double* out) {
  olb_sim* S = (olb_sim*)h;
  std::memcpy(out, S->f.data(), S->f.size() * sizeof(double));
}

void olb_set_populations(void* h, const double* in) {
  olb_sim* S = (olb_sim*)h;
  std::memcpy(S->f.data(), in, S->f.size() * sizeof(double));
}

// Per-species total mass of the stored state.
void olb_mass(void* h, double out[2]) {
  olb_sim* S = (olb_sim*)h;
  const size_t n = (size_t)S->Lx * S->Lz;
  for (int s = 0; s < 2; ++s) {
    double m = 0.0;
    for (size_t k = 0; k < 9 * n; ++k) m += S->f[s * 9 * n + k];
    out[s] = m;
  }
}

// Pre-collision fields of the next step, from the stored state, without changing it:
// out[0..4][Lz][Lx] = rho^A, rho^B, U_x, U_z, pressure.
void olb_fields(void* h, double* out) {
  olb_sim* S = (olb_sim*)h;
  Pre<double> P;
  compute_pre(*S, P);
  std::vector<double> p;
  pressure_field(*S, P, p);
  const size_t n = (size_t)S->Lx * S->Lz;
  std::memcpy(out, P.rho.data(), 2 * n * sizeof(double));
  std::memcpy(out + 2 * n, P.Ux.data(), n * sizeof(double));
  std::memcpy(out + 3 * n, P.Uz.data(), n * sizeof(double));
  std::memcpy(out + 4 * n, p.data(), n * sizeof(double));
}

// Structure-factor average of one field (0 rho, 1 c, 2 Ux, 3 Uz), [Lz][Lx] indexed (q_z, q_x).
int64_t olb_structure_factor(void* h, int field, double* out) {
  olb_sim* S = (olb_sim*)h;
  const size_t n = (size_t)S->Lx * S->Lz;
  for (size_t i = 0; i < n; ++i)
    out[i] = S->nsamples ? S->S_acc[(size_t)field * n + i] / (double)S->nsamples : 0.0;
  return S->nsamples;
}

// Correlations from the next sample on: field mask (bit f for field f), q_x mode indices.
void olb_set_correlations(void* h, int mask, int n_modes, const int* modes) {
  olb_sim* S = (olb_sim*)h;
  S->corr_mask = mask & 15;
  S->corr_nsamples = 0;
  S->corr_modes.assign(modes, modes + n_modes);
  const size_t LL = (size_t)S->Lz * S->Lz;
  S->R_acc.assign(4 * LL, 0.0);
  S->C_acc.assign(4 * (size_t)n_modes * LL * 2, 0.0);
}

// Averages over the samples: R (Lz x Lz) of a field; C of a field and mode (Lz x Lz complex).
int64_t olb_correlation(void* h, int field, double* out) {
  olb_sim* S = (olb_sim*)h;
  const size_t LL = (size_t)S->Lz * S->Lz;
  const int64_t n = S->corr_nsamples;
  for (size_t i = 0; i < LL; ++i) out[i] = n ? S->R_acc[field * LL + i] / (double)n : 0.0;
  return n;
}

int64_t olb_mode_correlation(void* h, int field, int mode_index, double* out) {
  olb_sim* S = (olb_sim*)h;
  const size_t LL = (size_t)S->Lz * S->Lz, nm = S->corr_modes.size();
  const double* C = S->C_acc.data() + ((size_t)field * nm + mode_index) * LL * 2;
  const int64_t n = S->corr_nsamples;
  for (size_t i = 0; i < 2 * LL; ++i) out[i] = n ? C[i] / (double)n : 0.0;
  return n;
}

// Time-averaged row means of field k (0 rho, 1 c, 2 Ux, 3 Uz, 4 P) at rows 0..Lz-1.
int64_t olb_profile(void* h, int field, double* out) {
  olb_sim* S = (olb_sim*)h;
  for (int z = 0; z < S->Lz; ++z)
    out[z] = S->nsamples ? S->prof_acc[(size_t)field * S->Lz + z] / (double)S->nsamples : 0.0;
  return S->nsamples;
}

int64_t olb_mean_pressure(void* h, double* last, double* avg) {
  olb_sim* S = (olb_sim*)h;
  *last = S->P_last;
  *avg = S->nsamples ? S->P_sum / (double)S->nsamples : 0.0;
  return S->nsamples;
}

// Noise moments xi^S_a of one site at step `step` for the current stored state's densities
// (used only for loc noise): out[0..8] species A, out[9..17] species B.
void olb_site_noise(void* h, int x, int z, int64_t step_index, double* out) {
  olb_sim* S = (olb_sim*)h;
  Pre<double> P;
  compute_pre(*S, P);
  const int n = S->Lx * S->Lz, i = z * S->Lx + x;
  double xi[2][9];
  site_noise(*S, P.rho[i], P.rho[n + i], site_counter(*S, x, z), (uint32_t)step_index, xi);
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a < 9; ++a) out[s * 9 + a] = xi[s][a];
}

// Threads of the row loops in a build with OpenMP (n > 0 sets them); returns the count in use,
// 1 in the plain build.
int olb_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void olb_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key, out);
}

void olb_site_normals(uint64_t seed, uint32_t lattice_id, uint32_t site, uint32_t step_index, double* out) {
  site_normals(seed, lattice_id, site, step_index, out);
}

// words: 2 n_pairs values (a_0, b_0, a_1, b_1, ...); out: 2 n_pairs normals in the same order.
void olb_box_muller(const uint32_t* words, int64_t n_pairs, double* out) {
  for (int64_t i = 0; i < n_pairs; ++i) box_muller(words[2 * i], words[2 * i + 1], out + 2 * i);
}

void olb_basis(double* T, double* w, double* N) {
  for (int a = 0; a < 9; ++a) {
    N[a] = B.N[a];
    for (int l = 0; l < 9; ++l) T[a * 9 + l] = B.T[a][l];
  }
  for (int l = 0; l < 9; ++l) w[l] = B.w[l];
}

void olb_dft2_power(const double* phi, int Lx, int Lz, double* out) { dft2_power(phi, Lx, Lz, out); }

// Gradient reference for the mean-pressure shift
//   L = (1/n) sum_{t<n} Pbar(t)|_{kT} - (1/n) sum_{t<n} Pbar(t)|_{kT=0}
// with respect to (G, lambda_s, lambda_d), by forward-mode dual numbers through both runs
// from the rest state.  grad[0..2] = dL/dG, dL/dlambda_s, dL/dlambda_d.
void olb_pressure_shift_grad(int Lx, int Lz, double lambda_s, double lambda_d, double lambda_e,
                             double lambda_q, double lambda_eps, double kT, double G, double grad_c0,
                             uint64_t seed, uint32_t lattice_id, int astar, int wall_fixed, int noise_loc,
                             int64_t nsteps, double* loss, double* grad) {
  double Lv[2];
  D3 Ld[2];
  for (int run = 0; run < 2; ++run) {
    Sim<D3> S;
    D3 Gd(G), lsd(lambda_s), ldd(lambda_d);
    Gd.d[0] = 1.0;
    lsd.d[1] = 1.0;
    ldd.d[2] = 1.0;
    set_params<D3>(S, Lx, Lz, lsd, ldd, lambda_e, lambda_q, lambda_eps, run == 0 ? kT : 0.0, Gd, grad_c0, seed,
                   lattice_id, astar, wall_fixed, noise_loc);
    S.accumulate_loss = true;
    for (int64_t k = 0; k < nsteps; ++k) step(S);
    Ld[run] = S.loss_sum / (double)nsteps;
    Lv[run] = Ld[run].v;
  }
  *loss = Lv[0] - Lv[1];
  for (int i = 0; i < 3; ++i) grad[i] = Ld[0].d[i] - Ld[1].d[i];
}

// The same loss in plain double precision (for finite differences of the oracle itself).
double olb_pressure_shift(int Lx, int Lz, double lambda_s, double lambda_d, double lambda_e, double lambda_q,
                          double lambda_eps, double kT, double G, double grad_c0, uint64_t seed,
                          uint32_t lattice_id, int astar, int wall_fixed, int noise_loc, int64_t nsteps) {
  double Lv[2];
  for (int run = 0; run < 2; ++run) {
    Sim<double> S;
    set_params<double>(S, Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, run == 0 ? kT : 0.0, G,
                       grad_c0, seed, lattice_id, astar, wall_fixed, noise_loc);
    S.accumulate_loss = true;
    for (int64_t k = 0; k < nsteps; ++k) step(S);
    Lv[run] = S.loss_sum / (double)nsteps;
  }
  return Lv[0] - Lv[1];
}

}  // extern "C"
