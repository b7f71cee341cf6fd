// lb_adjoint.cuh -- host interface of the adjoint sweep (lb_adjoint.cu): the gradient of the
// time-averaged mean-pressure shift with respect to (G, lambda_s, lambda_d).
#pragma once

#include "lb_internal.cuh"

namespace lbk {

// One warp per block: the transposed step runs at about 166 registers, so a lattice of a few
// ten thousand sites is fewer threads than the GPU holds, and the smallest blocks spread them
// most evenly over the SMs (measured on 256 x 128: 32 threads 0.476 s per gradient, 128
// threads 0.504 s).
constexpr int kAdjBlock = 32;
inline int adjoint_blocks(int n_sites) { return (n_sites + kAdjBlock - 1) / kAdjBlock; }

// Per-lattice constants of the transposed step, formed once on the host in double precision from
// the rates and noise amplitudes the device holds.  For sigma^2 = K (2 - lambda) lambda,
// d sigma / d lambda = sigma (1 - lambda) / ((2 - lambda) lambda).
struct AdjConst {
  double oml[9];  // 1 - lambda_a (relaxation, Eq. MRT)
  double ohl[6];  // 1 - lambda_a / 2 (second-order forcing, moments 1..5)
  double dsm;     // d sigma / d lambda_d of the momentum noise (moments 1, 2), hom noise
  double d4, d5;  // d sigma / d lambda_s of moments 4 and 5, hom noise
  // loc noise: sigma_mom = pm sqrt(rho^A rho^B / rho) and sigma^S_a = pa[a] sqrt(rho^S) with the
  // local densities; dpm = d pm / d lambda_d, dp4 and dp5 = d pa[4], pa[5] / d lambda_s
  double pm, dpm, pa[9], dp4, dp5;
  bool options;   // any of no a*, fixed wall composition, loc noise (the kernels that handle them)
  double w_loss;  // 1 / (T N): the loss's weight of one site's pressure at one step (set per call)
};

template <class real>
inline AdjConst adjoint_constants(const LatticeDev<real>& L) {
  AdjConst k;
  for (int a = 0; a < 9; ++a) k.oml[a] = 1 - (double)L.lam[a];
  for (int a = 0; a < 6; ++a) k.ohl[a] = 1 - 0.5 * (double)L.lam[a];
  auto dsigma = [](double sigma, double lam) { return sigma * (1 - lam) / ((2 - lam) * lam); };
  const double ld = (double)L.lam[1], ls = (double)L.lam[4];
  k.dsm = dsigma((double)L.sig_mom, ld);
  k.d4 = dsigma((double)L.sig[4], ls);
  k.d5 = dsigma((double)L.sig[5], ls);
  k.pm = (double)L.pref_mom;
  k.dpm = dsigma(k.pm, ld);
  for (int a = 0; a < 9; ++a) k.pa[a] = a >= 3 ? (double)L.pref[a] : 0.0;
  k.dp4 = dsigma(k.pa[4], ls);
  k.dp5 = dsigma(k.pa[5], ls);
  k.options = !(L.flags & DF_ASTAR) || (L.flags & (DF_WALL_FIXED | DF_NOISE_LOC));
  return k;
}

// The adjoint's blocks over a batch: the blocks of lattice i are first[i] .. first[i + 1] - 1
// (adjoint_blocks of its sites each), lat_of[b] the lattice of block b; so every block belongs to
// one lattice and a lattice's blocks and sums are those of the lattice alone.  Device arrays.
struct AdjMap {
  const int* lat_of;  // [n_blocks]
  const int* first;   // [n_lat + 1]
  int n_blocks, n_lat;
};

// One adjoint step of every lattice of the batch: from fbar (sensitivity to f*_k) and the forward
// state f_prev = f*_{k-1}, write fbar_prev and add this step's gradient share, block by block, to
// partials (3 doubles per block, zeroed before the sweep); then launch_adjoint_gradient sums each
// lattice's blocks into grads[3 i ..].  The site-indexed buffers hold the lattices one after
// another at their site offsets (LatticeDev::site_off): rho 2, fl and fbar 18, sb 4 doubles per
// site; the states have the context's layout (LatticeDev::f_off).  rho holds the densities of
// f_prev if rho_ready, else they are computed first; with f_next = f*_{k-2} given, its densities
// go to rho_next for the next step.  kcs: the lattices' AdjConst (device); options: any lattice
// uses a non-default option of the step; sign: +1 for the noisy run, -1 for the noiseless one
// (the loss weight of a site is sign w_loss).  The sensitivities are double precision for either
// state precision.
template <class real>
cudaError_t launch_adjoint_step(const real* f_prev, const real* f_next, const double* fbar, double* fbar_prev,
                                const LatticeDev<real>* lat, const RowConst<real>* rows, const AdjConst* kcs,
                                bool options, const AdjMap& map, uint32_t step, bool noise, double sign,
                                bool rho_ready, double* rho, double* rho_next, double* fl, double* sb,
                                double* partials, cudaStream_t s);
cudaError_t launch_adjoint_gradient(const double* partials, const AdjMap& map, double* grads, cudaStream_t s);

}  // namespace lbk
