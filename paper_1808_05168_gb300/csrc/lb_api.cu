// lb_api.cu -- host runtime behind the C interface of lb.h: contexts, device memory, work
// decomposition, step scheduling (direct launches, CUDA graphs, or one cooperative
// persistent launch per run of steps), sampling, autotuning of the tile shape.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lb_adjoint.cuh"
#include "lb_internal.cuh"

using namespace lbk;

namespace {

const double kRhoBar = 1.0;  // reference total density (Sec. II.A)
constexpr double kCBar0 = 0.5;  // reference concentration c_0(z = 0) (Sec. II.A)
const double kNorm[9] = {1.0, 1.0 / 3, 1.0 / 3, 4.0, 4.0 / 9, 1.0 / 9, 2.0 / 3, 2.0 / 3, 16.0};  // N_a, Table I

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// An NVTX range over a host call (profilers show where lb_step, the sampling, the autotuner and the
// adjoint sweeps enqueue their work; without a profiler attached it costs a branch).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct GraphKey {
  int64_t nsteps;
  std::vector<int64_t> samples;  // the steps of the segment that sample
  int cur;
  int mode;
  bool operator<(const GraphKey& o) const {
    return std::tie(nsteps, samples, cur, mode) < std::tie(o.nsteps, o.samples, o.cur, o.mode);
  }
};

}  // namespace

struct lb_ctx {
  // device memory: the caller's allocator when one was given, else cudaMalloc / cudaFree
  lb_alloc_fn alloc_fn = nullptr;
  lb_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  int n_lat = 0;
  int flags = 0;
  bool dev32 = false;
  std::vector<lb_params> params;
  std::vector<std::pair<int, int>> site_map;  // per lattice: (x0, Lx of the whole lattice), lb_set_site_map
  std::vector<int64_t> f_off, site_off;
  std::vector<int> row_off;
  int64_t n_f = 0, n_sites = 0;
  int n_rows = 0;
  int max_lattice_sites = 0;

  // tiles
  int tile_x = 128, rows_per_item = 64;
  bool tile_fixed = false, tuned = false;
  std::vector<WorkItem> items;

  // device memory
  void* d_lat = nullptr;    // LatticeDev<real>[n_lat]
  void* d_rows = nullptr;   // RowConst<real>[n_rows]
  WorkItem* d_items = nullptr;
  int d_items_cap = 0;
  void* f[2] = {nullptr, nullptr};
  void* fields = nullptr;   // 4 * n_sites reals
  void* pfield = nullptr;   // n_sites reals: sampled pressure
  double* prof_sum = nullptr;   // 5 * n_rows: z-profiles
  double* prof_comp = nullptr;
  int* d_row_lat = nullptr;     // n_rows: lattice of each global row
  // two-point correlations (lb_set_correlations)
  int corr_mask = 0;
  std::vector<int> corr_modes;
  double* corr_R = nullptr;
  double* corr_C = nullptr;
  size_t corr_R_n = 0, corr_C_n = 0;  // doubles
  int4* d_corr_real = nullptr;
  int4* d_corr_mode = nullptr;
  int* d_corr_modes = nullptr;
  int n_corr_real = 0, n_corr_mode = 0;
  int64_t corr_samples = 0;
  void* tmp = nullptr;      // 4 * n_sites complex
  double* acc_sum = nullptr;
  double* acc_comp = nullptr;
  double* partials = nullptr;
  int partials_cap = 0;
  DiagStats* stats = nullptr;
  DiagLattice* d_diag = nullptr;
  int2* d_row_tasks = nullptr;
  int2* d_col_tasks = nullptr;
  int n_row_tasks = 0, n_col_tasks = 0;
  int max_Lx = 0, max_Lz = 0;
  int sf_threads = 256, sf_cap = 4096;  // sample-step transforms (sf_threads, SfPlan)
  size_t sf_smem_rows = 0, sf_smem_cols = 0;
  int64_t* d_t = nullptr;
  unsigned* d_barrier = nullptr;  // the persistent launch's ticket counter (64-bit)
  unsigned* d_done = nullptr;     // persistent launch: steps completed per item
  int* d_nbr_off = nullptr;       // persistent launch: dependency lists of the items (CSR)
  int* d_nbr = nullptr;
  int sched_items_cap = 0, sched_nbr_cap = 0;
  CUtensorMap* d_tmaps = nullptr;  // bulk staging: 3-d tensor maps [buffer][lattice][run of 1, 2 links]
  bool tma = false;                // d_tmaps holds maps for the current tile
  int* d_err = nullptr;
  double* d_scratch = nullptr;  // 18 * max_lattice_sites doubles (populations I/O)
  double* d_mass = nullptr;
  size_t bytes = 0;

  std::vector<DiagLattice> diag;
  bool diag_ready = false;
  int cur = 0;
  int64_t t = 0, discard = 0, every = 0, nsamples = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int coop_grid = -1;
  int noise_mode = NOISE_OFF;  // NOISE_OFF, NOISE_HOM or NOISE_LOC for the whole batch
  bool bulk_ok = false;        // every lattice's rows are 16-byte aligned and bulk copies are allowed
  std::map<GraphKey, std::pair<cudaGraphExec_t, int64_t>> graphs;  // graph, kernels in it
  int64_t launches = 0;  // kernels enqueued by lb_step so far (graph replays included)
};

namespace {

// Every device buffer of a context comes from here and goes back through dev_free.
void* ctx_malloc(lb_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->alloc_fn) return c->alloc_fn(bytes, c->alloc_user);
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return q;
}

void dev_free(lb_ctx* c, void* p) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, c->alloc_user);
  else cudaFree(p);
}

template <class T>
int dev_alloc(lb_ctx* c, T** p, size_t bytes) {
  *p = (T*)ctx_malloc(c, bytes);
  if (!*p) return LB_ERR_OOM;
  c->bytes += bytes ? bytes : 16;
  return LB_OK;
}

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return LB_OK;
  return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
}

int check_params(const lb_params& p) {
  auto rate_ok = [](double l) { return std::isfinite(l) && l > 0.0 && l < 2.0; };
  if (p.Lx < 1 || p.Lz < 2) return LB_ERR_BAD_PARAM;
  if ((int64_t)p.Lx * p.Lz * 18 >= (int64_t)1 << 31) return LB_ERR_BAD_PARAM;
  if (!rate_ok(p.lambda_s) || !rate_ok(p.lambda_d) || !rate_ok(p.lambda_e) || !rate_ok(p.lambda_q) ||
      !rate_ok(p.lambda_eps))
    return LB_ERR_BAD_PARAM;
  if (!std::isfinite(p.kT) || p.kT < 0.0) return LB_ERR_BAD_PARAM;
  if (!std::isfinite(p.G) || p.G < 0.0) return LB_ERR_BAD_PARAM;
  if (!std::isfinite(p.grad_c0) || std::fabs(p.grad_c0) * p.Lz >= 1.0) return LB_ERR_BAD_PARAM;
  if (p.reserved != 0) return LB_ERR_BAD_PARAM;
  return LB_OK;
}

double c0_of(const lb_params& p, double z) { return kCBar0 + z * p.grad_c0; }

// Per-lattice device constants (Eqs. MRT, noise-bin-expl, noise-bin-expl-high, ne-acc).
template <class real>
LatticeDev<real> make_lattice(const lb_params& p, int flags, bool dev, int64_t f_off, int64_t site_off, int row_off) {
  LatticeDev<real> L;
  std::memset(&L, 0, sizeof(L));
  L.Lx = p.Lx;
  L.Lz = p.Lz;
  L.f_off = f_off;
  L.site_off = site_off;
  L.row_off = row_off;
  L.flags = 0;
  if (!(flags & LB_NO_ASTAR)) L.flags |= DF_ASTAR;
  if (flags & LB_WALL_FIXED) L.flags |= DF_WALL_FIXED;
  if (flags & LB_NOISE_LOC) L.flags |= DF_NOISE_LOC;
  if (p.kT > 0) L.flags |= DF_NOISE;
  L.key0 = (uint32_t)(p.seed & 0xffffffffu);
  L.key1 = (uint32_t)(p.seed >> 32);
  L.lattice_id = p.lattice_id;
  L.site_x0 = 0;
  L.site_Lx = p.Lx;
  const double lam[9] = {1.0, p.lambda_d, p.lambda_d, p.lambda_e, p.lambda_s, p.lambda_s, p.lambda_q, p.lambda_q,
                         p.lambda_eps};
  bool unit = true;
  for (int a = 0; a < 9; ++a) {
    L.lam[a] = (real)lam[a];
    L.omh[a] = (real)(1.0 - 0.5 * lam[a]);
    if (a >= 3 && lam[a] != 1.0) unit = false;
  }
  if (unit) L.flags |= DF_UNIT;
  L.G = (real)p.G;
  L.g3 = (real)(p.grad_c0 / 3.0);
  L.k9 = dev ? (real)(kRhoBar * p.grad_c0 / 9.0) : (real)0;
  L.k36 = dev ? (real)(kRhoBar * p.grad_c0 / 36.0) : (real)0;
  L.rho_bar_off = dev ? (real)0 : (real)kRhoBar;
  const double rA = kRhoBar * kCBar0, rB = kRhoBar * (1.0 - kCBar0);
  const double ld = p.lambda_d;
  L.sig_mom = (real)std::sqrt((2.0 - ld) * ld * p.kT * rA * rB / (rA + rB));
  L.pref_mom = (real)std::sqrt((2.0 - ld) * ld * p.kT);
  static_assert(kCBar0 == 0.5, "hom noise amplitudes assume equal reference densities");
  for (int a = 3; a < 9; ++a) {
    const double v = 3.0 * (2.0 - lam[a]) * lam[a] * kNorm[a] * p.kT;
    L.sig[a] = (real)std::sqrt(v * rA);
    L.pref[a] = (real)std::sqrt(v);
  }
  // folded coefficients (see LatticeDev::kA): constant factors of m^eq_3 (3), S_3 (6), S_4 (2),
  // and the weight 1/36 of the diagonal links, which the inverse transform then needs no more
  const bool loc = flags & LB_NOISE_LOC;
  for (int a = 0; a < 9; ++a) {
    const double invN = 1.0 / (36.0 * kNorm[a]);
    const double qf = a == 3 ? 3.0 : 1.0, sf = a == 3 ? 6.0 : (a == 4 ? 2.0 : 1.0);
    L.kA[a] = (real)((1.0 - lam[a]) * invN);
    L.kB[a] = (real)(a >= 1 && a <= 5 ? lam[a] * qf * invN : 0.0);
    L.kC[a] = (real)(a >= 1 && a <= 5 ? (1.0 - 0.5 * lam[a]) * sf * invN : 0.0);
    double sig = 0.0;
    if (a == 1 || a == 2) sig = loc ? std::sqrt((2.0 - ld) * ld * p.kT) : std::sqrt((2.0 - ld) * ld * p.kT * rA * rB / (rA + rB));
    else if (a >= 3) sig = std::sqrt(3.0 * (2.0 - lam[a]) * lam[a] * kNorm[a] * p.kT * (loc ? 1.0 : rA));
    L.kN[a] = (real)(sig * invN);
  }
  return L;
}

// Per-row background constants in double, with the wall ghosts of Sec. II.A.
struct RowD {
  double bgA, bgB, dbgA, dbgB, nbA, nbB, c0, ghost_cA, Pbg;
};

std::vector<RowD> make_rows(const lb_params& p, int flags, bool dev) {
  const int Lz = p.Lz;
  const bool fixed = flags & LB_WALL_FIXED;
  const double cw_bot = c0_of(p, -0.5 * Lz), cw_top = c0_of(p, 0.5 * Lz);
  auto bg = [&](int s, int z) -> double {  // z in -1..Lz
    if (!dev) return 0.0;
    double c;
    if (z < 0) c = fixed ? cw_bot : c0_of(p, 0 + 0.5 - 0.5 * Lz);
    else if (z >= Lz) c = fixed ? cw_top : c0_of(p, (Lz - 1) + 0.5 - 0.5 * Lz);
    else c = c0_of(p, z + 0.5 - 0.5 * Lz);
    return kRhoBar * (s == 0 ? c : 1.0 - c);
  };
  std::vector<RowD> rows(Lz);
  for (int z = 0; z < Lz; ++z) {
    RowD r;
    r.c0 = c0_of(p, z + 0.5 - 0.5 * Lz);
    r.bgA = bg(0, z);
    r.bgB = bg(1, z);
    r.dbgA = (bg(0, z + 1) - bg(0, z - 1)) / 6.0;
    r.dbgB = (bg(1, z + 1) - bg(1, z - 1)) / 6.0;
    r.nbA = 2.0 / 9.0 * (bg(0, z - 1) + bg(0, z) + bg(0, z + 1));
    r.nbB = 2.0 / 9.0 * (bg(1, z - 1) + bg(1, z) + bg(1, z + 1));
    r.ghost_cA = (z == 0) ? cw_bot : (z == Lz - 1 ? cw_top : 0.0);
    r.Pbg = (r.bgA + r.bgB) / 3.0 + 0.25 * p.G * (r.bgA * r.nbB + r.bgB * r.nbA);
    rows[z] = r;
  }
  return rows;
}

template <class real>
int upload_tables(lb_ctx* c) {
  std::vector<LatticeDev<real>> lat(c->n_lat);
  std::vector<RowConst<real>> rows(c->n_rows);
  c->diag.assign(c->n_lat, DiagLattice());
  for (int i = 0; i < c->n_lat; ++i) {
    const lb_params& p = c->params[i];
    lat[i] = make_lattice<real>(p, c->flags, c->dev32, c->f_off[i], c->site_off[i], c->row_off[i]);
    lat[i].site_x0 = c->site_map[i].first;
    lat[i].site_Lx = c->site_map[i].second;
    const std::vector<RowD> rd = make_rows(p, c->flags, c->dev32);
    double Pbg = 0.0, mA = 0.0, mB = 0.0;
    for (int z = 0; z < p.Lz; ++z) {
      const RowD& r = rd[z];
      RowConst<real> rc;
      rc.bgA = (real)r.bgA; rc.bgB = (real)r.bgB;
      rc.dbgA = (real)r.dbgA; rc.dbgB = (real)r.dbgB;
      rc.nbA = (real)r.nbA; rc.nbB = (real)r.nbB;
      rc.c0 = (real)r.c0; rc.ghost_cA = (real)r.ghost_cA;
      rows[c->row_off[i] + z] = rc;
      Pbg += r.Pbg;
      mA += r.bgA;
      mB += r.bgB;
    }
    DiagLattice& d = c->diag[i];
    d.Lx = p.Lx;
    d.Lz = p.Lz;
    d.site_off = c->site_off[i];
    d.row_off = c->row_off[i];
    d.P_bg_mean = Pbg / p.Lz;
    d.mass_bg[0] = mA * p.Lx;
    d.mass_bg[1] = mB * p.Lx;
    d.n_sites = (double)p.Lx * p.Lz;
  }
  int rc = dev_alloc(c, (char**)&c->d_lat, lat.size() * sizeof(LatticeDev<real>));
  if (rc) return rc;
  rc = dev_alloc(c, (char**)&c->d_rows, rows.size() * sizeof(RowConst<real>));
  if (rc) return rc;
  if (cudaMemcpy(c->d_lat, lat.data(), lat.size() * sizeof(LatticeDev<real>), cudaMemcpyHostToDevice) != cudaSuccess)
    return LB_ERR_CUDA;
  if (cudaMemcpy(c->d_rows, rows.data(), rows.size() * sizeof(RowConst<real>), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return LB_ERR_CUDA;
  return LB_OK;
}

void drop_graphs(lb_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  c->graphs.clear();
}

// Work items: lattices with more rows per item first (longest work first), each lattice's
// items contiguous so that its partial sums can be reduced in a fixed order.
// Work items of a batch (host only): per lattice, row chunks of `rows` rows, each split into
// column strips of tile_x columns; lattices with the longest chunks first.  range[i]: the items
// of lattice i.
void plan_items(const std::vector<int>& Lx, const std::vector<int>& Lz, int tile_x, int rows,
                std::vector<WorkItem>& items, std::vector<std::pair<int, int>>& range) {
  const int n = (int)Lx.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return std::min(rows, Lz[a]) > std::min(rows, Lz[b]); });
  items.clear();
  range.assign(n, {0, 0});
  for (int i : order) {
    const int begin = (int)items.size();
    for (int z0 = 0; z0 < Lz[i]; z0 += rows)
      for (int x0 = 0; x0 < Lx[i]; x0 += tile_x) items.push_back(WorkItem{i, x0, z0, std::min(z0 + rows, Lz[i])});
    range[i] = {begin, (int)items.size()};
  }
}

// Dependency lists of the persistent launch (host only; see the persistent kernels): for every
// item, the items of its lattice whose regions meet its rows z0 - 2 .. z1 + 1 and its columns
// x0 - 4 .. x0 + w + 3 (periodic in x), itself included.  The items of a lattice are ordered
// row chunk by row chunk, column strip by column strip, from range[lattice].first.
void plan_dependencies(const std::vector<int>& Lx, const std::vector<int>& Lz, const std::vector<WorkItem>& items,
                       const std::vector<std::pair<int, int>>& range, int tile_x, int rows, std::vector<int>& off,
                       std::vector<int>& nbr) {
  off.assign(items.size() + 1, 0);
  nbr.clear();
  nbr.reserve(items.size() * 9);
  std::vector<int> strips;
  for (size_t i = 0; i < items.size(); ++i) {
    const WorkItem& it = items[i];
    const int lx = Lx[it.lattice], lz = Lz[it.lattice];
    const int begin = range[it.lattice].first;
    const int nstrips = (lx + tile_x - 1) / tile_x;
    const int w = std::min(tile_x, lx - it.x0);
    const int ca = std::max(0, it.z0 - 2) / rows, cb = std::min(lz - 1, it.z1 + 1) / rows;
    strips.clear();
    const int len = w + 8;
    if (len >= lx) {
      for (int sx = 0; sx < nstrips; ++sx) strips.push_back(sx);
    } else {
      const int xs = ((it.x0 - 4) % lx + lx) % lx, xe = xs + len;  // columns [xs, xe), wrapping once
      for (int sx = xs / tile_x; sx <= (std::min(xe, lx) - 1) / tile_x; ++sx) strips.push_back(sx);
      if (xe > lx)
        for (int sx = 0; sx <= (xe - lx - 1) / tile_x; ++sx) strips.push_back(sx);
      std::sort(strips.begin(), strips.end());
      strips.erase(std::unique(strips.begin(), strips.end()), strips.end());
    }
    for (int ch = ca; ch <= cb; ++ch)
      for (int sx : strips) nbr.push_back(begin + ch * nstrips + sx);
    off[i + 1] = (int)nbr.size();
  }
}

void lattice_shapes(const lb_ctx* c, std::vector<int>& Lx, std::vector<int>& Lz) {
  Lx.resize(c->n_lat);
  Lz.resize(c->n_lat);
  for (int i = 0; i < c->n_lat; ++i) {
    Lx[i] = c->params[i].Lx;
    Lz[i] = c->params[i].Lz;
  }
}

// The dependency lists of the items on the device.
int build_schedule(lb_ctx* c, const std::vector<WorkItem>& items, const std::vector<std::pair<int, int>>& range,
                   int tile_x, int rows) {
  std::vector<int> Lx, Lz, off, nbr;
  lattice_shapes(c, Lx, Lz);
  plan_dependencies(Lx, Lz, items, range, tile_x, rows, off, nbr);
  const int n = (int)items.size(), m = (int)nbr.size();
  if (n + 1 > c->sched_items_cap) {
    if (c->d_done) {
      dev_free(c, c->d_done);
      dev_free(c, c->d_nbr_off);
      c->bytes -= (size_t)c->sched_items_cap * (sizeof(unsigned) + sizeof(int));
      c->d_done = nullptr;
      c->d_nbr_off = nullptr;
    }
    int rc = dev_alloc(c, &c->d_done, (size_t)(n + 1) * sizeof(unsigned));
    if (!rc) rc = dev_alloc(c, &c->d_nbr_off, (size_t)(n + 1) * sizeof(int));
    if (rc) return rc;
    c->sched_items_cap = n + 1;
  }
  if (m > c->sched_nbr_cap) {
    if (c->d_nbr) {
      dev_free(c, c->d_nbr);
      c->bytes -= (size_t)c->sched_nbr_cap * sizeof(int);
      c->d_nbr = nullptr;
    }
    int rc = dev_alloc(c, &c->d_nbr, (size_t)m * sizeof(int));
    if (rc) return rc;
    c->sched_nbr_cap = m;
  }
  if (cudaMemcpy(c->d_nbr_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      (m > 0 && cudaMemcpy(c->d_nbr, nbr.data(), (size_t)m * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
    return LB_ERR_CUDA;
  return LB_OK;
}

// The tensor maps of the bulk staging (see the bulk path of the step kernels): for both FP32 state
// buffers and every lattice with strips away from its x edges (Lx > 2 tile_x), the (A, B) pairs
// as [link][z][x] with a box of tile_x + 4 pairs (two halo columns per side), one row and one or
// two links.  Any map the driver does not accept switches the tensor copies off for the context
// (the 1-d copies remain).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    cudaGetLastError();
  }
  return fn;
}

// Tensor maps of the FP32 state: each (A, B) pair is one 8-byte element of a 3-d map [x][z][link]
// (an FP64 pair, 16 bytes, has no element type; those rows go by 1-d bulk copies).
int build_tmaps(lb_ctx* c, int tile_x) {
  c->tma = false;
  const int es = 8, pad = 2, bw = tile_x + 2 * pad;  // bytes per pair, halo columns
  if (!c->dev32 || !c->bulk_ok || (c->flags & LB_NO_TENSOR_MAPS) || !(tile_x == 32 || tile_x == 64 || tile_x == 128) ||
      bw > 256)
    return LB_OK;
  EncodeTiled enc = encode_tiled();
  if (!enc) return LB_OK;
  const size_t n = 4 * (size_t)c->n_lat;
  if (!c->d_tmaps) {
    int rc = dev_alloc(c, &c->d_tmaps, n * sizeof(CUtensorMap));
    if (rc) return rc;
  }
  std::vector<CUtensorMap> maps(n);
  std::memset(maps.data(), 0, n * sizeof(CUtensorMap));
  for (int buf = 0; buf < 2; ++buf)
    for (int i = 0; i < c->n_lat; ++i) {
      const lb_params& p = c->params[i];
      if (p.Lx <= 2 * tile_x) continue;  // no strip away from the x edges
      const cuuint64_t dims[3] = {(cuuint64_t)p.Lx, (cuuint64_t)p.Lz, 9};
      const cuuint64_t strides[2] = {(cuuint64_t)p.Lx * es, (cuuint64_t)p.Lx * p.Lz * es};
      const cuuint32_t estr[3] = {1, 1, 1};
      for (int run = 1; run <= 2; ++run) {
        const cuuint32_t box[3] = {(cuuint32_t)bw, 1, (cuuint32_t)run};
        void* base = (char*)c->f[buf] + (size_t)c->f_off[i] * sizeof(float);
        CUresult r = enc(&maps[((size_t)buf * c->n_lat + i) * 2 + (run - 1)], CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return LB_OK;
      }
    }
  if (cudaMemcpy(c->d_tmaps, maps.data(), n * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess)
    return LB_ERR_CUDA;
  c->tma = true;
  return LB_OK;
}

int build_items(lb_ctx* c, int tile_x, int rows) {
  std::vector<WorkItem> items;
  std::vector<std::pair<int, int>> range;
  {
    std::vector<int> Lx, Lz;
    lattice_shapes(c, Lx, Lz);
    plan_items(Lx, Lz, tile_x, rows, items, range);
  }
  if ((int)items.size() > c->d_items_cap) {
    if (c->d_items) {
      dev_free(c, c->d_items);
      c->bytes -= (size_t)c->d_items_cap * sizeof(WorkItem);
    }
    int rc = dev_alloc(c, &c->d_items, items.size() * sizeof(WorkItem));
    if (rc) return rc;
    c->d_items_cap = (int)items.size();
  }
  if ((int)items.size() > c->partials_cap) {
    if (c->partials) {
      dev_free(c, c->partials);
      c->bytes -= (size_t)c->partials_cap * 3 * sizeof(double);
    }
    int rc = dev_alloc(c, &c->partials, items.size() * 3 * sizeof(double));
    if (rc) return rc;
    c->partials_cap = (int)items.size();
  }
  if (cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
    return LB_ERR_CUDA;
  int rc = build_schedule(c, items, range, tile_x, rows);
  if (rc) return rc;
  c->items = items;
  for (int i = 0; i < c->n_lat; ++i) {
    c->diag[i].item_begin = range[i].first;
    c->diag[i].item_end = range[i].second;
  }
  if (c->d_diag &&
      cudaMemcpy(c->d_diag, c->diag.data(), c->diag.size() * sizeof(DiagLattice), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return LB_ERR_CUDA;
  c->tile_x = tile_x;
  c->rows_per_item = rows;
  c->coop_grid = -1;
  drop_graphs(c);
  return build_tmaps(c, tile_x);
}

int alloc_diag(lb_ctx* c) {
  if (c->diag_ready) return LB_OK;
  const size_t rs = c->dev32 ? sizeof(float) : sizeof(double);
  int rc = dev_alloc(c, (char**)&c->fields, 4 * (size_t)c->n_sites * rs);
  if (!rc) rc = dev_alloc(c, (char**)&c->pfield, (size_t)c->n_sites * rs);
  if (!rc) rc = dev_alloc(c, &c->prof_sum, 5 * (size_t)c->n_rows * sizeof(double));
  if (!rc) rc = dev_alloc(c, &c->prof_comp, 5 * (size_t)c->n_rows * sizeof(double));
  if (!rc) rc = dev_alloc(c, &c->d_row_lat, (size_t)c->n_rows * sizeof(int));
  if (!rc) rc = dev_alloc(c, (char**)&c->tmp, 4 * (size_t)c->n_sites * 2 * rs);
  if (!rc) rc = dev_alloc(c, &c->acc_sum, 4 * (size_t)c->n_sites * sizeof(double));
  if (!rc) rc = dev_alloc(c, &c->acc_comp, 4 * (size_t)c->n_sites * sizeof(double));
  if (rc) return rc;
  c->sf_threads = sf_threads(c->max_Lx, c->max_Lz);
  c->sf_cap = 16 * c->sf_threads;
  c->sf_smem_rows = c->sf_smem_cols = 0;
  const size_t cs = 2 * rs;  // one complex point
  std::vector<int2> rt, ct;
  for (int i = 0; i < c->n_lat; ++i) {
    const int Lx = c->params[i].Lx, Lz = c->params[i].Lz;
    const int R = sf_row_group(Lx, Lz, c->sf_cap), cq = sf_col_strip(Lx, Lz, c->sf_cap);
    for (int fld = 0; fld < 4; ++fld)
      for (int z0 = 0; z0 < Lz; z0 += R) rt.push_back(make_int2(i, fld * Lz + z0));
    for (int fld = 0; fld < 4; ++fld)
      for (int q = 0; q <= Lx / 2; q += cq) ct.push_back(make_int2(i, fld * Lx + q));  // S(-q) = S(q)
    // twiddles (n/2 + 1 slots) and the sequences, as laid out by the two kernels
    c->sf_smem_rows = std::max(c->sf_smem_rows, ((size_t)(Lx / 2 + 1) + (size_t)((R + 1) / 2) * sf_seq_stride(Lx)) * cs);
    c->sf_smem_cols = std::max(c->sf_smem_cols, ((size_t)(Lz / 2 + 1) + (size_t)cq * sf_seq_stride(Lz)) * cs);
  }
  rc = dev_alloc(c, &c->d_row_tasks, rt.size() * sizeof(int2));
  if (!rc) rc = dev_alloc(c, &c->d_col_tasks, ct.size() * sizeof(int2));
  if (rc) return rc;
  if (cudaMemcpy(c->d_row_tasks, rt.data(), rt.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_col_tasks, ct.data(), ct.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
    return LB_ERR_CUDA;
  c->n_row_tasks = (int)rt.size();
  c->n_col_tasks = (int)ct.size();
  std::vector<int> row_lat(c->n_rows);
  for (int i = 0; i < c->n_lat; ++i)
    for (int z = 0; z < c->params[i].Lz; ++z) row_lat[c->row_off[i] + z] = i;
  if (cudaMemcpy(c->d_row_lat, row_lat.data(), row_lat.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->prof_sum, 0, 5 * (size_t)c->n_rows * sizeof(double)) != cudaSuccess ||
      cudaMemset(c->prof_comp, 0, 5 * (size_t)c->n_rows * sizeof(double)) != cudaSuccess)
    return LB_ERR_CUDA;
  if (cudaMemset(c->acc_sum, 0, 4 * (size_t)c->n_sites * sizeof(double)) != cudaSuccess ||
      cudaMemset(c->acc_comp, 0, 4 * (size_t)c->n_sites * sizeof(double)) != cudaSuccess)
    return LB_ERR_CUDA;
  c->diag_ready = true;
  return LB_OK;
}

bool is_sample(const lb_ctx* c, int64_t t) {
  return c->every > 0 && t >= c->discard && (t - c->discard) % c->every == 0;
}

template <class real>
StepArgs<real> step_args(lb_ctx* c, int cur, int t_offset) {
  StepArgs<real> a;
  a.lat = (const LatticeDev<real>*)c->d_lat;
  a.rows = (const RowConst<real>*)c->d_rows;
  a.items = c->d_items;
  a.n_items = (int)c->items.size();
  a.src = (const real*)c->f[cur];
  a.dst = (real*)c->f[cur ^ 1];
  a.d_t = c->d_t;
  a.t_offset = t_offset;
  a.fields = (real*)c->fields;
  a.pfield = (real*)c->pfield;
  a.partials = c->partials;
  a.err = c->d_err;
  a.tmaps = c->tma ? c->d_tmaps : nullptr;
  a.n_lat = c->n_lat;
  a.src_buf = cur;
  return a;
}

template <class real>
cudaError_t enqueue_sample(lb_ctx* c) {
  NvtxRange r("lb sample step diagnostics");
  SfPlan p;
  p.lat = c->d_diag;
  p.row_tasks = c->d_row_tasks;
  p.col_tasks = c->d_col_tasks;
  p.n_row_tasks = c->n_row_tasks;
  p.n_col_tasks = c->n_col_tasks;
  p.threads = c->sf_threads;
  p.cap = c->sf_cap;
  p.smem_rows = c->sf_smem_rows;
  p.smem_cols = c->sf_smem_cols;
  p.prof_sum = c->prof_sum;
  p.prof_comp = c->prof_comp;
  p.n_rows = c->n_rows;
  cudaError_t e = launch_sf<real>(p, (const real*)c->fields, c->tmp, c->acc_sum, c->acc_comp, c->stream);
  if (e != cudaSuccess) return e;
  e = launch_profiles<real>(c->d_diag, c->d_row_lat, c->n_rows, (const real*)c->fields, (const real*)c->pfield,
                            c->prof_sum, c->prof_comp, c->stream);
  if (e != cudaSuccess) return e;
  c->launches += 4;
  if (c->corr_mask) {
    CorrPlan cp{c->d_diag, c->d_corr_real, c->n_corr_real, c->d_corr_mode, c->n_corr_mode, c->d_corr_modes,
                (int)c->corr_modes.size()};
    e = launch_corr<real>(cp, (const real*)c->fields, c->tmp, c->corr_R, c->corr_C, c->stream);
    if (e != cudaSuccess) return e;
    c->launches += (c->n_corr_real > 0) + (c->n_corr_mode > 0);
  }
  return launch_finalize(c->d_diag, c->n_lat, c->partials, c->stats, c->stream);
}

// Enqueue `n` steps starting from buffer `cur`, with sampling by the bit mask.  Direct
// launches: one step kernel per step.
template <class real>
cudaError_t enqueue_direct(lb_ctx* c, int cur, int64_t n, const std::vector<int64_t>& sample_offsets) {
  size_t si = 0;
  for (int64_t k = 0; k < n; ++k) {
    const bool sample = si < sample_offsets.size() && sample_offsets[si] == k;
    if (sample) ++si;
    cudaError_t e = launch_step<real>(step_args<real>(c, cur, (int)k), c->tile_x, sample, c->noise_mode, c->bulk_ok, c->stream);
    if (e != cudaSuccess) return e;
    c->launches += 1;
    if (sample) {
      e = enqueue_sample<real>(c);
      if (e != cudaSuccess) return e;
    }
    cur ^= 1;
  }
  c->launches += 1;
  return launch_advance(c->d_t, n, c->stream);
}

// Persistent: one cooperative launch per run of plain steps; a sample step that ends a run is an
// ordinary launch after it (with its sampling kernels), so that the persistent kernel carries the
// plain variant only.
template <class real>
cudaError_t enqueue_persistent(lb_ctx* c, int cur, int64_t n, const std::vector<int64_t>& sample_offsets) {
  if (c->coop_grid < 0) c->coop_grid = persistent_grid<real>(c->tile_x, c->noise_mode, c->bulk_ok);
  const int grid = std::min<int>(c->coop_grid, (int)c->items.size());
  if (grid <= 0) return cudaErrorCooperativeLaunchTooLarge;
  int64_t k = 0;
  size_t si = 0;
  while (k < n) {
    int64_t end = n;  // exclusive
    bool sample = false;
    if (si < sample_offsets.size()) {
      end = sample_offsets[si] + 1;
      sample = true;
      ++si;
    }
    const int64_t plain = end - k - (sample ? 1 : 0);
    cudaError_t e;
    if (plain > 0) {
      e = cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned long long), c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->d_done, 0, c->items.size() * sizeof(unsigned), c->stream);
      if (e != cudaSuccess) return e;
      const PersistArgs pa{reinterpret_cast<unsigned long long*>(c->d_barrier), c->d_done, c->d_nbr_off, c->d_nbr,
                           c->d_err, 2000, 0};
      e = launch_step_persistent<real>(step_args<real>(c, cur, (int)k), c->tile_x, (int)plain, c->noise_mode,
                                       c->bulk_ok, pa, grid, c->stream);
      if (e != cudaSuccess) return e;
      c->launches += 1;
      if (plain & 1) cur ^= 1;
    }
    if (sample) {
      e = launch_step<real>(step_args<real>(c, cur, (int)(end - 1)), c->tile_x, true, c->noise_mode, c->bulk_ok,
                            c->stream);
      if (e != cudaSuccess) return e;
      c->launches += 1;
      e = enqueue_sample<real>(c);
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
    k = end;
  }
  c->launches += 1;
  return launch_advance(c->d_t, n, c->stream);
}

template <class real>
cudaError_t enqueue(lb_ctx* c, int cur, int64_t n, const std::vector<int64_t>& so, bool persistent) {
  return persistent ? enqueue_persistent<real>(c, cur, n, so) : enqueue_direct<real>(c, cur, n, so);
}

template <class real>
int autotune(lb_ctx* c) {
  NvtxRange r("lb autotune");
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, int, int, int, int, int>, std::pair<int, int>> cache;
  const bool persistent = c->flags & LB_PERSISTENT;
  const auto key =
      std::make_tuple(c->n_lat, c->n_sites, c->max_Lx, c->max_Lz, (int)c->dev32, c->noise_mode, (int)persistent);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return build_items(c, it->second.first, it->second.second);
  }
  const int txs[] = {32, 64, 128, 256};
  const int rows[] = {2, 4, 8, 16, 32, 64, 128, 256, 1 << 30};
  float best = 1e30f;
  int bx = c->tile_x, br = c->rows_per_item;
  std::vector<std::tuple<float, int, int>> trials;  // (ms, tile_x, rows)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tx : txs) {
    if (tx > 2 * c->max_Lx && tx > 64) continue;
    int last = -1;
    for (int r : rows) {
      const int rr = std::min(r, c->max_Lz);
      if (rr == last) continue;
      last = rr;
      if (build_items(c, tx, rr) != LB_OK) continue;
      // state is untouched: every trial reads f[cur] and writes f[cur ^ 1]; the persistent
      // launch is timed as it schedules (tickets, per-item waits) in its trial mode, in which
      // every step reads f[cur]
      const int reps = persistent ? 6 : 4;
      const int grid =
          persistent ? std::min<int>(persistent_grid<real>(tx, c->noise_mode, c->bulk_ok), (int)c->items.size()) : 0;
      auto trial = [&](int steps) {
        if (!persistent) {
          for (int k = 0; k < steps; ++k)
            launch_step<real>(step_args<real>(c, c->cur, 0), tx, false, c->noise_mode, c->bulk_ok, c->stream);
          return;
        }
        cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned long long), c->stream);
        cudaMemsetAsync(c->d_done, 0, c->items.size() * sizeof(unsigned), c->stream);
        const PersistArgs pa{reinterpret_cast<unsigned long long*>(c->d_barrier), c->d_done, c->d_nbr_off, c->d_nbr,
                             c->d_err, 2000, 1};
        launch_step_persistent<real>(step_args<real>(c, c->cur, 0), tx, steps, c->noise_mode, c->bulk_ok, pa, grid,
                                     c->stream);
      };
      if (persistent && grid <= 0) continue;
      trial(2);
      cudaEventRecord(e0, c->stream);
      trial(reps);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      trials.emplace_back(ms, tx, rr);
      best = std::min(best, ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // among the shapes within 0.5% of the fastest (timing noise), the one with the longest items
  // (fewest halo rows and items), then the fastest of those: a stable choice from run to run
  {
    float bms = 1e30f;
    int brr = -1;
    for (const auto& t : trials) {
      const float ms = std::get<0>(t);
      const int rr = std::get<2>(t);
      if (ms > best * 1.005f) continue;
      if (rr > brr || (rr == brr && ms < bms)) {
        brr = rr;
        bms = ms;
        bx = std::get<1>(t);
        br = rr;
      }
    }
  }
  {
    std::lock_guard<std::mutex> g(mu);
    cache[key] = {bx, br};
  }
  return build_items(c, bx, br);
}

template <class real>
int step_impl(lb_ctx* c, int64_t n) {
  NvtxRange r("lb_step");
  if (c->flags & LB_AUTOTUNE && !c->tuned && !c->tile_fixed) {
    int rc = autotune<real>(c);
    if (rc) return rc;
    c->tuned = true;
  }
  const bool persistent = c->flags & LB_PERSISTENT;
  const bool graph = c->flags & LB_GRAPH;
  int64_t done = 0;
  while (done < n) {
    // segment: everything left (direct launches), or what one graph holds: up to 64 per-step
    // launches, or up to 4096 steps in persistent launches
    int64_t cap = persistent ? 4096 : 64;
    if (c->every > 0 && c->every <= cap) cap -= cap % c->every;  // full segments share their sample phase
    const int64_t seg = graph ? std::min<int64_t>(n - done, cap) : (n - done);
    std::vector<int64_t> so;
    for (int64_t k = 0; k < seg; ++k)
      if (is_sample(c, c->t + done + k)) so.push_back(k);
    if (!so.empty() && !c->diag_ready) return LB_ERR_STATE;
    cudaError_t e;
    if (graph) {
      const GraphKey key{seg, so, c->cur, persistent ? 1 : 0};
      auto it = c->graphs.find(key);
      if (it == c->graphs.end()) {
        cudaGraph_t gr;
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(e);
        const int64_t before = c->launches;
        cudaError_t ee = enqueue<real>(c, c->cur, seg, so, persistent);
        const int64_t in_graph = c->launches - before;
        c->launches = before;
        e = cudaStreamEndCapture(c->stream, &gr);
        if (ee != cudaSuccess) return cuda_err(ee);
        if (e != cudaSuccess) return cuda_err(e);
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_err(e);
        if (c->graphs.size() > 32) drop_graphs(c);
        it = c->graphs.emplace(key, std::make_pair(ex, in_graph)).first;
      }
      e = cudaGraphLaunch(it->second.first, c->stream);
      c->launches += it->second.second;
    } else {
      e = enqueue<real>(c, c->cur, seg, so, persistent);
    }
    if (e != cudaSuccess) return cuda_err(e);
    c->nsamples += (int64_t)so.size();
    if (c->corr_mask) c->corr_samples += (int64_t)so.size();
    if (seg & 1) c->cur ^= 1;
    c->t += seg;
    done += seg;
  }
  return LB_OK;
}

int create_impl(lb_ctx** out, int n, const lb_params* ps, int flags, lb_alloc_fn alloc_fn = nullptr,
                lb_free_fn free_fn = nullptr, void* alloc_user = nullptr) {
  NvtxRange r("lb_create");
  if (!out) return LB_ERR_BAD_PARAM;
  *out = nullptr;
  if (n < 1 || !ps) return LB_ERR_BAD_PARAM;
  const int known = LB_PREC_DEV32 | LB_NO_ASTAR | LB_WALL_FIXED | LB_NOISE_LOC | LB_GRAPH | LB_PERSISTENT | LB_AUTOTUNE |
                    LB_NO_BULK | LB_NO_TENSOR_MAPS;
  if (flags & ~known) return LB_ERR_BAD_PARAM;
  for (int i = 0; i < n; ++i) {
    int rc = check_params(ps[i]);
    if (rc) return rc;
  }
  if (!alloc_fn != !free_fn) return LB_ERR_BAD_PARAM;
  lb_ctx* c = new (std::nothrow) lb_ctx();
  if (!c) return LB_ERR_OOM;
  c->alloc_fn = alloc_fn;
  c->free_fn = free_fn;
  c->alloc_user = alloc_user;
  c->n_lat = n;
  c->flags = flags;
  c->dev32 = flags & LB_PREC_DEV32;
  c->params.assign(ps, ps + n);
  for (int i = 0; i < n; ++i) c->site_map.emplace_back(0, ps[i].Lx);
  int64_t foff = 0, soff = 0;
  int roff = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t sites = (int64_t)ps[i].Lx * ps[i].Lz;
    c->f_off.push_back(foff);
    c->site_off.push_back(soff);
    c->row_off.push_back(roff);
    foff += 18 * sites;
    // keep every lattice's block 16-byte aligned
    foff = (foff + 3) & ~(int64_t)3;
    soff += sites;
    roff += ps[i].Lz;
    c->max_lattice_sites = std::max<int>(c->max_lattice_sites, (int)sites);
    c->max_Lx = std::max(c->max_Lx, ps[i].Lx);
    c->max_Lz = std::max(c->max_Lz, ps[i].Lz);
    if (ps[i].kT > 0) c->noise_mode = (flags & LB_NOISE_LOC) ? NOISE_LOC : NOISE_HOM;
  }
  c->n_f = foff;
  c->n_sites = soff;
  {
    const int align = 2;  // rows of pairs 16-byte aligned, and at least the two halo columns
    c->bulk_ok = !(flags & LB_NO_BULK);
    for (int i = 0; i < n; ++i)
      if (ps[i].Lx % align != 0) c->bulk_ok = false;
  }
  c->n_rows = roff;
  const size_t rs = c->dev32 ? sizeof(float) : sizeof(double);
  int rc = LB_OK;
  rc = dev_alloc(c, (char**)&c->f[0], c->n_f * rs);
  if (!rc) rc = dev_alloc(c, (char**)&c->f[1], c->n_f * rs);
  if (!rc) rc = dev_alloc(c, &c->stats, n * sizeof(DiagStats));
  if (!rc) rc = dev_alloc(c, &c->d_diag, n * sizeof(DiagLattice));
  if (!rc) rc = dev_alloc(c, &c->d_t, sizeof(int64_t));
  if (!rc) rc = dev_alloc(c, &c->d_barrier, 4 * sizeof(unsigned));
  if (!rc) rc = dev_alloc(c, &c->d_err, sizeof(int));
  if (!rc) rc = dev_alloc(c, &c->d_mass, 2 * sizeof(double));
  if (!rc && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) rc = LB_ERR_CUDA;
  c->stream = c->own_stream;
  if (!rc) rc = c->dev32 ? upload_tables<float>(c) : upload_tables<double>(c);
  if (!rc && (c->dev32 ? prepare_step<float>(256) : prepare_step<double>(256)) != cudaSuccess) rc = LB_ERR_CUDA;
  if (!rc && (cudaMemset(c->stats, 0, n * sizeof(DiagStats)) != cudaSuccess ||
              cudaMemset(c->d_t, 0, sizeof(int64_t)) != cudaSuccess ||
              cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess))
    rc = LB_ERR_CUDA;
  if (!rc) {
    // default tile: 128 columns; rows per item chosen so that the grid has a few waves, down to
    // 16 rows, or to 2 when a state buffer fits well inside L2 (32 MB): short items re-read two
    // halo rows each, which then come from L2 (on 256 x 128: 16 items of 16 rows 0.149 s per
    // 2 x 2000 steps, 128 items of 2 rows 0.132 s)
    int rows = c->max_Lz;
    const int64_t cols = [&] { int64_t s = 0; for (auto& p : c->params) s += (p.Lx + 127) / 128; return s; }();
    const int min_rows = c->n_f * rs <= ((size_t)32 << 20) ? 2 : 16;
    while (rows > min_rows && cols * ((c->max_Lz + rows - 1) / rows) < 4 * 152) rows /= 2;
    rc = build_items(c, 128, rows);
  }
  if (!rc) {
    for (int i = 0; i < n && !rc; ++i) {
      BgParams bp{ps[i].Lx, ps[i].Lz, c->dev32 ? 1 : 0, kRhoBar, ps[i].grad_c0};
      cudaError_t e = c->dev32 ? launch_init_rest<float>((float*)c->f[0] + c->f_off[i], bp, nullptr)
                               : launch_init_rest<double>((double*)c->f[0] + c->f_off[i], bp, nullptr);
      if (e != cudaSuccess) rc = cuda_err(e);
    }
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = LB_ERR_CUDA;
  }
  if (rc) {
    lb_destroy(c);
    return rc;
  }
  *out = c;
  return LB_OK;
}

int sync_and_check(lb_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return LB_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LB_ERR_CUDA;
  if (err) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return LB_ERR_TIMEOUT;
  }
  return LB_OK;
}

int lattice_ok(lb_ctx* c, int lattice) { return c && lattice >= 0 && lattice < c->n_lat; }

int ensure_scratch(lb_ctx* c) {
  if (c->d_scratch) return LB_OK;
  return dev_alloc(c, &c->d_scratch, (size_t)18 * c->max_lattice_sites * sizeof(double));
}

}  // namespace

namespace lbk {

namespace {
// Device (or managed) memory that the current device can address without peer access: memory of
// the current device, or managed memory.
bool device_pointer_here(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  if (at.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.device == dev;
}
}  // namespace

int power_spectrum_args_ok(const double* field, int Lx, int Lz, const double* out) {
  if (!field || !out || !is_pow2(Lx) || !is_pow2(Lz) || Lx < 2 || Lz < 2 || Lx > 8192 || Lz > 8192)
    return LB_ERR_BAD_PARAM;
  if (!device_pointer_here(field) || !device_pointer_here(out)) return LB_ERR_BAD_PARAM;
  return LB_OK;
}

int prepare_power_spectrum_current_device() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LB_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(mu);
  if (!done[dev]) {
    if (prepare_power_spectrum() != cudaSuccess) return LB_ERR_CUDA;
    done[dev] = true;
  }
  return LB_OK;
}

}  // namespace lbk

namespace {

// ---- adjoint sweep for the gradient of the mean-pressure shift -----------------------------
// Every lattice of the context at once: losses[i] and grads[3 i ..] per lattice (either may be
// null; grads null: the loss alone).
template <class real>
int pressure_shift_impl(lb_ctx* c, int64_t T, int64_t C, double* grads, double* losses) {
  NvtxRange r("lb_pressure_shift_gradient");
  const int n = c->n_lat;
  const size_t S = c->n_f;         // reals per state: every lattice at its f_off
  const size_t NS = c->n_sites;    // sites of the batch: every lattice at its site_off
  const int64_t nck = (T + C - 1) / C;
  const bool want_grad = grads != nullptr;
  cudaStream_t st = c->stream;
  // the adjoint's blocks, lattice by lattice, and the lattices' constants of the transposed step
  std::vector<int> first(n + 1, 0), lat_of;
  std::vector<AdjConst> kcs(n);
  bool options = false;
  for (int i = 0; i < n; ++i) {
    const int nb = adjoint_blocks(c->params[i].Lx * c->params[i].Lz);
    first[i + 1] = first[i] + nb;
    lat_of.insert(lat_of.end(), nb, i);
    kcs[i] = adjoint_constants(
        make_lattice<real>(c->params[i], c->flags, c->dev32, c->f_off[i], c->site_off[i], c->row_off[i]));
    kcs[i].w_loss = 1.0 / ((double)T * (double)(c->params[i].Lx * c->params[i].Lz));
    options = options || kcs[i].options;
  }
  const int nblk = first[n];
  std::vector<void*> owned;
  auto alloc = [&](size_t bytes) -> void* {
    void* q = ctx_malloc(c, bytes);
    if (q) owned.push_back(q);
    return q;
  };
  // the noisy run (index 0) and the noiseless run (1) are independent until their losses and
  // gradients are combined: each has its own buffers and its own stream, so that their small
  // kernels overlap on the GPU
  struct Run {
    cudaStream_t s = nullptr;
    real *ck = nullptr, *ring = nullptr, *cur = nullptr, *fields = nullptr, *pfield = nullptr;
    double *fb = nullptr, *rho = nullptr, *fl = nullptr, *sb = nullptr, *partials = nullptr, *gpart = nullptr;
    DiagStats* stats = nullptr;
    int noise = NOISE_OFF;
    double sign = 1.0;
    int fcur = 0;
  } runs[2];
  cudaStream_t s1 = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  auto release = [&]() {
    cudaStreamSynchronize(st);
    if (s1) cudaStreamSynchronize(s1);
    for (void* q : owned) dev_free(c, q);
    if (s1) cudaStreamDestroy(s1);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
  };
  bool got = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (!got) {
    release();
    return LB_ERR_CUDA;
  }
  for (int q = 0; q < 2; ++q) {
    Run& R = runs[q];
    R.s = q == 0 ? st : s1;
    R.noise = q == 0 ? c->noise_mode : NOISE_OFF;
    R.sign = q == 0 ? 1.0 : -1.0;
    R.ck = (real*)alloc(nck * S * sizeof(real));
    R.cur = (real*)alloc(2 * S * sizeof(real));
    R.fields = (real*)alloc(4 * NS * sizeof(real));
    R.pfield = (real*)alloc(NS * sizeof(real));
    R.partials = (double*)alloc((size_t)3 * c->items.size() * sizeof(double));
    R.stats = (DiagStats*)alloc((size_t)n * sizeof(DiagStats));
    got = got && R.ck && R.cur && R.fields && R.pfield && R.partials && R.stats;
    if (want_grad) {
      R.ring = (real*)alloc(C * S * sizeof(real));
      R.fb = (double*)alloc(2 * S * sizeof(double));
      R.rho = (double*)alloc(4 * NS * sizeof(double));  // two density sets
      R.fl = (double*)alloc(S * sizeof(double));
      R.sb = (double*)alloc(4 * NS * sizeof(double));
      R.gpart = (double*)alloc((size_t)3 * nblk * sizeof(double));
      got = got && R.ring && R.fb && R.rho && R.fl && R.sb && R.gpart;
    }
  }
  double* d_grad = (double*)alloc((size_t)6 * n * sizeof(double));  // per run
  int64_t* zero_t = (int64_t*)alloc(sizeof(int64_t));
  int* d_map = want_grad ? (int*)alloc((size_t)(nblk + n + 1) * sizeof(int)) : nullptr;
  AdjConst* d_kcs = want_grad ? (AdjConst*)alloc((size_t)n * sizeof(AdjConst)) : nullptr;
  if (!got || !d_grad || !zero_t || (want_grad && (!d_map || !d_kcs))) {
    release();
    return LB_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  AdjMap map{nullptr, nullptr, nblk, n};
  if (want_grad) {
    ok(cudaMemcpy(d_map, lat_of.data(), (size_t)nblk * sizeof(int), cudaMemcpyHostToDevice));
    ok(cudaMemcpy(d_map + nblk, first.data(), (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    ok(cudaMemcpy(d_kcs, kcs.data(), (size_t)n * sizeof(AdjConst), cudaMemcpyHostToDevice));
    map.lat_of = d_map;
    map.first = d_map + nblk;
  }
  ok(cudaMemsetAsync(zero_t, 0, sizeof(int64_t), st));
  ok(cudaMemsetAsync(d_grad, 0, (size_t)6 * n * sizeof(double), st));
  ok(cudaEventRecord(ev[0], st));  // the second run's stream starts after the set-up
  ok(cudaStreamWaitEvent(s1, ev[0], 0));
  auto args = [&](const Run& R, const real* src, real* dst, int64_t k) {
    StepArgs<real> a = step_args<real>(c, 0, 0);
    a.src = src;
    a.dst = dst;
    a.tmaps = nullptr;  // the context's tensor maps describe its own state buffers, not these
    a.d_t = zero_t;
    a.t_offset = (int)k;
    a.fields = R.fields;
    a.pfield = R.pfield;
    a.partials = R.partials;
    return a;
  };
  // forward runs from rest, step by step in both streams: checkpoints f*_{c-1} before every C-th
  // step, pressure of every step
  {
    NvtxRange rr("lb adjoint: forward runs");
    for (Run& R : runs) {
      if (want_grad) ok(cudaMemsetAsync(R.gpart, 0, (size_t)3 * nblk * sizeof(double), R.s));
      for (int i = 0; i < n; ++i) {
        const lb_params& p = c->params[i];
        const BgParams bp{p.Lx, p.Lz, c->dev32 ? 1 : 0, kRhoBar, p.grad_c0};
        ok(launch_init_rest<real>(R.cur + c->f_off[i], bp, R.s));
      }
      ok(cudaMemsetAsync(R.stats, 0, (size_t)n * sizeof(DiagStats), R.s));
    }
    for (int64_t k = 0; k < T && e == cudaSuccess; ++k)
      for (Run& R : runs) {
        real* src = R.cur + (k & 1) * S;
        real* dst = R.cur + ((k + 1) & 1) * S;
        if (k % C == 0)
          ok(cudaMemcpyAsync(R.ck + (k / C) * S, src, S * sizeof(real), cudaMemcpyDeviceToDevice, R.s));
        ok(launch_step<real>(args(R, src, dst, k), c->tile_x, true, R.noise, c->bulk_ok, R.s));
        ok(launch_finalize(c->d_diag, n, R.partials, R.stats, R.s));
      }
  }
  // reverse sweeps, one checkpoint segment at a time in both streams; a run's sign (+ noisy,
  // - noiseless) enters through the loss weight alpha = sign / (T N) of each lattice, to which the
  // whole sweep is linear
  if (want_grad && e == cudaSuccess) {
    NvtxRange rr("lb adjoint: reverse sweeps");
    for (Run& R : runs) ok(cudaMemsetAsync(R.fb, 0, S * sizeof(double), R.s));
    for (int64_t seg = nck - 1; seg >= 0 && e == cudaSuccess; --seg) {
      const int64_t c0 = seg * C, len = std::min<int64_t>(C, T - c0);
      for (Run& R : runs) {
        ok(cudaMemcpyAsync(R.ring, R.ck + seg * S, S * sizeof(real), cudaMemcpyDeviceToDevice, R.s));
        for (int64_t i = 1; i < len; ++i)
          ok(launch_step<real>(args(R, R.ring + (i - 1) * S, R.ring + i * S, c0 + i - 1), c->tile_x, false, R.noise,
                               c->bulk_ok, R.s));
      }
      // the densities of each step's state come with the previous step's gather (within a
      // segment; at its top they are computed on their own)
      int rcur = 0;
      for (int64_t k = c0 + len - 1; k >= c0 && e == cudaSuccess; --k) {
        for (Run& R : runs) {
          double* rho_k = R.rho + (size_t)rcur * 2 * NS;
          double* rho_n = R.rho + (size_t)(1 - rcur) * 2 * NS;
          ok(launch_adjoint_step<real>(R.ring + (k - c0) * S, k > c0 ? R.ring + (k - 1 - c0) * S : nullptr,
                                       R.fb + R.fcur * S, R.fb + (1 - R.fcur) * S, (const LatticeDev<real>*)c->d_lat,
                                       (const RowConst<real>*)c->d_rows, d_kcs, options, map, (uint32_t)k,
                                       R.noise != NOISE_OFF, R.sign, k < c0 + len - 1, rho_k, rho_n, R.fl, R.sb,
                                       R.gpart, R.s));
          R.fcur = 1 - R.fcur;
        }
        rcur = 1 - rcur;
      }
    }
    for (int q = 0; q < 2 && e == cudaSuccess; ++q)
      ok(launch_adjoint_gradient(runs[q].gpart, map, d_grad + (size_t)3 * n * q, runs[q].s));
  }
  // join the second stream, then read the results
  ok(cudaEventRecord(ev[1], s1));
  ok(cudaStreamWaitEvent(st, ev[1], 0));
  std::vector<DiagStats> hs(2 * (size_t)n);
  std::vector<double> hg(6 * (size_t)n, 0.0);
  ok(cudaMemcpyAsync(hs.data(), runs[0].stats, (size_t)n * sizeof(DiagStats), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(hs.data() + n, runs[1].stats, (size_t)n * sizeof(DiagStats), cudaMemcpyDeviceToHost, st));
  if (want_grad) ok(cudaMemcpyAsync(hg.data(), d_grad, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  release();
  if (e != cudaSuccess) return cuda_err(e);
  for (const DiagStats& x : hs)
    if (x.nonfinite) return LB_ERR_NONFINITE;
  for (int i = 0; i < n; ++i) {
    if (losses) losses[i] = (hs[i].P_sum + hs[i].P_comp) / (double)T - (hs[n + i].P_sum + hs[n + i].P_comp) / (double)T;
    if (want_grad)
      for (int k = 0; k < 3; ++k) grads[3 * i + k] = hg[3 * i + k] + hg[(size_t)3 * n + 3 * i + k];
  }
  int err = 0;
  if (cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && err) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return LB_ERR_TIMEOUT;
  }
  return LB_OK;
}

int pressure_shift_checked(lb_ctx* c, int64_t steps, int64_t ckpt_every, double* grads, double* losses) {
  if (!c || steps < 1 || ckpt_every < 1 || ckpt_every > steps) return LB_ERR_BAD_PARAM;
  for (int i = 0; i < c->n_lat; ++i)
    if (c->site_map[i] != std::make_pair(0, c->params[i].Lx)) return LB_ERR_STATE;
  if (steps >= ((int64_t)1 << 31)) return LB_ERR_BAD_PARAM;
  int rc = sync_and_check(c);
  if (rc) return rc;
  return c->dev32 ? pressure_shift_impl<float>(c, steps, ckpt_every, grads, losses)
                  : pressure_shift_impl<double>(c, steps, ckpt_every, grads, losses);
}

}  // namespace

extern "C" {

int lb_pressure_shift_gradient(lb_ctx* c, int64_t steps, int64_t ckpt_every, double grad[3], double* loss) {
  if (c && c->n_lat != 1) return LB_ERR_STATE;
  return pressure_shift_checked(c, steps, ckpt_every, grad, loss);
}

int lb_pressure_shift_gradient_batch(lb_ctx* c, int64_t steps, int64_t ckpt_every, double* grads, double* losses) {
  return pressure_shift_checked(c, steps, ckpt_every, grads, losses);
}

int lb_create(lb_ctx** out, int Lx, int Lz, double lambda_s, double lambda_d, double lambda_e, double lambda_q,
              double lambda_eps, double kT, double G, double grad_c0, uint64_t seed, int flags) {
  lb_params p;
  std::memset(&p, 0, sizeof(p));
  p.Lx = Lx;
  p.Lz = Lz;
  p.lambda_s = lambda_s;
  p.lambda_d = lambda_d;
  p.lambda_e = lambda_e;
  p.lambda_q = lambda_q;
  p.lambda_eps = lambda_eps;
  p.kT = kT;
  p.G = G;
  p.grad_c0 = grad_c0;
  p.seed = seed;
  p.lattice_id = 0;
  return create_impl(out, 1, &p, flags);
}

int lb_create_batch(lb_ctx** out, int n, const lb_params* params, int flags) {
  return create_impl(out, n, params, flags);
}

int lb_create_batch_with_allocator(lb_ctx** out, int n, const lb_params* params, int flags, lb_alloc_fn alloc_fn,
                                   lb_free_fn free_fn, void* user) {
  if (!alloc_fn || !free_fn) {
    if (out) *out = nullptr;
    return LB_ERR_BAD_PARAM;
  }
  return create_impl(out, n, params, flags, alloc_fn, free_fn, user);
}

int lb_set_stream(lb_ctx* c, void* stream) {
  if (!c) return LB_ERR_BAD_PARAM;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->own_stream;
  if (c->stream != s) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LB_ERR_CUDA;
    drop_graphs(c);
  }
  c->stream = s;
  return LB_OK;
}

int lb_set_sampling(lb_ctx* c, int64_t discard, int64_t every) {
  if (!c || discard < 0 || every < 0) return LB_ERR_BAD_PARAM;
  if (every > 0) {
    for (auto& p : c->params)
      if (!is_pow2(p.Lx) || !is_pow2(p.Lz) || p.Lx < 2 || p.Lx > 8192 || p.Lz > 8192) return LB_ERR_BAD_PARAM;
    int rc = alloc_diag(c);
    if (rc) return rc;
    cudaError_t e = c->dev32 ? prepare_sf<float>(c->sf_smem_rows, c->sf_smem_cols)
                             : prepare_sf<double>(c->sf_smem_rows, c->sf_smem_cols);
    if (e != cudaSuccess) return cuda_err(e);
  }
  c->discard = discard;
  c->every = every;
  drop_graphs(c);
  return LB_OK;
}

int lb_set_tile(lb_ctx* c, int tile_x, int rows_per_item) {
  if (!c) return LB_ERR_BAD_PARAM;
  if (!(tile_x == 32 || tile_x == 64 || tile_x == 128 || tile_x == 256) || rows_per_item < 1)
    return LB_ERR_BAD_PARAM;
  int rc = build_items(c, tile_x, std::min(rows_per_item, c->max_Lz));
  if (rc) return rc;
  c->tile_fixed = true;
  return LB_OK;
}

int lb_get_tile(lb_ctx* c, int* tile_x, int* rows_per_item) {
  if (!c) return LB_ERR_BAD_PARAM;
  if (tile_x) *tile_x = c->tile_x;
  if (rows_per_item) *rows_per_item = c->rows_per_item;
  return LB_OK;
}

int lb_step(lb_ctx* c, int64_t n) {
  if (!c || n < 0) return LB_ERR_BAD_PARAM;
  if (n == 0) return LB_OK;
  return c->dev32 ? step_impl<float>(c, n) : step_impl<double>(c, n);
}

int lb_synchronize(lb_ctx* c) {
  if (!c) return LB_ERR_BAD_PARAM;
  return sync_and_check(c);
}

int lb_time(lb_ctx* c, int64_t* t) {
  if (!c || !t) return LB_ERR_BAD_PARAM;
  *t = c->t;
  return LB_OK;
}

int lb_num_lattices(lb_ctx* c, int* n) {
  if (!c || !n) return LB_ERR_BAD_PARAM;
  *n = c->n_lat;
  return LB_OK;
}

int lb_lattice_shape(lb_ctx* c, int lattice, int* Lx, int* Lz) {
  if (!lattice_ok(c, lattice)) return LB_ERR_BAD_PARAM;
  if (Lx) *Lx = c->params[lattice].Lx;
  if (Lz) *Lz = c->params[lattice].Lz;
  return LB_OK;
}

int lb_structure_factor(lb_ctx* c, int lattice, int field, int mode, double* out, size_t n_out,
                        int64_t* n_samples) {
  if (!lattice_ok(c, lattice) || field < 0 || field > 3 || !out || (mode != LB_SF_QXQZ && mode != LB_SF_QX))
    return LB_ERR_BAD_PARAM;
  const int Lx = c->params[lattice].Lx, Lz = c->params[lattice].Lz;
  const size_t need = mode == LB_SF_QXQZ ? (size_t)Lx * Lz : (size_t)Lx;
  if (n_out != need) return LB_ERR_SIZE;
  int rc = sync_and_check(c);
  if (rc) return rc;
  if (n_samples) *n_samples = c->nsamples;
  if (!c->diag_ready || c->nsamples == 0) {
    std::fill(out, out + need, 0.0);
    return LB_OK;
  }
  const size_t full = (size_t)Lx * Lz;
  const size_t off = 4 * (size_t)c->site_off[lattice] + (size_t)field * full;
  // LB_SF_QX needs the q_z = 0 row only (q_x > Lx/2 comes from row 0 as well)
  const size_t ncopy = mode == LB_SF_QXQZ ? full : (size_t)Lx;
  std::vector<double> s(ncopy), k(ncopy);
  if (cudaMemcpy(s.data(), c->acc_sum + off, ncopy * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(k.data(), c->acc_comp + off, ncopy * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LB_ERR_CUDA;
  // accumulated: q_x = 0 .. Lx/2 (Kahan sums: total = sum - comp); the rest by S(q) = S(-q)
  const double inv = 1.0 / (double)c->nsamples;
  const int rows_out = mode == LB_SF_QXQZ ? Lz : 1;
  for (int n = 0; n < rows_out; ++n)
    for (int q = 0; q < Lx; ++q) {
      const int nn = q <= Lx / 2 ? n : (Lz - n) % Lz;
      const int qq = q <= Lx / 2 ? q : Lx - q;
      const size_t src = (size_t)nn * Lx + qq;
      out[(size_t)n * Lx + q] = (s[src] - k[src]) * inv;
    }
  return LB_OK;
}

namespace {
void corr_free(lb_ctx* c) {
  void* ptrs[] = {c->corr_R, c->corr_C, c->d_corr_real, c->d_corr_mode, c->d_corr_modes};
  for (void* p : ptrs) dev_free(c, p);
  c->bytes -= (c->corr_R_n + c->corr_C_n) * sizeof(double) +
              ((size_t)c->n_corr_real + (size_t)c->n_corr_mode) * sizeof(int4) + c->corr_modes.size() * sizeof(int);
  c->corr_R = c->corr_C = nullptr;
  c->d_corr_real = c->d_corr_mode = nullptr;
  c->d_corr_modes = nullptr;
  c->corr_R_n = c->corr_C_n = 0;
  c->n_corr_real = c->n_corr_mode = 0;
  c->corr_modes.clear();
  c->corr_mask = 0;
  c->corr_samples = 0;
}
}  // namespace

int lb_set_correlations(lb_ctx* c, int field_mask, int n_modes, const int* modes) {
  if (!c || field_mask < 0 || field_mask > 15 || n_modes < 0 || n_modes > LB_CORR_MAX_MODES ||
      (n_modes > 0 && !modes))
    return LB_ERR_BAD_PARAM;
  for (int m = 0; m < n_modes; ++m)
    for (const lb_params& p : c->params)
      if (modes[m] < 0 || modes[m] >= p.Lx) return LB_ERR_BAD_PARAM;
  int rc = sync_and_check(c);
  if (rc) return rc;
  drop_graphs(c);
  corr_free(c);
  if (field_mask == 0) return LB_OK;
  for (const lb_params& p : c->params)
    if (!is_pow2(p.Lx) || !is_pow2(p.Lz) || p.Lx < 2 || p.Lx > 8192 || p.Lz > 8192) return LB_ERR_BAD_PARAM;
  rc = alloc_diag(c);
  if (rc) return rc;
  // offsets and tiles
  std::vector<int4> rt, mt;
  size_t rn = 0, cn = 0;
  for (int i = 0; i < c->n_lat; ++i) {
    const int Lz = c->params[i].Lz, nt = (Lz + CORR_TILE - 1) / CORR_TILE;
    c->diag[i].r_off = (int64_t)rn;
    c->diag[i].c_off = (int64_t)cn;
    rn += 4 * (size_t)Lz * Lz;
    cn += 4 * (size_t)n_modes * Lz * Lz * 2;
    for (int f = 0; f < 4; ++f) {
      if (!(field_mask & (1 << f))) continue;
      for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
          rt.push_back(make_int4(i, f, a, b));
          for (int m = 0; m < n_modes; ++m) mt.push_back(make_int4(i, f * n_modes + m, a, b));
        }
    }
  }
  // each size is recorded once its buffer exists, so that corr_free releases exactly those
  rc = dev_alloc(c, &c->corr_R, rn * sizeof(double));
  if (!rc) c->corr_R_n = rn;
  if (!rc && cn) rc = dev_alloc(c, &c->corr_C, cn * sizeof(double));
  if (!rc) c->corr_C_n = cn;
  if (!rc) rc = dev_alloc(c, &c->d_corr_real, rt.size() * sizeof(int4));
  if (!rc) c->n_corr_real = (int)rt.size();
  if (!rc && !mt.empty()) rc = dev_alloc(c, &c->d_corr_mode, mt.size() * sizeof(int4));
  if (!rc) c->n_corr_mode = (int)mt.size();
  if (!rc && n_modes) rc = dev_alloc(c, &c->d_corr_modes, (size_t)n_modes * sizeof(int));
  if (!rc) c->corr_modes.assign(modes, modes + n_modes);
  if (rc) {
    corr_free(c);
    return rc;
  }
  if (cudaMemset(c->corr_R, 0, rn * sizeof(double)) != cudaSuccess ||
      (cn && cudaMemset(c->corr_C, 0, cn * sizeof(double)) != cudaSuccess) ||
      cudaMemcpy(c->d_corr_real, rt.data(), rt.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!mt.empty() &&
       cudaMemcpy(c->d_corr_mode, mt.data(), mt.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (n_modes && cudaMemcpy(c->d_corr_modes, modes, (size_t)n_modes * sizeof(int), cudaMemcpyHostToDevice) !=
                      cudaSuccess) ||
      cudaMemcpy(c->d_diag, c->diag.data(), c->diag.size() * sizeof(DiagLattice), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    corr_free(c);
    return LB_ERR_CUDA;
  }
  c->corr_mask = field_mask;
  return LB_OK;
}

int lb_correlation(lb_ctx* c, int lattice, int field, double* out, size_t n_out, int64_t* n_samples) {
  if (!lattice_ok(c, lattice) || field < 0 || field > 3 || !out) return LB_ERR_BAD_PARAM;
  const int Lz = c->params[lattice].Lz;
  const size_t LL = (size_t)Lz * Lz;
  if (n_out != LL) return LB_ERR_SIZE;
  if (!(c->corr_mask & (1 << field))) return LB_ERR_STATE;
  int rc = sync_and_check(c);
  if (rc) return rc;
  if (n_samples) *n_samples = c->corr_samples;
  if (c->corr_samples == 0) {
    std::fill(out, out + LL, 0.0);
    return LB_OK;
  }
  if (cudaMemcpy(out, c->corr_R + c->diag[lattice].r_off + (size_t)field * LL, LL * sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return LB_ERR_CUDA;
  const double inv = 1.0 / (double)c->corr_samples;
  for (size_t i = 0; i < LL; ++i) out[i] *= inv;
  return LB_OK;
}

int lb_mode_correlation(lb_ctx* c, int lattice, int field, int mode_index, double* out, size_t n_out,
                        int64_t* n_samples) {
  if (!lattice_ok(c, lattice) || field < 0 || field > 3 || !out || mode_index < 0 ||
      mode_index >= (int)c->corr_modes.size())
    return LB_ERR_BAD_PARAM;
  const int Lz = c->params[lattice].Lz;
  const size_t LL = (size_t)Lz * Lz, nm = c->corr_modes.size();
  if (n_out != 2 * LL) return LB_ERR_SIZE;
  if (!(c->corr_mask & (1 << field))) return LB_ERR_STATE;
  int rc = sync_and_check(c);
  if (rc) return rc;
  if (n_samples) *n_samples = c->corr_samples;
  if (c->corr_samples == 0) {
    std::fill(out, out + 2 * LL, 0.0);
    return LB_OK;
  }
  const size_t off = c->diag[lattice].c_off + (((size_t)field * nm + mode_index) * LL) * 2;
  if (cudaMemcpy(out, c->corr_C + off, 2 * LL * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LB_ERR_CUDA;
  const double inv = 1.0 / (double)c->corr_samples;
  for (size_t i = 0; i < 2 * LL; ++i) out[i] *= inv;
  return LB_OK;
}

int lb_profile(lb_ctx* c, int lattice, int field, double* out, size_t n_out, int64_t* n_samples) {
  if (!lattice_ok(c, lattice) || field < 0 || field > LB_FIELD_P || !out) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  if (n_out != (size_t)p.Lz) return LB_ERR_SIZE;
  int rc = sync_and_check(c);
  if (rc) return rc;
  if (n_samples) *n_samples = c->nsamples;
  if (!c->diag_ready || c->nsamples == 0) {
    std::fill(out, out + p.Lz, 0.0);
    return LB_OK;
  }
  const size_t off = (size_t)field * c->n_rows + c->row_off[lattice];
  std::vector<double> s(p.Lz), k(p.Lz);
  if (cudaMemcpy(s.data(), c->prof_sum + off, p.Lz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(k.data(), c->prof_comp + off, p.Lz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LB_ERR_CUDA;
  // the accumulated row means are of deviations: add rho_bar, c_0(z) or the row's background
  // pressure (zero in FP64 mode) back
  const std::vector<RowD> rd = make_rows(p, c->flags, c->dev32);
  const double inv = 1.0 / (double)c->nsamples;
  for (int z = 0; z < p.Lz; ++z) {
    double v = (s[z] + k[z]) * inv;
    if (field == LB_FIELD_RHO) v += kRhoBar;
    else if (field == LB_FIELD_C) v += rd[z].c0;
    else if (field == LB_FIELD_P) v += rd[z].Pbg;
    out[z] = v;
  }
  return LB_OK;
}

int lb_mean_pressure(lb_ctx* c, int lattice, double* last, double* time_avg) {
  if (!lattice_ok(c, lattice)) return LB_ERR_BAD_PARAM;
  int rc = sync_and_check(c);
  if (rc) return rc;
  DiagStats st;
  if (cudaMemcpy(&st, c->stats + lattice, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return LB_ERR_CUDA;
  if (st.nonfinite) return LB_ERR_NONFINITE;
  if (last) *last = st.P_last;
  if (time_avg) *time_avg = c->nsamples ? (st.P_sum + st.P_comp) / (double)c->nsamples : 0.0;
  return LB_OK;
}

int lb_mass(lb_ctx* c, int lattice, double out[2]) {
  if (!lattice_ok(c, lattice) || !out) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  BgParams bp{p.Lx, p.Lz, c->dev32 ? 1 : 0, kRhoBar, p.grad_c0};
  cudaError_t e = c->dev32 ? launch_mass<float>((const float*)c->f[c->cur] + c->f_off[lattice], bp, c->d_mass, c->stream)
                           : launch_mass<double>((const double*)c->f[c->cur] + c->f_off[lattice], bp, c->d_mass,
                                                 c->stream);
  if (e != cudaSuccess) return cuda_err(e);
  int rc = sync_and_check(c);
  if (rc) return rc;
  if (cudaMemcpy(out, c->d_mass, 2 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return LB_ERR_CUDA;
  return LB_OK;
}

int lb_get_populations(lb_ctx* c, int lattice, double* out, size_t n) {
  if (!lattice_ok(c, lattice) || !out) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  if (n != (size_t)18 * p.Lx * p.Lz) return LB_ERR_SIZE;
  int rc = ensure_scratch(c);
  if (rc) return rc;
  BgParams bp{p.Lx, p.Lz, c->dev32 ? 1 : 0, kRhoBar, p.grad_c0};
  cudaError_t e = c->dev32 ? launch_to_absolute<float>((const float*)c->f[c->cur] + c->f_off[lattice], bp,
                                                       c->d_scratch, c->stream)
                           : launch_to_absolute<double>((const double*)c->f[c->cur] + c->f_off[lattice], bp,
                                                        c->d_scratch, c->stream);
  if (e != cudaSuccess) return cuda_err(e);
  rc = sync_and_check(c);
  if (rc) return rc;
  if (cudaMemcpy(out, c->d_scratch, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return LB_ERR_CUDA;
  return LB_OK;
}

int lb_set_populations(lb_ctx* c, int lattice, const double* in, size_t n) {
  if (!lattice_ok(c, lattice) || !in) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  if (n != (size_t)18 * p.Lx * p.Lz) return LB_ERR_SIZE;
  int rc = ensure_scratch(c);
  if (rc) return rc;
  rc = sync_and_check(c);
  if (rc) return rc;
  if (cudaMemcpy(c->d_scratch, in, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return LB_ERR_CUDA;
  BgParams bp{p.Lx, p.Lz, c->dev32 ? 1 : 0, kRhoBar, p.grad_c0};
  cudaError_t e = c->dev32 ? launch_from_absolute<float>(c->d_scratch, bp, (float*)c->f[c->cur] + c->f_off[lattice],
                                                         c->stream)
                           : launch_from_absolute<double>(c->d_scratch, bp,
                                                          (double*)c->f[c->cur] + c->f_off[lattice], c->stream);
  if (e != cudaSuccess) return cuda_err(e);
  return sync_and_check(c);
}

int lb_set_site_map(lb_ctx* c, int lattice, int x0, int Lx_global) {
  if (!lattice_ok(c, lattice)) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  if (Lx_global < p.Lx || x0 < 0 || x0 >= Lx_global || (int64_t)Lx_global * p.Lz >= ((int64_t)1 << 31))
    return LB_ERR_BAD_PARAM;
  int rc = sync_and_check(c);
  if (rc) return rc;
  c->site_map[lattice] = {x0, Lx_global};
  // the lattice's device constants, rebuilt with the new map (graphs read them at run time)
  if (c->dev32) {
    LatticeDev<float> L = make_lattice<float>(p, c->flags, true, c->f_off[lattice], c->site_off[lattice],
                                              c->row_off[lattice]);
    L.site_x0 = x0;
    L.site_Lx = Lx_global;
    if (cudaMemcpy((LatticeDev<float>*)c->d_lat + lattice, &L, sizeof(L), cudaMemcpyHostToDevice) != cudaSuccess)
      return LB_ERR_CUDA;
  } else {
    LatticeDev<double> L = make_lattice<double>(p, c->flags, false, c->f_off[lattice], c->site_off[lattice],
                                                c->row_off[lattice]);
    L.site_x0 = x0;
    L.site_Lx = Lx_global;
    if (cudaMemcpy((LatticeDev<double>*)c->d_lat + lattice, &L, sizeof(L), cudaMemcpyHostToDevice) != cudaSuccess)
      return LB_ERR_CUDA;
  }
  return LB_OK;
}

namespace {
int columns_impl(lb_ctx* c, int lattice, int x_first, int n_cols, void* buf, bool export_) {
  if (!lattice_ok(c, lattice) || !buf) return LB_ERR_BAD_PARAM;
  const lb_params& p = c->params[lattice];
  if (n_cols < 1 || x_first < 0 || x_first > p.Lx - n_cols) return LB_ERR_BAD_PARAM;
  cudaPointerAttributes at;
  int dev = -1;
  if (cudaPointerGetAttributes(&at, buf) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LB_ERR_BAD_PARAM;
  }
  if (!(at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev)))
    return LB_ERR_BAD_PARAM;
  cudaError_t e = c->dev32 ? launch_columns<float>((float*)c->f[c->cur] + c->f_off[lattice], p.Lx, p.Lz, x_first,
                                                   n_cols, (float*)buf, export_, c->stream)
                           : launch_columns<double>((double*)c->f[c->cur] + c->f_off[lattice], p.Lx, p.Lz, x_first,
                                                    n_cols, (double*)buf, export_, c->stream);
  return cuda_err(e);
}
}  // namespace

int lb_export_columns(lb_ctx* c, int lattice, int x_first, int n_cols, void* device_out) {
  return columns_impl(c, lattice, x_first, n_cols, device_out, true);
}

int lb_import_columns(lb_ctx* c, int lattice, int x_first, int n_cols, const void* device_in) {
  return columns_impl(c, lattice, x_first, n_cols, const_cast<void*>(device_in), false);
}

namespace {
// ---- checkpoint / resume -------------------------------------------------------------------
// Layout of a checkpoint (host memory, native byte order): the header, then per lattice its site
// map (x0, Lx of the whole lattice), the stored state of every lattice (n_f values of the storage
// type), the per-lattice statistics, and, when the diagnostics are allocated, the structure-factor
// and profile accumulators (sums and compensations), then the correlation accumulators if any.
constexpr uint64_t kCkptMagic = 0x3130545043424c4cull;  // "LLBCKPT01" without the first L
constexpr uint32_t kCkptVersion = 2;  // 2: the state as (A, B) pairs
constexpr int kResultFlags = LB_PREC_DEV32 | LB_NO_ASTAR | LB_WALL_FIXED | LB_NOISE_LOC;

struct CkptHeader {
  uint64_t magic;
  uint32_t version, n_lat;
  int32_t flags, corr_mask;
  int64_t t, discard, every, nsamples, corr_samples;
  int32_t n_modes, diag_ready;
  int32_t modes[LB_CORR_MAX_MODES];
  uint64_t params_hash;
  uint64_t bytes;
};

// FNV-1a over the lattices' parameters (sizes, rates, kT, G, gradient, seeds, ids)
uint64_t params_hash(const lb_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* b = reinterpret_cast<const unsigned char*>(c->params.data());
  for (size_t i = 0; i < c->params.size() * sizeof(lb_params); ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

size_t state_bytes(const lb_ctx* c) { return (size_t)c->n_f * (c->dev32 ? sizeof(float) : sizeof(double)); }

size_t ckpt_bytes(const lb_ctx* c, bool diag_ready, bool corr) {
  size_t n = sizeof(CkptHeader) + (size_t)c->n_lat * 2 * sizeof(int32_t) + state_bytes(c) +
             (size_t)c->n_lat * sizeof(DiagStats);
  if (diag_ready) n += (2 * 4 * (size_t)c->n_sites + 2 * 5 * (size_t)c->n_rows) * sizeof(double);
  if (corr) n += (c->corr_R_n + c->corr_C_n) * sizeof(double);
  return n;
}
}  // namespace

int lb_checkpoint_bytes(lb_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LB_ERR_BAD_PARAM;
  *bytes = ckpt_bytes(c, c->diag_ready, c->corr_mask != 0);
  return LB_OK;
}

int lb_save_checkpoint(lb_ctx* c, void* host_buf, size_t bytes) {
  if (!c || !host_buf) return LB_ERR_BAD_PARAM;
  const bool corr = c->corr_mask != 0;
  const size_t need = ckpt_bytes(c, c->diag_ready, corr);
  if (bytes != need) return LB_ERR_SIZE;
  int rc = sync_and_check(c);
  if (rc) return rc;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kCkptMagic;
  h.version = kCkptVersion;
  h.n_lat = (uint32_t)c->n_lat;
  h.flags = c->flags & kResultFlags;
  h.corr_mask = c->corr_mask;
  h.t = c->t;
  h.discard = c->discard;
  h.every = c->every;
  h.nsamples = c->nsamples;
  h.corr_samples = c->corr_samples;
  h.n_modes = (int32_t)c->corr_modes.size();
  h.diag_ready = c->diag_ready ? 1 : 0;
  for (int m = 0; m < h.n_modes; ++m) h.modes[m] = c->corr_modes[m];
  h.params_hash = params_hash(c);
  h.bytes = need;
  char* p = static_cast<char*>(host_buf);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (int i = 0; i < c->n_lat; ++i) {
    const int32_t m[2] = {c->site_map[i].first, c->site_map[i].second};
    std::memcpy(p, m, sizeof(m));
    p += sizeof(m);
  }
  auto from_device = [&](const void* d, size_t n) {
    if (cudaMemcpy(p, d, n, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    p += n;
    return true;
  };
  bool ok = from_device(c->f[c->cur], state_bytes(c)) && from_device(c->stats, (size_t)c->n_lat * sizeof(DiagStats));
  if (ok && c->diag_ready) {
    const size_t ns = 4 * (size_t)c->n_sites * sizeof(double), nr = 5 * (size_t)c->n_rows * sizeof(double);
    ok = from_device(c->acc_sum, ns) && from_device(c->acc_comp, ns) && from_device(c->prof_sum, nr) &&
         from_device(c->prof_comp, nr);
  }
  if (ok && corr) ok = from_device(c->corr_R, c->corr_R_n * sizeof(double)) &&
                       (c->corr_C_n == 0 || from_device(c->corr_C, c->corr_C_n * sizeof(double)));
  return ok ? LB_OK : LB_ERR_CUDA;
}

int lb_load_checkpoint(lb_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf || bytes < sizeof(CkptHeader)) return LB_ERR_BAD_PARAM;
  CkptHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kCkptMagic || h.version != kCkptVersion || h.bytes != bytes || h.n_modes < 0 ||
      h.n_modes > LB_CORR_MAX_MODES)
    return LB_ERR_BAD_PARAM;
  if ((int)h.n_lat != c->n_lat || h.flags != (c->flags & kResultFlags) || h.params_hash != params_hash(c))
    return LB_ERR_STATE;
  // start from cleared statistics (a context that sampled before keeps no stale sums), then the
  // same sampling and correlations (this allocates what the checkpoint needs)
  int rc = lb_reset_statistics(c);
  if (rc) return rc;
  rc = lb_set_sampling(c, h.discard, h.every);
  if (!rc && h.diag_ready && !c->diag_ready) rc = alloc_diag(c);
  if (!rc) rc = lb_set_correlations(c, h.corr_mask, h.n_modes, h.modes);
  if (rc) return rc;
  if (ckpt_bytes(c, h.diag_ready != 0, h.corr_mask != 0) != bytes) return LB_ERR_SIZE;
  const char* p = static_cast<const char*>(host_buf) + sizeof(h);
  for (int i = 0; i < c->n_lat; ++i) {
    int32_t m[2];
    std::memcpy(m, p, sizeof(m));
    p += sizeof(m);
    if (m[0] != c->site_map[i].first || m[1] != c->site_map[i].second) {
      rc = lb_set_site_map(c, i, m[0], m[1]);
      if (rc) return rc;
    }
  }
  auto to_device = [&](void* d, size_t n) {
    if (cudaMemcpy(d, p, n, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    p += n;
    return true;
  };
  c->cur = 0;
  bool ok = to_device(c->f[0], state_bytes(c)) && to_device(c->stats, (size_t)c->n_lat * sizeof(DiagStats));
  if (ok && h.diag_ready) {
    const size_t ns = 4 * (size_t)c->n_sites * sizeof(double), nr = 5 * (size_t)c->n_rows * sizeof(double);
    ok = to_device(c->acc_sum, ns) && to_device(c->acc_comp, ns) && to_device(c->prof_sum, nr) &&
         to_device(c->prof_comp, nr);
  }
  if (ok && h.corr_mask) ok = to_device(c->corr_R, c->corr_R_n * sizeof(double)) &&
                              (c->corr_C_n == 0 || to_device(c->corr_C, c->corr_C_n * sizeof(double)));
  // the step count, on the host and in the device counter that keys the noise
  if (ok) ok = cudaMemcpy(c->d_t, &h.t, sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) return LB_ERR_CUDA;
  c->t = h.t;
  c->nsamples = h.nsamples;
  c->corr_samples = h.corr_samples;
  drop_graphs(c);
  return LB_OK;
}

int lb_reset_statistics(lb_ctx* c) {
  if (!c) return LB_ERR_BAD_PARAM;
  int rc = sync_and_check(c);
  if (rc) return rc;
  c->nsamples = 0;
  if (cudaMemset(c->stats, 0, c->n_lat * sizeof(DiagStats)) != cudaSuccess) return LB_ERR_CUDA;
  if (c->diag_ready) {
    if (cudaMemset(c->acc_sum, 0, 4 * (size_t)c->n_sites * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->acc_comp, 0, 4 * (size_t)c->n_sites * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->prof_sum, 0, 5 * (size_t)c->n_rows * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->prof_comp, 0, 5 * (size_t)c->n_rows * sizeof(double)) != cudaSuccess)
      return LB_ERR_CUDA;
  }
  c->corr_samples = 0;
  if ((c->corr_R && cudaMemset(c->corr_R, 0, c->corr_R_n * sizeof(double)) != cudaSuccess) ||
      (c->corr_C && cudaMemset(c->corr_C, 0, c->corr_C_n * sizeof(double)) != cudaSuccess))
    return LB_ERR_CUDA;
  return LB_OK;
}

int lb_kernel_launches(lb_ctx* c, int64_t* n) {
  if (!c || !n) return LB_ERR_BAD_PARAM;
  *n = c->launches;
  return LB_OK;
}

int lb_device_bytes(lb_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LB_ERR_BAD_PARAM;
  *bytes = c->bytes;
  return LB_OK;
}

const char* lb_error_string(int code) {
  switch (code) {
    case LB_OK: return "ok";
    case LB_ERR_BAD_PARAM: return "argument out of range";
    case LB_ERR_OOM: return "out of device memory";
    case LB_ERR_CUDA: return "CUDA runtime error";
    case LB_ERR_NONFINITE: return "non-finite mass or pressure";
    case LB_ERR_TIMEOUT: return "device-side wait timed out";
    case LB_ERR_SIZE: return "buffer has the wrong number of elements";
    case LB_ERR_STATE: return "call not valid in the current state";
    default: return "unknown error";
  }
}

void lb_destroy(lb_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  void* ptrs[] = {c->d_lat,   c->d_rows,     c->d_items,    c->f[0],      c->f[1],       c->fields,
                  c->tmp,     c->acc_sum,    c->acc_comp,   c->partials,  c->stats,      c->d_diag,
                  c->d_row_tasks, c->d_col_tasks, c->d_t, c->d_barrier, c->d_err, c->d_scratch, c->d_mass,
                  c->pfield, c->prof_sum, c->prof_comp, c->d_row_lat, c->corr_R, c->corr_C, c->d_corr_real,
                  c->d_corr_mode, c->d_corr_modes, c->d_done, c->d_nbr_off, c->d_nbr, c->d_tmaps};
  for (void* p : ptrs) dev_free(c, p);
  delete c;
}

int lb_power_spectrum(const double* field, int Lx, int Lz, double* out, void* stream) {
  int rc = power_spectrum_args_ok(field, Lx, Lz, out);
  if (rc) return rc;
  rc = prepare_power_spectrum_current_device();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  void* tmp = nullptr;
  if (cudaMallocAsync(&tmp, (size_t)Lx * Lz * 2 * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return LB_ERR_OOM;
  }
  cudaError_t e = launch_power_spectrum(field, Lx, Lz, out, tmp, s);
  cudaError_t f = cudaFreeAsync(tmp, s);
  if (e != cudaSuccess || f != cudaSuccess) return LB_ERR_CUDA;
  return LB_OK;
}

int lb_debug_barrier(int blocks, int expected, int spin_limit) {
  if (blocks < 1 || blocks > 64 || expected < 1 || expected > 64 || spin_limit < 1 || spin_limit > 10000)
    return LB_ERR_BAD_PARAM;
  int dev = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return LB_ERR_STATE;
  unsigned* done = nullptr;
  int* list = nullptr;
  int* err = nullptr;
  int hl[64];
  for (int i = 0; i < expected; ++i) hl[i] = i;
  int rc = LB_OK;
  if (cudaMalloc(&done, 64 * sizeof(unsigned)) != cudaSuccess || cudaMalloc(&list, 64 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    rc = LB_ERR_OOM;
  if (!rc && (cudaMemset(done, 0, 64 * sizeof(unsigned)) != cudaSuccess || cudaMemset(err, 0, sizeof(int)) != cudaSuccess ||
              cudaMemcpy(list, hl, expected * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
    rc = LB_ERR_CUDA;
  if (!rc) {
    cudaError_t e = launch_barrier_probe(blocks, expected, spin_limit, done, list, err, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = LB_ERR_CUDA;
  }
  int h = 0;
  if (!rc && cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = LB_ERR_CUDA;
  if (!rc && h) rc = LB_ERR_TIMEOUT;
  cudaGetLastError();
  if (done) cudaFree(done);
  if (list) cudaFree(list);
  if (err) cudaFree(err);
  return rc;
}

int lb_debug_schedule(int n_lat, const int* Lx, const int* Lz, int tile_x, int rows, int* items_out,
                      int64_t items_cap, int* off_out, int* nbr_out, int64_t nbr_cap, int64_t* n_items,
                      int64_t* n_nbr) {
  if (n_lat < 1 || !Lx || !Lz || tile_x < 1 || rows < 1 || !n_items || !n_nbr) return LB_ERR_BAD_PARAM;
  int64_t sites = 0;
  for (int i = 0; i < n_lat; ++i) {
    if (Lx[i] < 1 || Lz[i] < 1) return LB_ERR_BAD_PARAM;
    sites += (int64_t)Lx[i] * Lz[i];
  }
  if (sites > (int64_t(1) << 26)) return LB_ERR_BAD_PARAM;
  const std::vector<int> lx(Lx, Lx + n_lat), lz(Lz, Lz + n_lat);
  std::vector<WorkItem> items;
  std::vector<std::pair<int, int>> range;
  std::vector<int> off, nbr;
  plan_items(lx, lz, tile_x, rows, items, range);
  plan_dependencies(lx, lz, items, range, tile_x, rows, off, nbr);
  *n_items = (int64_t)items.size();
  *n_nbr = (int64_t)nbr.size();
  if (items_cap < *n_items || nbr_cap < *n_nbr) return LB_ERR_SIZE;
  if (!items_out || !off_out || (*n_nbr > 0 && !nbr_out)) return LB_ERR_BAD_PARAM;
  for (size_t i = 0; i < items.size(); ++i) {
    items_out[4 * i + 0] = items[i].lattice;
    items_out[4 * i + 1] = items[i].x0;
    items_out[4 * i + 2] = items[i].z0;
    items_out[4 * i + 3] = items[i].z1;
  }
  std::copy(off.begin(), off.end(), off_out);
  std::copy(nbr.begin(), nbr.end(), nbr_out);
  return LB_OK;
}

int lb_debug_fma_rate(int precision, double* flops_per_s) {
  if ((precision != LB_PREC_FP64 && precision != LB_PREC_DEV32) || !flops_per_s) return LB_ERR_BAD_PARAM;
  cudaError_t e = measure_fma_rate(precision == LB_PREC_FP64, flops_per_s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_err(e);
  }
  return LB_OK;
}

int lb_debug_box_muller(int precision, const uint32_t* host_words, int64_t n_pairs, double* host_out) {
  if ((precision != LB_PREC_FP64 && precision != LB_PREC_DEV32) || n_pairs < 0 || n_pairs > (int64_t(1) << 24))
    return LB_ERR_BAD_PARAM;
  if (n_pairs == 0) return LB_OK;
  if (!host_words || !host_out) return LB_ERR_BAD_PARAM;
  uint32_t* dw = nullptr;
  double* dout = nullptr;
  if (cudaMalloc(&dw, (size_t)n_pairs * 2 * sizeof(uint32_t)) != cudaSuccess) return LB_ERR_OOM;
  if (cudaMalloc(&dout, (size_t)n_pairs * 2 * sizeof(double)) != cudaSuccess) {
    cudaFree(dw);
    return LB_ERR_OOM;
  }
  int rc = LB_OK;
  if (cudaMemcpy(dw, host_words, (size_t)n_pairs * 2 * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = LB_ERR_CUDA;
  if (!rc) {
    cudaError_t e = precision == LB_PREC_FP64 ? launch_debug_normals<double>(dw, n_pairs, dout, nullptr)
                                              : launch_debug_normals<float>(dw, n_pairs, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(host_out, dout, (size_t)n_pairs * 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = LB_ERR_CUDA;
  }
  cudaFree(dw);
  cudaFree(dout);
  return rc;
}

}  // extern "C"
