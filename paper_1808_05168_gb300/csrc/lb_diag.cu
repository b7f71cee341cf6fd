// lb_diag.cu -- diagnostics of the fluctuating LB method: structure factors (Appendix A,
// Eqs. SF1 and integral, on the lattice: S(q) = |delta phi(q)|^2 with the unitary 2D
// transform), mean mechanical pressure and per-species mass (Sec. II.A, III.C), plus the
// utility kernels that convert between stored and absolute populations.
//
// Structure factors: the step kernel writes the four fields of every site on a sample step;
// here one block per group of rows transforms them along x (two real rows per complex
// transform) and one block per strip of adjacent q_x transforms the columns along z, squares,
// scales by 1 / (Lx Lz) and adds the result to double-precision Kahan (compensated)
// accumulators.
#include <algorithm>

#include "lb_internal.cuh"

namespace lbk {

template <class real>
struct Cplx {
  real re, im;
};

namespace {

template <class real>
__device__ __forceinline__ void twiddle(int k, int n, real& c, real& s);
template <>
__device__ __forceinline__ void twiddle<float>(int k, int n, float& c, float& s) {
  // exp(-2 pi i k / n); k / n is exact in binary for power-of-two n
  sincospif(-2.0f * (float)k / (float)n, &s, &c);
}
template <>
__device__ __forceinline__ void twiddle<double>(int k, int n, double& c, double& s) {
  sincospi(-2.0 * (double)k / (double)n, &s, &c);
}

// In-place iterative radix-2 transform X_k = sum_j x_j exp(-2 pi i j k / n) of n = 2^logn
// points held in bit-reversed order in shared memory; tw holds exp(-2 pi i k / n), k < n/2.
template <class real>
__device__ void fft_inplace(Cplx<real>* s, const Cplx<real>* tw, int n, int logn) {
  for (int lg = 1; lg <= logn; ++lg) {
    const int half = 1 << (lg - 1);
    const int stride = n >> lg;  // twiddle index step for this stage
    for (int j = threadIdx.x; j < (n >> 1); j += blockDim.x) {
      const int pos = j & (half - 1);
      const int i0 = ((j >> (lg - 1)) << lg) + pos, i1 = i0 + half;
      const Cplx<real> w = tw[pos * stride];
      const Cplx<real> b = s[i1], a = s[i0];
      const real tr = w.re * b.re - w.im * b.im;
      const real ti = w.re * b.im + w.im * b.re;
      s[i0] = Cplx<real>{a.re + tr, a.im + ti};
      s[i1] = Cplx<real>{a.re - tr, a.im - ti};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }

// Twiddle tables of the sample-step transforms, exp(-2 pi i k / n) for k < n/2, every power of
// two n = 2 .. 8192 at offset n/2 - 1; filled once per device by prepare_sf.
constexpr int TW_TABLE = 8192;
__device__ Cplx<float> g_tw_f[TW_TABLE];
__device__ Cplx<double> g_tw_d[TW_TABLE];
template <class real>
__device__ __forceinline__ Cplx<real>* tw_table();
template <>
__device__ __forceinline__ Cplx<float>* tw_table<float>() { return g_tw_f; }
template <>
__device__ __forceinline__ Cplx<double>* tw_table<double>() { return g_tw_d; }

template <class real>
__global__ void fill_tw_tables_kernel() {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < TW_TABLE - 1; i += gridDim.x * blockDim.x) {
    const int n = 2 << (31 - __clz(i + 1));  // the table holding entry i: n/2 - 1 <= i < n - 1
    const int k = i - (n / 2 - 1);
    real c, sn;
    twiddle<real>(k, n, c, sn);
    tw_table<real>()[i] = Cplx<real>{c, sn};
  }
}

// The twiddles of an n-point transform into shared memory, from the table.
template <class real>
__device__ void load_twiddles(Cplx<real>* tw, int n) {
  const Cplx<real>* t = tw_table<real>() + (n / 2 - 1);
  for (int k = threadIdx.x; k < (n >> 1); k += blockDim.x) tw[k] = t[k];
}

template <class real>
__device__ void fill_twiddles(Cplx<real>* tw, int n) {
  for (int k = threadIdx.x; k < (n >> 1); k += blockDim.x) {
    real c, s;
    twiddle<real>(k, n, c, s);
    tw[k] = Cplx<real>{c, s};
  }
}

__device__ __forceinline__ void neumaier_add(double& sum, double& comp, double v) {
  const double t = sum + v;
  if (fabs(sum) >= fabs(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

// ---- sample-step transforms: self-sorting (Stockham) radix-16/8/4/2 passes --------------------
// A pass of radix R over sequences of n points that have already been combined in spans of Ns
// (Ns = product of the earlier radices): butterfly j (k = j mod Ns) takes the points j + r n/R,
// r = 0 .. R-1, turns point r by exp(-2 pi i r k / (Ns R)), forms their R-point DFT in registers
// and stores output q at (j - k) R + k + q Ns.  After the last pass the sequence holds its DFT
// X_k = sum_j x_j exp(-2 pi i j k / n) in natural order (the autosort formulation of Stockham's
// FFT, e.g. Govindaraju et al., SC 2008).  Each thread holds 16 points per pass; a barrier
// separates its loads from its stores, so one buffer serves every pass.

template <class real>
__device__ __forceinline__ Cplx<real> cmul(Cplx<real> a, Cplx<real> b) {
  return Cplx<real>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// cos and sin of 2 pi k / 16, k = 0 .. 7
__host__ __device__ constexpr double cos16(int k) {
  return k == 0 ? 1.0
       : k == 1 ? 0.92387953251128675613
       : k == 2 ? 0.70710678118654752440
       : k == 3 ? 0.38268343236508977173
       : k == 4 ? 0.0
       : k == 5 ? -0.38268343236508977173
       : k == 6 ? -0.70710678118654752440
                : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int k) { return k <= 4 ? cos16(4 - k) : cos16(k - 4); }

// x exp(-2 pi i k / 16) for a compile-time k in 0 .. 7 (after unrolling), without products where
// the factor is 1 or -i.
template <class real>
__device__ __forceinline__ Cplx<real> turn16(Cplx<real> x, int k) {
  if (k == 0) return x;
  if (k == 4) return Cplx<real>{x.im, -x.re};
  const real c = (real)cos16(k), s = (real)sin16(k);
  return Cplx<real>{x.re * c + x.im * s, x.im * c - x.re * s};
}

// i (0 .. 2^bits - 1, bits <= 4) with its bits reversed
__host__ __device__ constexpr int bitrev_small(int i, int bits) {
  return (((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3)) >> (4 - bits);
}

// In-order R-point DFT of v[0 .. R-1] in registers (R = 2, 4, 8, 16): radix-2 butterflies on the
// bit-reversed inputs.
template <class real, int R>
__device__ __forceinline__ void dft_regs(Cplx<real>* v) {
  constexpr int bits = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
  Cplx<real> t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[bitrev_small(i, bits)];
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
      for (int p = 0; p < h; ++p) {
        const Cplx<real> a = t[g + p], b = turn16(t[g + p + h], p * (8 / h));
        t[g + p] = Cplx<real>{a.re + b.re, a.im + b.im};
        t[g + p + h] = Cplx<real>{a.re - b.re, a.im - b.im};
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

// One pass over `seqs` sequences of n points at s + seq * sf_seq_stride(n) (point p at p + p/16);
// tw: exp(-2 pi i e / n) for e < n/2.
template <class real, int R>
__device__ __forceinline__ void stockham_pass(Cplx<real>* s, const Cplx<real>* tw, int n, int Ns, int seqs) {
  constexpr int BPT = 16 / R;  // butterflies per thread
  const int nb = n / R, lnb = 31 - __clz(nb);
  const int total = seqs * nb, SS = sf_seq_stride(n);
  const int unit = n / (Ns * R), h = n >> 1;
  Cplx<real> v[16];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      const int seq = b >> lnb, j = b & (nb - 1), k = j & (Ns - 1);
      const Cplx<real>* src = s + seq * SS;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int p = j + r * nb;
        v[i * R + r] = src[p + (p >> 4)];
      }
      if (k != 0) {
        const int st = k * unit;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const int e = r * st;  // < n
          const Cplx<real> w = tw[e < h ? e : e - h];
          const Cplx<real> ws = e < h ? w : Cplx<real>{-w.re, -w.im};
          v[i * R + r] = cmul(v[i * R + r], ws);
        }
      }
      dft_regs<real, R>(v + i * R);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * blockDim.x;
    if (b < total) {
      const int seq = b >> lnb, j = b & (nb - 1), k = j & (Ns - 1);
      Cplx<real>* dst = s + seq * SS;
      const int d = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int p = d + r * Ns;
        dst[p + (p >> 4)] = v[i * R + r];
      }
    }
  }
  __syncthreads();
}

// DFT of `seqs` sequences of n = 2^m points in place (seqs n <= 16 blockDim.x): radix-16 passes,
// then one pass of the remaining radix.
template <class real>
__device__ void stockham_fft(Cplx<real>* s, const Cplx<real>* tw, int n, int seqs) {
  int left = 31 - __clz(n), Ns = 1;
  for (; left >= 4; left -= 4, Ns <<= 4) stockham_pass<real, 16>(s, tw, n, Ns, seqs);
  if (left == 3) stockham_pass<real, 8>(s, tw, n, Ns, seqs);
  else if (left == 2) stockham_pass<real, 4>(s, tw, n, Ns, seqs);
  else if (left == 1) stockham_pass<real, 2>(s, tw, n, Ns, seqs);
}

// Global loads per thread that the transforms issue before they wait for the first (row pass,
// column pass; fewer in double precision, whose registers hold the 16 points of a pass).
template <class real>
struct SfBatch {
  static constexpr int rows = sizeof(real) == 4 ? 8 : 4, cols = sizeof(real) == 4 ? 4 : 2;
};

// Row pass: one block per (lattice, field * Lz + z0), rows z0 .. z0 + R - 1 with
// R = sf_row_group(Lx, Lz, cap).  Rows 2c and 2c + 1 of the group enter as the real and imaginary
// parts of sequence c, so one complex transform gives both: with Z = DFT(a + i b),
// A_q = (Z_q + conj Z_{n-q}) / 2 and B_q = (Z_q - conj Z_{n-q}) / (2 i).  q_x = 0 .. Lx/2 of every
// row goes to tmp; the q_x = 0 bin is the row sum, whose mean goes to the profile.
template <class real>
__global__ void __launch_bounds__(512) sf_rows_kernel(const DiagLattice* lat, const int2* tasks, const real* fields, Cplx<real>* tmp,
                               double* prof_sum, double* prof_comp, int n_rows, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int2 task = tasks[blockIdx.x];
  const DiagLattice L = lat[task.x];
  const int n = L.Lx, logn = 31 - __clz(n), H = sf_half(n), SS = sf_seq_stride(n);
  const int R = sf_row_group(n, L.Lz, cap), seqs = (R + 1) >> 1;
  Cplx<real>* tw = reinterpret_cast<Cplx<real>*>(smem);
  Cplx<real>* s = tw + ((n >> 1) + 1);
  load_twiddles<real>(tw, n);
  const real* src = fields + 4 * L.site_off + (int64_t)task.y * n;
  const int total = seqs * n, T = blockDim.x;
  // loads in batches of SfBatch<real>::rows per thread, all issued before their shared-memory stores
  for (int base = threadIdx.x; base < total; base += SfBatch<real>::rows * T) {
    real a[SfBatch<real>::rows], b[SfBatch<real>::rows];
#pragma unroll
    for (int i = 0; i < SfBatch<real>::rows; ++i) {
      const int idx = base + i * T;
      if (idx < total) {
        const int c = idx >> logn, j = idx & (n - 1);
        a[i] = src[(int64_t)(2 * c) * n + j];
        b[i] = 2 * c + 1 < R ? src[(int64_t)(2 * c + 1) * n + j] : real(0);
      }
    }
#pragma unroll
    for (int i = 0; i < SfBatch<real>::rows; ++i) {
      const int idx = base + i * T;
      if (idx < total) {
        const int c = idx >> logn, j = idx & (n - 1);
        s[c * SS + j + (j >> 4)] = Cplx<real>{a[i], b[i]};
      }
    }
  }
  __syncthreads();
  stockham_fft<real>(s, tw, n, seqs);
  Cplx<real>* out = tmp + 4 * L.site_off + (int64_t)task.y * H;
  {
    const int dc = T / H, dq = T - dc * H;
    int c = threadIdx.x / H, q = threadIdx.x - c * H;
    for (int idx = threadIdx.x; idx < seqs * H; idx += T) {
      const int qm = (n - q) & (n - 1);
      const Cplx<real> Z = s[c * SS + q + (q >> 4)], M = s[c * SS + qm + (qm >> 4)];
      const real hf = real(0.5);
      out[(int64_t)(2 * c) * H + q] = Cplx<real>{hf * (Z.re + M.re), hf * (Z.im - M.im)};
      if (2 * c + 1 < R) out[(int64_t)(2 * c + 1) * H + q] = Cplx<real>{hf * (Z.im + M.im), hf * (M.re - Z.re)};
      c += dc;
      q += dq;
      if (q >= H) {
        q -= H;
        ++c;
      }
    }
  }
  const int fld = task.y / L.Lz, z0 = task.y - fld * L.Lz;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const Cplx<real> Z0 = s[(r >> 1) * SS];
    const int64_t k = (int64_t)fld * n_rows + L.row_off + z0 + r;
    neumaier_add(prof_sum[k], prof_comp[k], (double)((r & 1) ? Z0.im : Z0.re) / (double)n);
  }
}

// Kahan summation of non-negative terms: the estimate of the total is sum - comp.
__device__ __forceinline__ void kahan_add(double& sum, double& comp, double v) {
  const double y = v - comp;
  const double t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// Column pass: one block per (lattice, field * Lx + q_x0), the strip of cq = sf_col_strip(Lx, Lz,
// cap) adjacent q_x from q_x0 (fewer at the end of q_x = 0 .. Lx/2; the fields are real, so
// S(-q) = S(q) and the rest is filled by symmetry when the spectrum is read out).  Rows of the
// strip are read and accumulated with contiguous accesses; the power is formed in the working
// precision and added to a double-precision Kahan sum.
template <class real>
__global__ void __launch_bounds__(512) sf_cols_kernel(const DiagLattice* lat, const int2* tasks, const Cplx<real>* tmp, double* acc_sum,
                               double* acc_comp, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int2 task = tasks[blockIdx.x];
  const DiagLattice L = lat[task.x];
  const int n = L.Lz, Lx = L.Lx, H = sf_half(Lx), SS = sf_seq_stride(n);
  const int fld = task.y / Lx, qx0 = task.y - fld * Lx;
  const int cq = sf_col_strip(Lx, n, cap), w = min(cq, H - qx0);
  Cplx<real>* tw = reinterpret_cast<Cplx<real>*>(smem);
  Cplx<real>* s = tw + ((n >> 1) + 1);
  load_twiddles<real>(tw, n);
  const Cplx<real>* in = tmp + 4 * L.site_off + (int64_t)fld * H * n + qx0;  // compact row transforms
  const int64_t base = 4 * L.site_off + (int64_t)fld * Lx * n + qx0;     // accumulators
  // point idx = j w + c of the strip (row j, column c); threads step idx by T, so (j, c) advance
  // by (dj, dc) with a carry
  const int T = blockDim.x, total = w * n, dj = T / w, dc = T - dj * w;
  const int j0 = threadIdx.x / w, c0 = threadIdx.x - j0 * w;
  auto advance = [&](int& j, int& c) {
    j += dj;
    c += dc;
    if (c >= w) {
      c -= w;
      ++j;
    }
  };
  {
    int j = j0, c = c0;
    for (int b0 = threadIdx.x; b0 < total; b0 += SfBatch<real>::cols * T) {
      Cplx<real> x[SfBatch<real>::cols];
      int at[SfBatch<real>::cols];
#pragma unroll
      for (int i = 0; i < SfBatch<real>::cols; ++i) {
        if (b0 + i * T < total) x[i] = in[(int64_t)j * H + c];
        at[i] = c * SS + j + (j >> 4);
        advance(j, c);
      }
#pragma unroll
      for (int i = 0; i < SfBatch<real>::cols; ++i)
        if (b0 + i * T < total) s[at[i]] = x[i];
    }
  }
  __syncthreads();
  stockham_fft<real>(s, tw, n, w);
  const real scale = real(1) / ((real)Lx * (real)n);
  int j = j0, c = c0;
  for (int b0 = threadIdx.x; b0 < total; b0 += SfBatch<real>::cols * T) {
    double sm[SfBatch<real>::cols], cp[SfBatch<real>::cols];
    real pw[SfBatch<real>::cols];
    int64_t o[SfBatch<real>::cols];
#pragma unroll
    for (int i = 0; i < SfBatch<real>::cols; ++i) {
      if (b0 + i * T < total) {
        const Cplx<real> v = s[c * SS + j + (j >> 4)];
        pw[i] = (v.re * v.re + v.im * v.im) * scale;
        o[i] = base + (int64_t)j * Lx + c;
        sm[i] = acc_sum[o[i]];
        cp[i] = acc_comp[o[i]];
      }
      advance(j, c);
    }
#pragma unroll
    for (int i = 0; i < SfBatch<real>::cols; ++i) {
      if (b0 + i * T < total) {
        kahan_add(sm[i], cp[i], (double)pw[i]);
        acc_sum[o[i]] = sm[i];
        acc_comp[o[i]] = cp[i];
      }
    }
  }
}

// ---- power spectrum of one real field (one snapshot, written out, nothing accumulated) -----
// Row pass: block z transforms row z of phi along x into tmp.
__global__ void ps_rows_kernel(const double* __restrict__ phi, int Lx, int Lz, Cplx<double>* __restrict__ tmp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int z = blockIdx.x, n = Lx, logn = ilog2(n);
  Cplx<double>* s = reinterpret_cast<Cplx<double>*>(smem);
  Cplx<double>* tw = s + n;
  fill_twiddles<double>(tw, n);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int r = (int)(__brev((unsigned)j) >> (32 - logn));
    s[r] = Cplx<double>{phi[(int64_t)z * Lx + j], 0.0};
  }
  __syncthreads();
  fft_inplace<double>(s, tw, n, logn);
  for (int j = threadIdx.x; j < n; j += blockDim.x) tmp[(int64_t)z * Lx + j] = s[j];
}

// Column pass: block b transforms columns [b cq, (b + 1) cq) along z and writes |X|^2 / (Lx Lz).
__global__ void ps_cols_kernel(const Cplx<double>* __restrict__ tmp, int Lx, int Lz, int cq, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = Lz, logn = ilog2(n), half = n >> 1, lcq = ilog2(cq), q0 = blockIdx.x * cq;
  Cplx<double>* tw = reinterpret_cast<Cplx<double>*>(smem);
  Cplx<double>* s = tw + half;
  fill_twiddles<double>(tw, n);
  for (int idx = threadIdx.x; idx < n * cq; idx += blockDim.x) {
    const int j = idx >> lcq, c = idx & (cq - 1);
    const int r = (int)(__brev((unsigned)j) >> (32 - logn));
    s[c * n + r] = tmp[(int64_t)j * Lx + q0 + c];
  }
  __syncthreads();
  for (int lg = 1; lg <= logn; ++lg) {
    const int hs = 1 << (lg - 1), stride = n >> lg;
    for (int idx = threadIdx.x; idx < half * cq; idx += blockDim.x) {
      const int c = idx / half, jj = idx - c * half;
      Cplx<double>* sc = s + c * n;
      const int pos = jj & (hs - 1);
      const int i0 = ((jj >> (lg - 1)) << lg) + pos, i1 = i0 + hs;
      const Cplx<double> w = tw[pos * stride], b = sc[i1], a = sc[i0];
      const double tr = w.re * b.re - w.im * b.im, ti = w.re * b.im + w.im * b.re;
      sc[i0] = Cplx<double>{a.re + tr, a.im + ti};
      sc[i1] = Cplx<double>{a.re - tr, a.im - ti};
    }
    __syncthreads();
  }
  const double scale = 1.0 / ((double)Lx * (double)n);
  for (int idx = threadIdx.x; idx < n * cq; idx += blockDim.x) {
    const int j = idx >> lcq, c = idx & (cq - 1);
    const Cplx<double> v = s[c * n + j];
    out[(int64_t)j * Lx + q0 + c] = (v.re * v.re + v.im * v.im) * scale;
  }
}

// One warp per lattice: lanes strided over the lattice's items, then a fixed butterfly, so the
// order of the sums is fixed (deterministic) and a lattice of many items costs a few loads per
// lane rather than one long chain.
__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void finalize_kernel(const DiagLattice* lat, int n_lat, const double* partials, DiagStats* stats) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n_lat) return;  // the whole warp
  const DiagLattice L = lat[i];
  double p = 0, ma = 0, mb = 0;
  for (int k = L.item_begin + lane; k < L.item_end; k += 32) {
    p += partials[3 * k];
    ma += partials[3 * k + 1];
    mb += partials[3 * k + 2];
  }
  p = warp_total(p);
  ma = warp_total(ma);
  mb = warp_total(mb);
  if (lane != 0) return;
  DiagStats st = stats[i];
  const double P = L.P_bg_mean + p / L.n_sites;
  st.P_last = P;
  neumaier_add(st.P_sum, st.P_comp, P);
  st.massA_last = L.mass_bg[0] + ma;
  st.massB_last = L.mass_bg[1] + mb;
  if (!isfinite(P) || !isfinite(st.massA_last) || !isfinite(st.massB_last)) st.nonfinite = 1;
  stats[i] = st;
}

// Mass of the stored state of one lattice: one block per species, fixed summation order.
template <class real>
__global__ void mass_kernel(const real* f, BgParams bp, double* out) {
  const int s = blockIdx.x;
  const int64_t LzLx = (int64_t)bp.Lx * bp.Lz;
  double acc = 0.0;  // over the pairs [link][z][x], species s of each
  for (int64_t k = threadIdx.x; k < 9 * LzLx; k += blockDim.x) acc += (double)f[2 * k + s];
  __shared__ double red[1024];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double bg = 0.0;
    if (bp.dev) {
      for (int z = 0; z < bp.Lz; ++z) {
        const double c0 = 0.5 + (z + 0.5 - 0.5 * bp.Lz) * bp.grad_c0;
        bg += bp.rho_bar * (s == 0 ? c0 : 1.0 - c0);
      }
      bg *= bp.Lx;
    }
    out[s] = bg + red[0];
  }
}

__device__ __forceinline__ double weight_of(int l) { return l == 0 ? 4.0 / 9.0 : (l <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

__device__ __forceinline__ double background(const BgParams& bp, int s, int l, int z) {
  if (!bp.dev) return 0.0;
  const double c0 = 0.5 + (z + 0.5 - 0.5 * bp.Lz) * bp.grad_c0;
  return weight_of(l) * bp.rho_bar * (s == 0 ? c0 : 1.0 - c0);
}

// The API layout [species][link][z][x] (index k) against the stored pairs (state_index).
template <class real>
__global__ void to_absolute_kernel(const real* f, BgParams bp, double* out) {
  const int64_t LzLx = (int64_t)bp.Lx * bp.Lz, n = 18 * LzLx;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int sl = (int)(k / LzLx), s = sl / 9, l = sl - 9 * s;
    const int64_t r = k - sl * LzLx;
    const int z = (int)(r / bp.Lx);
    out[k] = (double)f[state_index(s, l, 0, 0, bp.Lx, LzLx) + 2 * r] + background(bp, s, l, z);
  }
}

template <class real>
__global__ void from_absolute_kernel(const double* in, BgParams bp, real* f) {
  const int64_t LzLx = (int64_t)bp.Lx * bp.Lz, n = 18 * LzLx;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int sl = (int)(k / LzLx), s = sl / 9, l = sl - 9 * s;
    const int64_t r = k - sl * LzLx;
    const int z = (int)(r / bp.Lx);
    f[state_index(s, l, 0, 0, bp.Lx, LzLx) + 2 * r] = (real)(in[k] - background(bp, s, l, z));
  }
}

// Rest state f^S_l = w_l rho_bar c^S_0(z) (stored as zero deviations in deviation mode).
template <class real>
__global__ void init_rest_kernel(real* f, BgParams bp) {
  const int64_t LzLx = (int64_t)bp.Lx * bp.Lz, n = 18 * LzLx;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (bp.dev) {
      f[k] = real(0);
    } else {  // element k of the stored pairs: species k mod 2 of pair k / 2
      const int64_t q = k >> 1;
      const int s = (int)(k & 1), l = (int)(q / LzLx);
      const int z = (int)((q - l * LzLx) / bp.Lx);
      const double c0 = 0.5 + (z + 0.5 - 0.5 * bp.Lz) * bp.grad_c0;
      f[k] = (real)(weight_of(l) * bp.rho_bar * (s == 0 ? c0 : 1.0 - c0));
    }
  }
}

// Columns x_first .. x_first + n - 1 of every (species, link) plane, to (to_buf) or from a packed
// buffer [9 * species + link][Lz][n] (the API layout); thread k handles element k of the buffer.
template <class real>
__global__ void columns_kernel(real* f, int Lx, int Lz, int x_first, int n, real* buf, bool to_buf) {
  const int64_t total = (int64_t)18 * Lz * n, LzLx = (int64_t)Lx * Lz;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = k / n;  // plane * Lz + z
    const int j = (int)(k - row * n), sl = (int)(row / Lz), z = (int)(row - (int64_t)sl * Lz), s = sl / 9;
    real* g = f + state_index(s, sl - 9 * s, z, x_first + j, Lx, LzLx);
    if (to_buf) buf[k] = *g;
    else *g = buf[k];
  }
}

// Fused multiply-add throughput: eight independent chains per thread x <- x a + b (|a| < 1, so the
// values stay bounded), enough resident warps to fill every pipe; the sum keeps the chains live.
template <class T>
__global__ void fma_rate_kernel(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-6;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace

cudaError_t measure_fma_rate(bool fp64, double* flops_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int threads = 256, blocks = 8 * sms, iters = fp64 ? 2048 : 16384;
  void* out = nullptr;
  e = cudaMalloc(&out, (size_t)threads * blocks * sizeof(double));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto run = [&]() {
    if (fp64) fma_rate_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.9999999, 1e-9);
    else fma_rate_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.9999f, 1e-6f);
  };
  float best = 1e30f;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    run();  // warm-up
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
      cudaEventRecord(e0);
      run();
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess) best = std::min(best, ms);
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess) *flops_per_s = 2.0 * 8 * iters * (double)threads * blocks / (best * 1e-3);
  return e;
}

template <class real>
cudaError_t launch_columns(real* f, int Lx, int Lz, int x_first, int n, real* buf, bool to_buf, cudaStream_t s) {
  const int64_t total = (int64_t)18 * Lz * n;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  columns_kernel<real><<<blocks, 256, 0, s>>>(f, Lx, Lz, x_first, n, buf, to_buf);
  return cudaGetLastError();
}

template <class real>
cudaError_t prepare_sf(size_t smem_rows, size_t smem_cols) {
  fill_tw_tables_kernel<real><<<(TW_TABLE + 255) / 256, 256>>>();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(sf_rows_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sf_cols_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols);
}

template <class real>
cudaError_t launch_sf(const SfPlan& p, const real* fields, void* tmp, double* acc_sum, double* acc_comp,
                      cudaStream_t s) {
  sf_rows_kernel<real><<<p.n_row_tasks, p.threads, p.smem_rows, s>>>(p.lat, p.row_tasks, fields, (Cplx<real>*)tmp,
                                                                     p.prof_sum, p.prof_comp, p.n_rows, p.cap);
  sf_cols_kernel<real><<<p.n_col_tasks, p.threads, p.smem_cols, s>>>(p.lat, p.col_tasks, (const Cplx<real>*)tmp,
                                                                     acc_sum, acc_comp, p.cap);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const DiagLattice* d_lat, int n_lat, const double* partials, DiagStats* stats,
                            cudaStream_t s) {
  finalize_kernel<<<(n_lat + 3) / 4, 128, 0, s>>>(d_lat, n_lat, partials, stats);  // 4 lattices per block
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_mass(const real* f, const BgParams& bp, double* out2, cudaStream_t s) {
  mass_kernel<real><<<2, 1024, 0, s>>>(f, bp, out2);
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_to_absolute(const real* f, const BgParams& bp, double* out, cudaStream_t s) {
  to_absolute_kernel<real><<<1024, 256, 0, s>>>(f, bp, out);
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_from_absolute(const double* in, const BgParams& bp, real* f, cudaStream_t s) {
  from_absolute_kernel<real><<<1024, 256, 0, s>>>(in, bp, f);
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_init_rest(real* f, const BgParams& bp, cudaStream_t s) {
  init_rest_kernel<real><<<1024, 256, 0, s>>>(f, bp);
  return cudaGetLastError();
}

// Dynamic shared memory of the one-snapshot passes for transforms of up to 8192 points: the
// points plus half as many twiddles, 16 bytes each (196,608 bytes, within the 227 KB a block may
// opt in to).
constexpr size_t kPsSmemMax = (8192 + 4096) * sizeof(Cplx<double>);

// Columns per block of the one-snapshot column pass: up to 16, as many as fit in kPsSmemMax (one
// column of 8192 points fills it).
static int ps_column_strip(int Lx, int Lz) {
  int cq = 16;
  while (cq > 1 && ((size_t)Lz * cq + Lz / 2) * sizeof(Cplx<double>) > kPsSmemMax) cq >>= 1;
  return cq < Lx ? cq : Lx;
}

cudaError_t prepare_power_spectrum() {
  cudaError_t e = cudaFuncSetAttribute(ps_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPsSmemMax);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(ps_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPsSmemMax);
}

cudaError_t launch_power_spectrum(const double* field, int Lx, int Lz, double* out, void* tmp, cudaStream_t s) {
  const int cq = ps_column_strip(Lx, Lz);
  ps_rows_kernel<<<Lz, 256, (size_t)(Lx + Lx / 2) * sizeof(Cplx<double>), s>>>(field, Lx, Lz, (Cplx<double>*)tmp);
  ps_cols_kernel<<<Lx / cq, 256, ((size_t)Lz * cq + Lz / 2) * sizeof(Cplx<double>), s>>>(
      (const Cplx<double>*)tmp, Lx, Lz, cq, out);
  return cudaGetLastError();
}

// z-profile of the pressure (Sec. III.C): warp r of the grid sums global row r of the sampled
// pressure over x in a fixed order (lane-strided partial sums in the working precision, four
// values at a time, then in double and a butterfly) and adds the row mean to the compensated sum.
template <class real>
__global__ void profile_kernel(const DiagLattice* __restrict__ lat, const int* __restrict__ row_lat, int n_rows,
                               const real* __restrict__ pfield, double* __restrict__ prof_sum,
                               double* __restrict__ prof_comp) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;  // whole warps
  const DiagLattice& L = lat[row_lat[r]];
  const int Lx = L.Lx, z = r - L.row_off;
  const real* p0 = pfield + L.site_off + (int64_t)z * Lx;
  double acc = 0.0;
  if ((Lx & 3) == 0) {
    for (int x = lane * 4; x < Lx; x += 128) acc += (double)((p0[x] + p0[x + 1]) + (p0[x + 2] + p0[x + 3]));
  } else {
    for (int x = lane; x < Lx; x += 32) acc += (double)p0[x];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) neumaier_add(prof_sum[4 * (int64_t)n_rows + r], prof_comp[4 * (int64_t)n_rows + r], acc / (double)Lx);
}

template <class real>
cudaError_t launch_profiles(const DiagLattice* lat, const int* row_lat, int n_rows, const real* fields,
                            const real* pfield, double* prof_sum, double* prof_comp, cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  const int64_t blocks = ((int64_t)n_rows * 32 + 255) / 256;
  profile_kernel<real><<<(unsigned)blocks, 256, 0, s>>>(lat, row_lat, n_rows, pfield, prof_sum, prof_comp);
  (void)fields;
  return cudaGetLastError();
}

// Real-space correlation of one sample: block (CORR_TILE^2 threads) per (lattice, field, z tile,
// z' tile); x runs in chunks of 32 staged in shared memory, each chunk's products summed in the
// working precision and the chunk sums in double.
template <class real>
__global__ void corr_real_kernel(const DiagLattice* __restrict__ lat, const int4* __restrict__ tasks,
                                 const real* __restrict__ fields, double* __restrict__ R) {
  constexpr int T = CORR_TILE;
  __shared__ real a[32][T + 1], b[32][T + 1];
  const int4 t = tasks[blockIdx.x];
  const DiagLattice& L = lat[t.x];
  const int Lx = L.Lx, Lz = L.Lz, fld = t.y, z0 = t.z * T, zp0 = t.w * T;
  const int tz = threadIdx.x % T, tzp = threadIdx.x / T;
  const real* f = fields + 4 * L.site_off + (int64_t)fld * Lx * Lz;
  double acc = 0.0;
  for (int x0 = 0; x0 < Lx; x0 += 32) {
    for (int i = threadIdx.x; i < 32 * T; i += T * T) {
      const int xx = i & 31, zz = i >> 5, x = x0 + xx, z = z0 + zz, zp = zp0 + zz;
      a[xx][zz] = (x < Lx && z < Lz) ? f[(int64_t)z * Lx + x] : real(0);
      b[xx][zz] = (x < Lx && zp < Lz) ? f[(int64_t)zp * Lx + x] : real(0);
    }
    __syncthreads();
    real sum = 0;
#pragma unroll 8
    for (int xx = 0; xx < 32; ++xx) sum += a[xx][tz] * b[xx][tzp];
    acc += (double)sum;
    __syncthreads();
  }
  const int z = z0 + tz, zp = zp0 + tzp;
  if (z < Lz && zp < Lz) R[L.r_off + ((int64_t)fld * Lz + z) * Lz + zp] += acc / (double)Lx;
}

// Mode correlation of one sample: thread per (z, z') of a tile, from the row transforms
// X(q, z) = sum_x dphi(x, z) exp(-i q x) (unnormalised): C += conj(X(q, z)) X(q, z') / Lx.
template <class real>
__global__ void corr_mode_kernel(const DiagLattice* __restrict__ lat, const int4* __restrict__ tasks,
                                 const int* __restrict__ modes, int n_modes, const Cplx<real>* __restrict__ tmp,
                                 double* __restrict__ C) {
  constexpr int T = CORR_TILE;
  const int4 t = tasks[blockIdx.x];
  const DiagLattice& L = lat[t.x];
  const int Lx = L.Lx, Lz = L.Lz, fld = t.y / n_modes, m = t.y - fld * n_modes, k = modes[m];
  const int z = t.z * T + (int)threadIdx.x % T, zp = t.w * T + (int)threadIdx.x / T;
  if (z >= Lz || zp >= Lz) return;
  const int H = sf_half(Lx);
  const Cplx<real>* X = tmp + 4 * L.site_off + (int64_t)fld * Lz * H;
  // q_x > Lx/2 from the conjugate symmetry of a real field's transform
  const int kk = k < H ? k : Lx - k;
  const double sg = k < H ? 1.0 : -1.0;
  const Cplx<real> u = X[(int64_t)z * H + kk], v = X[(int64_t)zp * H + kk];
  const double ur = u.re, ui = sg * (double)u.im, vr = v.re, vi = sg * (double)v.im, inv = 1.0 / (double)Lx;
  double* c = C + L.c_off + ((((int64_t)fld * n_modes + m) * Lz + z) * Lz + zp) * 2;
  c[0] += (ur * vr + ui * vi) * inv;
  c[1] += (ur * vi - ui * vr) * inv;
}

template <class real>
cudaError_t launch_corr(const CorrPlan& p, const real* fields, const void* tmp, double* R, double* C, cudaStream_t s) {
  if (p.n_real_tasks > 0)
    corr_real_kernel<real><<<p.n_real_tasks, CORR_TILE * CORR_TILE, 0, s>>>(p.lat, p.real_tasks, fields, R);
  if (p.n_mode_tasks > 0)
    corr_mode_kernel<real><<<p.n_mode_tasks, CORR_TILE * CORR_TILE, 0, s>>>(
        p.lat, p.mode_tasks, p.modes, p.n_modes, (const Cplx<real>*)tmp, C);
  return cudaGetLastError();
}

#define LB_INST(real)                                                                                        \
  template cudaError_t prepare_sf<real>(size_t, size_t);                                                     \
  template cudaError_t launch_sf<real>(const SfPlan&, const real*, void*, double*, double*, cudaStream_t);   \
  template cudaError_t launch_mass<real>(const real*, const BgParams&, double*, cudaStream_t);               \
  template cudaError_t launch_to_absolute<real>(const real*, const BgParams&, double*, cudaStream_t);        \
  template cudaError_t launch_from_absolute<real>(const double*, const BgParams&, real*, cudaStream_t);      \
  template cudaError_t launch_init_rest<real>(real*, const BgParams&, cudaStream_t);                         \
  template cudaError_t launch_columns<real>(real*, int, int, int, int, real*, bool, cudaStream_t);           \
  template cudaError_t launch_profiles<real>(const DiagLattice*, const int*, int, const real*, const real*,    \
                                             double*, double*, cudaStream_t);                                \
  template cudaError_t launch_corr<real>(const CorrPlan&, const real*, const void*, double*, double*, cudaStream_t);
LB_INST(float)
LB_INST(double)

}  // namespace lbk
