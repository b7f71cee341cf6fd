/*
 * lb.h -- C interface of the GB300 library for the fluctuating two-species D2Q9 lattice
 * Boltzmann method of Belardinelli, Sbragaglia, Benzi & Ciliberto, "Lattice Boltzmann
 * simulations of non-equilibrium fluctuations in a non-ideal binary mixture"
 * (arXiv:1808.05168).
 *
 * The problem (Sec. II.A): a binary mixture A/B on an Lx x Lz D2Q9 lattice, periodic in x,
 * between two solid walls at z = +-Lz/2 (mid-way bounce-back), with an imposed linear
 * concentration profile c_0(z) = 1/2 + z grad_c0 (Fig. 1), reference density rho_bar = 1.
 * One step (Eq. LB) streams both species, computes the non-ideal inter-species force
 * (Eq. aNI, coupling G) with its a* correction (footnote to Eq. ne-acc), the gradient force
 * (Eq. ne-acc), the barycentric velocity (Eq. bar), and relaxes every moment of Table I at its
 * own rate (Eq. MRT) with second-order forcing and Gaussian noise whose variances obey the
 * fluctuation-dissipation theorem (Eqs. noise-bin-expl, noise-bin-expl-high).  The
 * diagnostics are the structure factors of Appendix A (Eqs. SF1, integral) and the mean
 * mechanical pressure of Sec. III.C (Eq. EQUATIONofSTATE in the bulk).
 *
 * Conventions for every call below:
 *  - a call returns LB_OK (0) or a negative LB_ERR_* code; nothing aborts or throws;
 *  - host buffers are owned by the caller; sizes are element counts and are checked;
 *  - lb_step only enqueues work on the context's stream; calls that return values to the
 *    host synchronise that stream first;
 *  - device memory is owned by the context and freed by lb_destroy;
 *  - a context is used by one host thread at a time.
 */
#ifndef LB_GB300_H
#define LB_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define LB_OK 0
#define LB_ERR_BAD_PARAM (-1) /* an argument is out of its documented range            */
#define LB_ERR_OOM (-2)       /* device memory could not be allocated                   */
#define LB_ERR_CUDA (-3)      /* a CUDA runtime call failed                             */
#define LB_ERR_NONFINITE (-4) /* a sampled mass or pressure is not finite               */
#define LB_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up                     */
#define LB_ERR_SIZE (-6)      /* a caller buffer has the wrong element count            */
#define LB_ERR_STATE (-7)     /* the call is not valid in the context's current state   */

/* ---- flags of lb_create / lb_create_batch ------------------------------------------- */
#define LB_PREC_FP64 0x00  /* populations stored and collided in double precision        */
#define LB_PREC_DEV32 0x01 /* float deviations from the weighted background w_l rho_bar
                              c^S_0(z); double-precision sums for mass, pressure and the
                              time averages                                               */
#define LB_NO_ASTAR 0x02   /* drop the a* diffusion correction (footnote to Eq. ne-acc)   */
#define LB_WALL_FIXED 0x04 /* wall ghost densities for the non-ideal force take the fixed
                              wall composition c_0(+-Lz/2) instead of copying the adjacent
                              fluid row's composition (Sec. II.A)                          */
#define LB_NOISE_LOC 0x08  /* noise variances with the local densities ("loc", Sec. III.B)
                              instead of the reference values ("hom")                      */
#define LB_GRAPH 0x10      /* run lb_step through captured CUDA graphs                     */
#define LB_PERSISTENT 0x20 /* one cooperative launch per run of plain steps, all lattices of
                              the batch: work items handed out in order, each waiting
                              (bounded) for its neighbours' previous step; a sample step
                              follows as an ordinary launch                              */
#define LB_AUTOTUNE 0x40   /* time the candidate tile shapes on the first lb_step          */
#define LB_NO_BULK 0x80    /* stage populations with per-thread copies even where rows are
                              16-byte aligned (bulk copies are used by default there)     */
#define LB_NO_TENSOR_MAPS 0x100 /* bulk staging with 1-d copies only: no 3-d tensor copies of
                              runs of links (used by default in FP32 for strips away from
                              the periodic x edges with tiles of up to 128 columns)       */

/* ---- structure-factor fields and modes (Appendix A) ---------------------------------- */
#define LB_FIELD_RHO 0 /* delta rho = rho - rho_bar                                         */
#define LB_FIELD_C 1   /* delta c = c - c_0(z)                                              */
#define LB_FIELD_UX 2  /* U_x of Eq. (bar)                                                  */
#define LB_FIELD_UZ 3  /* U_z of Eq. (bar)                                                  */
#define LB_FIELD_P 4   /* mechanical pressure, half the trace of the pressure tensor (profiles
                          only: lb_profile)                                                 */
#define LB_SF_QXQZ 0   /* S(q_x, q_z): Lz x Lx doubles, [n][k] at q_z = 2 pi n / Lz,
                          q_x = 2 pi k / Lx                                                 */
#define LB_SF_QX 1     /* S(q_x, q_z = 0): Lx doubles                                       */

/* Parameters of one lattice (Sec. II.A, Eq. MRT, Table I).  Relaxation rates lie in (0, 2):
 * lambda_s (moments 4, 5; viscosity, Eq. vis), lambda_d (moments 1, 2; diffusion, Eq. diff),
 * lambda_e (moment 3), lambda_q (moments 6, 7), lambda_eps (moment 8).  kT >= 0; G >= 0;
 * grad_c0 is the imposed gradient (wall-to-wall difference / Lz) with |grad_c0| Lz < 1.
 * seed keys the Philox4x32-10 noise stream; lattice_id is its third counter word, so two
 * lattices with one seed and different ids draw independent noise. */
typedef struct lb_params {
  int32_t Lx, Lz;
  double lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps;
  double kT, G, grad_c0;
  uint64_t seed;
  uint32_t lattice_id;
  uint32_t reserved; /* must be 0 */
} lb_params;

typedef struct lb_ctx lb_ctx;

/* Create one lattice (lattice_id 0) in the rest state f^S_l = w_l rho_bar c^S_0(z).
 * Lx >= 1, Lz >= 2, Lx * Lz < 2^31.  *out receives the context (NULL on failure). */
int lb_create(lb_ctx** out, int Lx, int Lz, double lambda_s, double lambda_d, double lambda_e, double lambda_q,
              double lambda_eps, double kT, double G, double grad_c0, uint64_t seed, int flags);

/* Create a batch of n >= 1 independent lattices (each may have its own size and
 * parameters), advanced together by lb_step in one launch per step. */
int lb_create_batch(lb_ctx** out, int n, const lb_params* params, int flags);

/* Device memory from the caller: as lb_create_batch, but every device buffer the context holds
 * (state, tables, diagnostics, correlations, and the temporaries of lb_pressure_shift_gradient)
 * is obtained with alloc_fn(bytes, user) and returned with free_fn(ptr, user), e.g. from a
 * framework's caching allocator on the current device.  alloc_fn returns a device pointer
 * aligned to at least 256 bytes, or NULL (the call then fails with LB_ERR_OOM); free_fn is called
 * once for every pointer, after the context's work on it has finished, at the latest in
 * lb_destroy.  Both functions must stay valid for the context's lifetime; both are required
 * (LB_ERR_BAD_PARAM otherwise).  lb_power_spectrum is not affected (it takes no context). */
typedef void* (*lb_alloc_fn)(size_t bytes, void* user);
typedef void (*lb_free_fn)(void* ptr, void* user);
int lb_create_batch_with_allocator(lb_ctx** out, int n, const lb_params* params, int flags, lb_alloc_fn alloc_fn,
                                   lb_free_fn free_fn, void* user);

/* Run on a caller-owned cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream);
 * NULL selects the context's own non-blocking stream (the default after lb_create).
 * Pending work on the previous stream is waited for first. */
int lb_set_stream(lb_ctx* ctx, void* cuda_stream);

/* Sample the diagnostics on steps t >= discard with (t - discard) % every == 0; every = 0
 * turns sampling off (the default).  Sampling uses the pre-collision state of step t.  The
 * structure factors are taken by power-of-two transforms: with every > 0 each lattice must have
 * Lx and Lz powers of two with 2 <= Lx <= 8192 and Lz <= 8192 (LB_ERR_BAD_PARAM otherwise; the
 * paper's lattices are all of that kind). */
int lb_set_sampling(lb_ctx* ctx, int64_t discard, int64_t every);

/* Fix the tile shape: tile_x columns per block (32, 64, 128 or 256) and rows_per_item rows
 * per work item (>= 1; larger values are clipped to Lz).  Overrides LB_AUTOTUNE. */
int lb_set_tile(lb_ctx* ctx, int tile_x, int rows_per_item);
int lb_get_tile(lb_ctx* ctx, int* tile_x, int* rows_per_item);

/* Advance every lattice by n >= 0 steps (asynchronous on the context's stream). */
int lb_step(lb_ctx* ctx, int64_t n);

/* Wait for the context's stream; reports a device-side error flag (LB_ERR_TIMEOUT). */
int lb_synchronize(lb_ctx* ctx);

/* Number of steps taken so far. */
int lb_time(lb_ctx* ctx, int64_t* t);

int lb_num_lattices(lb_ctx* ctx, int* n);
int lb_lattice_shape(lb_ctx* ctx, int lattice, int* Lx, int* Lz);

/* Time-averaged structure factor of one field (LB_FIELD_*) of one lattice, as the mean of
 * |delta phi(q)|^2 over the samples, with the unitary transform (Lx Lz)^(-1/2)
 * (Appendix A).  n_out must be Lx * Lz for LB_SF_QXQZ and Lx for LB_SF_QX.
 * *n_samples (may be NULL) receives the sample count. */
int lb_structure_factor(lb_ctx* ctx, int lattice, int field, int mode, double* host_out, size_t n_out,
                        int64_t* n_samples);

/* z-profile of one field of one lattice (Sec. III.C, the average total pressure and density
 * profiles): for rows j = 0..Lz-1 (height z_j = j + 1/2 - Lz/2), the average over the samples of
 * the row mean (1/Lx) sum_x phi(x, z_j) of the absolute field phi = rho, c, U_x, U_z (LB_FIELD_RHO,
 * LB_FIELD_C, LB_FIELD_UX, LB_FIELD_UZ) or the mechanical pressure P (LB_FIELD_P), all taken on
 * the pre-collision state of the sample steps.  host_out: caller-owned, n_out == Lz doubles, else
 * LB_ERR_SIZE.  Zeros before the first sample; *n_samples (may be NULL) receives the count. */
int lb_profile(lb_ctx* ctx, int lattice, int field, double* host_out, size_t n_out, int64_t* n_samples);

/* Two-point correlations of the sampled fields (Sec. III.A-B real-space correlations,
 * Eqs. VELOCITY_CORR and CONCENTRATION_CORR; Appendix A mixed correlation C(q_x, z, z')),
 * accumulated on every sample step from this call on (the count restarts here and at
 * lb_reset_statistics).  field_mask: bit f set for field f (LB_FIELD_RHO .. LB_FIELD_UZ), 0 turns
 * them off; modes: n_modes <= LB_CORR_MAX_MODES mode indices k (q_x = 2 pi k / Lx, 0 <= k < Lx of
 * every lattice) whose mixed correlations are kept.  Same lattice-size rule as lb_set_sampling.
 * Device memory: 8 (4 + 8 n_modes) sum_lattices Lz^2 bytes. */
#define LB_CORR_MAX_MODES 16
int lb_set_correlations(lb_ctx* ctx, int field_mask, int n_modes, const int* modes);

/* Equal-x real-space correlation <dphi(x, z) dphi(x, z')> of one field of one lattice, averaged
 * over x and the samples: host_out[z * Lz + z'], n_out == Lz * Lz doubles (LB_ERR_SIZE otherwise);
 * LB_ERR_STATE if the field is not enabled by lb_set_correlations. */
int lb_correlation(lb_ctx* ctx, int lattice, int field, double* host_out, size_t n_out, int64_t* n_samples);

/* Mixed correlation C(q_x, z, z') = <dphi(q_x, z)^* dphi(q_x, z')> of Appendix A for the
 * mode_index-th mode of lb_set_correlations, with the unitary partial transform
 * dphi(q_x, z) = Lx^(-1/2) sum_x dphi(x, z) exp(-i q_x x): host_out[2 (z * Lz + z') + {0, 1}] =
 * (real, imaginary) part, n_out == 2 Lz^2 doubles; errors as lb_correlation. */
int lb_mode_correlation(lb_ctx* ctx, int lattice, int field, int mode_index, double* host_out, size_t n_out,
                        int64_t* n_samples);

/* Spatial mean of the mechanical pressure (Sec. III.C) at the latest sample, and its average
 * over all samples (compensated double-precision sum).  Either pointer may be NULL. */
int lb_mean_pressure(lb_ctx* ctx, int lattice, double* last, double* time_avg);

/* Per-species total mass sum_r sum_l f^S_l of the stored state, in double precision
 * (exactly conserved by the method up to rounding, Sec. II.A). */
int lb_mass(lb_ctx* ctx, int lattice, double out[2]);

/* Copy the stored (post-collision) populations of one lattice as absolute values in double
 * precision, layout [species][link][z][x] (2 * 9 * Lz * Lx values).  Links follow Fig. 1:
 * c_0 = 0, c_1 = (1,0), c_2 = (0,1), c_3 = (-1,0), c_4 = (0,-1), c_5 = (1,1), c_6 = (-1,1),
 * c_7 = (-1,-1), c_8 = (1,-1). */
int lb_get_populations(lb_ctx* ctx, int lattice, double* host_out, size_t n);
int lb_set_populations(lb_ctx* ctx, int lattice, const double* host_in, size_t n);

/* ---- x-slab decomposition of one large lattice ---------------------------------------------
 * The lattice is periodic in x and its walls bound z (Sec. II.A), so it can be cut into slabs of
 * columns, one per process (or GPU).  A site's update reads the populations within two columns
 * (streaming brings them from one column away and the non-ideal force, Eq. aNI, needs the
 * densities of the neighbouring columns), so a slab owning columns [x0, x0 + w) of a lattice
 * Lx_global wide is stepped as a lattice of w + 4 columns whose first and last two are halo
 * columns: after every step its own w columns are exact, and the halos are refilled from the
 * neighbours' boundary columns (two each side) before the next step.  The windows' results then
 * equal the undivided lattice's bit for bit.  Diagnostics (sampling, correlations, the
 * mean-pressure gradient) see the whole window, halos included, and are not meant for slabs. */

/* Noise counters of an x-slab window: from this call on, the Philox site counter of column x,
 * row z of the lattice is z * Lx_global + (x + x0) mod Lx_global, that of column x + x0 of the
 * undivided lattice (Sec. II.B noise; the default is x0 = 0, Lx_global = Lx).  For a slab owning
 * [x_s, x_s + w) with two halo columns on each side, x0 = (x_s - 2) mod Lx_global.  Requires
 * Lx <= Lx_global, 0 <= x0 < Lx_global and Lx_global * Lz < 2^31 (LB_ERR_BAD_PARAM otherwise).
 * Synchronises the context's stream; lb_pressure_shift_gradient refuses a context with a
 * non-default map (LB_ERR_STATE). */
int lb_set_site_map(lb_ctx* ctx, int lattice, int x0, int Lx_global);

/* Copy columns [x_first, x_first + n_cols) of all 18 planes of the lattice's current stored state
 * to (export) or from (import) a packed device buffer laid out [species * 9 + link][z][column],
 * 18 * Lz * n_cols values of the storage type: float deviations from the background
 * w_l rho_bar c^S_0(z) with LB_PREC_DEV32, absolute doubles with LB_PREC_FP64 (two slabs of one
 * lattice share the background, so the raw values move between them unchanged).  The buffer is
 * device (or managed) memory of the current device, owned by the caller (the halo exchange sends
 * it to the neighbour).  Stream-ordered on the context's stream; returns before the copy is done.
 * 1 <= n_cols, 0 <= x_first <= Lx - n_cols; a host pointer or another device's memory returns
 * LB_ERR_BAD_PARAM before anything is launched. */
int lb_export_columns(lb_ctx* ctx, int lattice, int x_first, int n_cols, void* device_out);
int lb_import_columns(lb_ctx* ctx, int lattice, int x_first, int n_cols, const void* device_in);

/* Power spectrum of one snapshot of a real field (Appendix A, Eqs. SF1 and integral on the
 * lattice): out[n * Lx + k] = |sum_{x,z} phi[z * Lx + x] exp(-2 pi i (k x / Lx + n z / Lz))|^2
 * / (Lx Lz).  field and out are device pointers to Lx * Lz doubles (x fastest; out may not
 * alias field), in memory of the current device (or managed memory); Lx and Lz are powers of two
 * in 2..8192.  Host pointers, another device's memory or other sizes return LB_ERR_BAD_PARAM
 * before anything is launched.  Stream-ordered on `stream` (NULL: legacy default stream), which also
 * orders a device scratch of Lx * Lz * 16 bytes allocated and freed with cudaMallocAsync /
 * cudaFreeAsync; returns before the result is ready. */
int lb_power_spectrum(const double* field, int Lx, int Lz, double* out, void* stream);

/* lb_power_spectrum for callers that must not allocate device memory (the paper has no
 * counterpart; this is a deployment aid).  Some callers cannot call cudaMalloc, cudaFree or any
 * allocating routine where they need a spectrum: code running while another owner captures a
 * CUDA graph, processes whose device memory is owned by another framework's pool, or loops that
 * must never wait on an allocator.  Same arguments, checks (LB_ERR_BAD_PARAM), result and stream
 * ordering as lb_power_spectrum, and in addition Lx * Lz <= LB_NOALLOC_MAX_POINTS (larger
 * products return LB_ERR_SIZE);
 * the intermediate transform lives in a fixed 4 MiB array compiled into the library, which
 * every GPU that loads the library holds until the process exits.  The first call on a device
 * (with that device current) looks up the array's device address and sets the kernels'
 * attributes, so make that first call before any stream capture.  Every call shares the one
 * array: calls whose work overlaps on the GPU (different streams, or different host threads)
 * race on it and give wrong results; the array needs no clearing, since each call overwrites
 * what it reads. */
#define LB_NOALLOC_MAX_POINTS (1 << 18)
int lb_power_spectrum_noalloc(const double* field, int Lx, int Lz, double* out, void* stream);

/* Gradient of the time-averaged mean-pressure shift on a fixed noise stream,
 *   L = (1/T) sum_{t<T} Pbar(t)|_{kT} - (1/T) sum_{t<T} Pbar(t)|_{kT=0},
 * both runs from the rest state with the context's parameters (Pbar(t): spatial mean of the
 * mechanical pressure of Sec. III.C on the pre-collision state of step t; the kT = 0 run is the
 * noiseless companion of Eqs. EQP/NEQP), with respect to (G, lambda_s, lambda_d); lambda_e,
 * lambda_q, lambda_eps and kT are held fixed.  grad[0..2] = dL/dG, dL/dlambda_s, dL/dlambda_d
 * by a hand-written reverse sweep of the step that recomputes the forward states from
 * checkpoints taken every ckpt_every steps (1 <= ckpt_every <= steps); grad may be NULL to get
 * the loss alone.  The context's own state, step count and statistics are not touched.
 * Requires a single-lattice context (LB_ERR_STATE otherwise); every option of the step is
 * differentiated: a* on or off (LB_NO_ASTAR), copy-rule or fixed-composition wall ghosts
 * (LB_WALL_FIXED), hom or loc noise (LB_NOISE_LOC, whose amplitudes follow the local densities).
 * The runs with and without noise are independent until they are combined and run on two
 * streams (the context's and one of the call's own), each with its own buffers.  Device memory:
 * about 2 (steps/ckpt_every + ckpt_every + 5) states, allocated for the call and freed before it
 * returns.  Synchronous. */
int lb_pressure_shift_gradient(lb_ctx* ctx, int64_t steps, int64_t ckpt_every, double grad[3], double* loss);

/* lb_pressure_shift_gradient for every lattice of a batch in one sweep: each lattice's own loss
 * L_i (its runs with and without noise, the spatial mean over its own sites) in losses[i] and its
 * gradient in grads[3 i .. 3 i + 2] (host arrays of n_lat and 3 n_lat doubles; either may be
 * NULL, grads NULL gives the losses alone).  A lattice's results equal those of a context that
 * holds it alone, bit for bit.  Device memory: as above, for the states of the whole batch. */
int lb_pressure_shift_gradient_batch(lb_ctx* ctx, int64_t steps, int64_t ckpt_every, double* grads,
                                     double* losses);

/* Clear the structure-factor and pressure accumulators (the step count is kept). */
int lb_reset_statistics(lb_ctx* ctx);

/* Checkpoint and resume (the paper's averages are taken over long stationary runs, Sec. III and
 * Appendix A; this lets such a run stop and continue).  A checkpoint holds the context's whole
 * dynamic state: the stored populations of every lattice (storage type), the step count (which
 * keys the noise), the site maps, the sampling and correlation settings, and every accumulator
 * (structure factors, profiles, correlations, pressure and mass statistics, sample counts).
 * lb_checkpoint_bytes gives its size for the context as it is now; lb_save_checkpoint writes it to
 * a caller-owned host buffer of exactly that many bytes (LB_ERR_SIZE otherwise), after the
 * context's pending work; lb_load_checkpoint restores one into a context created with the same
 * lattices (parameters, seeds, ids) and the same result-affecting flags (precision, a*, wall
 * rule, noise) -- LB_ERR_STATE otherwise, LB_ERR_BAD_PARAM for a buffer that is not a checkpoint
 * of this format.  The launch flags (graphs, persistent launch, tile) may differ: a resumed run
 * then reproduces the uninterrupted one bit for bit, except that another tile groups the
 * double-precision pressure sums differently (a few units in the last place).  Synchronous. */
int lb_checkpoint_bytes(lb_ctx* ctx, size_t* bytes);
int lb_save_checkpoint(lb_ctx* ctx, void* host_buf, size_t bytes);
int lb_load_checkpoint(lb_ctx* ctx, const void* host_buf, size_t bytes);

/* Number of kernels lb_step has enqueued on the device so far (every step kernel, every
 * diagnostics kernel, every step-counter update; kernels inside replayed graphs included). */
int lb_kernel_launches(lb_ctx* ctx, int64_t* n);

/* Bytes of device memory held by the context. */
int lb_device_bytes(lb_ctx* ctx, size_t* bytes);

const char* lb_error_string(int code);
void lb_destroy(lb_ctx* ctx);

/* Test hook for the bounded waits of LB_PERSISTENT (an item waits until the items around it
 * have completed the previous step): launches a grid of `blocks` co-resident blocks; each marks
 * itself done and waits until blocks 0 .. expected-1 are.  With expected > blocks the wait must
 * give up after spin_limit milliseconds and the call returns LB_ERR_TIMEOUT; with expected <=
 * blocks it returns LB_OK.  1 <= blocks, expected <= 64 and 1 <= spin_limit <= 10000, else
 * LB_ERR_BAD_PARAM. */
int lb_debug_barrier(int blocks, int expected, int spin_limit);

/* Host-only test hook (needs no GPU) for the work decomposition of lb_create_batch and the
 * dependency lists of LB_PERSISTENT: for n_lat lattices of Lx[i] x Lz[i] sites (>= 1 each, at
 * most 2^26 sites in all) cut into items of tile_x columns x `rows` rows, items_out receives 4
 * ints per item (lattice, x0, z0, z1: columns x0 .. x0 + tile_x - 1 clipped to Lx, rows z0 ..
 * z1 - 1) in launch order, off_out n_items + 1 offsets and nbr_out the item indices each item
 * waits for in the persistent launch (nbr_out[off_out[i] .. off_out[i + 1])).  *n_items and
 * *n_nbr are always set; buffers smaller than those (items_cap in items, nbr_cap in indices)
 * return LB_ERR_SIZE without writing them, so a first call with zero capacities sizes them.
 * All buffers are caller-owned host memory; off_out holds n_items + 1 ints. */
int lb_debug_schedule(int n_lat, const int* Lx, const int* Lz, int tile_x, int rows, int* items_out,
                      int64_t items_cap, int* off_out, int* nbr_out, int64_t nbr_cap, int64_t* n_items,
                      int64_t* n_nbr);

/* Test hook for the Gaussian noise of the step kernels (Sec. II.B): the Box-Muller normals that
 * the kernels of precision `precision` (LB_PREC_FP64 or LB_PREC_DEV32) form from Philox word
 * pairs.  host_words: 2 n_pairs words (a_0, b_0, a_1, b_1, ...), u1 from a_i sets the radius
 * sqrt(-2 ln u1) and u2 from b_i the angle 2 pi u2, with u = (2 (k mod 2^23) + 1) 2^-24;
 * host_out: 2 n_pairs doubles, the pair (r cos 2 pi u2, r sin 2 pi u2) of each.  Both buffers are
 * caller-owned host memory; 0 <= n_pairs <= 2^24, else LB_ERR_BAD_PARAM.  Synchronous. */
int lb_debug_box_muller(int precision, const uint32_t* host_words, int64_t n_pairs, double* host_out);

/* Measurement aid (the paper has no counterpart): the fused multiply-add rate of the current
 * device in flops per second (2 per FMA), LB_PREC_FP64 for double and LB_PREC_DEV32 for float
 * scalar FMAs, from a kernel of eight independent FMA chains per thread over 8 blocks of 256
 * threads per SM, best of five timed launches after a warm-up; the ceiling against which the
 * FP64 path, bound by its double-precision arithmetic, is measured.  Synchronous; allocates and
 * frees a scratch of 8 bytes per thread. */
int lb_debug_fma_rate(int precision, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif
