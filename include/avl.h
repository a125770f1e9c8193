/*
 * avl.h -- C ABI of the GB300 library for the Vlasov-Hybrid (VHS) time step.
 *
 * One time step follows Fig. 2 of the paper: reconstruct the phase-space
 * density f of every species on its (x, v) grid from the markers (Sec. 2,
 * Eq. 4), take the velocity moment rho (Eq. 14), solve Poisson's equation
 * spectrally for E (Sec. 3.1, Eq. 5 / Eq. 6a-c), gather E at every marker
 * with the same cloud-in-cell weights and push the markers (Sec. 2).  All of
 * it runs in hand-written sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Units and conventions
 *   - Normalised units by default: Poisson reads dE/dx = poisson_const * rho
 *     (poisson_const = 1 normalised, 4 pi for the paper's CGS form, Eq. 2).
 *   - x spans [0, L) in nx cells of width dx = L/nx, periodic.  Velocity
 *     dimension d of species s spans [vmin[d], vmax[d]) in nv[d] cells
 *     (Sec. 3.1, Fig. 3).  Grid values sit at cell centres.
 *   - Phase-space arrays returned to the caller are row-major
 *     [x][vx] (1d1v) or [x][vx][vy][vz] (1d3v), FP64.
 *   - Marker arrays are structure-of-arrays, FP64: x[n], v[nvdim][n]
 *     (component-major), f[n].  The library keeps markers binned in its own
 *     order; avl_get_markers returns them in that (unspecified) order.
 *
 * Ownership and errors
 *   - A context owns all its device memory; the caller owns every buffer it
 *     passes.  No call frees or retains caller memory.
 *   - Every call returns an avl_status and never aborts; avl_last_error gives
 *     a message for the last failing call on that context.
 *   - Work is enqueued on the context's CUDA stream in call order.  Calls with
 *     on_device = 0 (host buffers) return after the copy has completed; calls
 *     with on_device = 1 only enqueue the copy on the context stream.
 *   - A context is not thread-safe.  One context uses one GPU (the device
 *     current at avl_create).
 */
#ifndef AVL_H
#define AVL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AVL_OK = 0,
    AVL_EINVAL = 1,    /* bad argument: the message names it */
    AVL_ENOMEM = 2,    /* device allocation failed */
    AVL_ECUDA = 3,     /* CUDA runtime error: the message carries the CUDA text */
    AVL_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    AVL_ESTATE = 5,    /* call not valid in the context's current state */
    AVL_ENUMERIC = 6   /* NaN or Inf found in the fields or diagnostics */
} avl_status;

enum { AVL_FP64 = 0, AVL_FP32 = 1 };
enum { AVL_MAX_SPECIES = 8 };

typedef struct avl_ctx avl_ctx;

/* Simulation domain (Sec. 3.1, Sec. 3.3 numerical parameters).
 * precision AVL_FP64: markers, deposit and grid in FP64.
 * precision AVL_FP32: marker position = int32 cell + FP32 offset, velocity
 *   and value in FP32, deposit sums in FP32 (1d1v: the numerator as
 *   deviations from the previous reconstruction within a chunk, float-float
 *   over chunks, f = num / den in float-float; 1d3v: plain); the Poisson
 *   solve, the charge-neutral k = 0 handling and the diagnostics stay FP64.
 * nvdim = 1: one chunk's deposit window (at least 7 velocity rows x nx
 *   cells, 12 B per cell in FP32, 16 B in FP64) must fit one CTA's shared
 *   memory, which bounds nx near 2400 (FP32) / 1800 (FP64); beyond it
 *   avl_init_markers and avl_set_markers return AVL_EINVAL.  FP64 marker
 *   positions are kept as 64-bit fixed-point counts of 2^-52 cells (in
 *   both dimensions), which also needs nx < 2048.
 * nvdim = 3 (Sec. 2 with three velocity dimensions: the field accelerates
 *   v_x, an optional static background magnetic field, avl_set_bfield, turns
 *   v) needs nx <= 1024 (FP32) or nx <= 512 (FP64), nv[0] in [2, 1024],
 *   nv[1], nv[2] in [2, 4096] and fewer than 2^31 grid cells; all species of
 *   a context share nvdim. */
typedef struct {
    int32_t nvdim;          /* 1 (1d1v) or 3 (1d3v) */
    int32_t nx;             /* cells in x, >= 4 */
    double L;               /* domain length */
    double dt;              /* time step */
    double poisson_const;   /* 1 normalised, 4 pi CGS */
    int32_t softening;      /* 1: Eq. 6 (sinc-softened), 0: Eq. 5 */
    int32_t precision;      /* AVL_FP64 or AVL_FP32 */
} avl_domain;

/* One species (Sec. 3.3): charge and mass of a physical particle, velocity
 * grid.  mobile = 0 makes a fixed background: never pushed, its density is
 * reconstructed once and keeps contributing to rho. */
typedef struct {
    double q;
    double m;
    int32_t mobile;
    int32_t nv[3];          /* nv[1] = nv[2] = 1 for 1d1v */
    double vmin[3];
    double vmax[3];
} avl_species;

/* Initial distribution (Sec. 3.3, Eq. 11; Eq. 17):
 *   f0(x, v) = sum_b beam_n[b] prod_d M(v_d; beam_u[b][d], beam_vth[b][d])
 *              * (1 + sum_m amp[m] cos(2 pi mode[m] x / L + phase[m])),
 *   M(v; u, s) = exp(-(v-u)^2 / (2 s^2)) / (sqrt(2 pi) s). */
typedef struct {
    int32_t nbeam;          /* 1..4 */
    double beam_n[4];
    double beam_u[4][3];
    double beam_vth[4][3];
    int32_t nmode;          /* 0..64 */
    int32_t mode[64];
    double amp[64];
    double phase[64];
} avl_f0;

/* Create a context for nspecies species (1..AVL_MAX_SPECIES) on the current
 * device.  cuda_stream: a cudaStream_t to enqueue all work on, or NULL to let
 * the context create its own non-blocking stream.  Errors: AVL_EINVAL for an
 * unsupported shape (message says which), AVL_ENOMEM. */
avl_status avl_create(const avl_domain* dom, const avl_species* sp, int32_t nspecies,
                      void* cuda_stream, avl_ctx** out);

/* Release all device memory of the context (after draining its stream).
 * NULL is ignored; a run of a batch is released with its batch. */
void avl_destroy(avl_ctx* ctx);

/* Message for the last failing call on ctx ("" if none).  ctx may be NULL,
 * in which case the message of the last failing avl_create is returned. */
const char* avl_last_error(const avl_ctx* ctx);

/* Marker creation (Sec. 2; Sec. 3.1): lattice[0..3] = markers per cell
 * along x, vx, vy, vz (ppc = product; lattice[2] = lattice[3] = 1 for 1d1v).
 * Marker (cell, sub-point) sits at the centre of its sub-cell plus a jitter
 * uniform in [-jitter/2, jitter/2) sub-cells per dimension, drawn from
 * SplitMix64 with stream index (species << 48) | (4 * marker + dim), marker =
 * cell * ppc + sub-point (row-major indices).  Marker value f_l = f0 at the
 * marker.  Then f, rho and E are recomputed for the new markers.
 * Errors: AVL_EINVAL (bad species, lattice, or f0 counts; jitter outside
 * [0, 1]), AVL_ENOMEM. */
avl_status avl_init_markers(avl_ctx* ctx, int32_t s, const int32_t lattice[4],
                            const avl_f0* f0, uint64_t seed, double jitter);

/* Replace the markers of species s by n caller markers (FP64, layout above,
 * x in [0, L)); on_device selects device or host pointers.  Then f, rho and E
 * are recomputed.  Errors: AVL_EINVAL (n <= 0 or too large, x outside [0, L),
 * non-finite values), AVL_ENOMEM. */
avl_status avl_set_markers(avl_ctx* ctx, int32_t s, int64_t n, const double* x,
                           const double* v, const double* f, int32_t on_device);

/* Number of markers of species s.  Errors: AVL_EINVAL (species index out of
 * range, NULL n). */
avl_status avl_marker_count(avl_ctx* ctx, int32_t s, int64_t* n);

/* Copy the markers of species s out as FP64 (layout above, library order).
 * Errors: AVL_EINVAL (species index out of range), AVL_ESTATE (no markers). */
avl_status avl_get_markers(avl_ctx* ctx, int32_t s, double* x, double* v, double* f,
                           int32_t on_device);

/* Advance nsteps full time steps (Fig. 2): gather + push of every mobile
 * species, reconstruction (Eq. 4), moment (Eq. 14), Poisson (Eq. 6), and the
 * diagnostics of the new state.  Enqueued asynchronously (a CUDA graph per
 * step).  Errors: AVL_ESTATE if a mobile species has no markers. */
avl_status avl_step(avl_ctx* ctx, int32_t nsteps);

/* Field history for marker refinement (not used by the step itself): from
 * this call on, the electric field of every state (E after each step, or
 * after a re-creation of markers) is kept in a device buffer of
 * (max_steps + 1) x nx FP64 values that the call allocates (the previous one
 * is freed); slot 0 takes the current E.  Call it before avl_init_markers of
 * the species to be refined.  Errors: AVL_EINVAL (max_steps outside
 * [1, 2^24], a batch), AVL_ENOMEM. */
avl_status avl_record_history(avl_ctx* ctx, int32_t max_steps);

/* Marker refinement by tracing back to the initial state (Sec. 2: markers of
 * very different weight can share a cell; a phase-space patch that needs more
 * resolution later is traced back to the initial state and given more
 * markers there), 1d1v.  Adds lattice[0] x lattice[1] markers in every cell
 * of the box [box[0], box[1]) x [box[2], box[3]) (x cells x velocity rows) of
 * species s at the current time, on the jittered sub-lattice of
 * avl_init_markers (seed and jitter as there; use a seed other than the
 * creation's).  Each new marker is traced back to the species' creation by
 * the inverse of the kick-drift step, x_n = x_{n+1} - v_{n+1} dt (periodic),
 * v_n = v_{n+1} - (q/m) dt E^n(x_n), through the recorded fields, and takes
 * f = f0 (the creation's f0) at the foot; f is constant along
 * characteristics, and the reconstruction of Eq. 4 weighs denser markers by
 * their overlap only.  The species is then re-laid out and f, rho and E are
 * recomputed for the enlarged marker set (as avl_set_markers does).  The
 * adjoint is no longer available for the species (its markers are not the
 * creation lattice).  *added_opt (if not NULL) receives the number added.
 * Errors: AVL_EINVAL (nvdim 3, box outside the grid, lattice < 1 or more than
 * 4096 points, jitter outside [0, 1], 2^31 markers), AVL_ESTATE (markers not
 * from avl_init_markers, or no history covering every step since their
 * creation). */
avl_status avl_refine_markers(avl_ctx* ctx, int32_t s, const int32_t* box, const int32_t* lattice, uint64_t seed,
                              double jitter, int64_t* added_opt);

/* Static background magnetic field B = (B_x, B_y, B_z) of a 1d3v context
 * (Sec. 3.2: the full Boris push of the 1d3v version; Sec. 3.3: the time step
 * should resolve a gyration with at least 2 pi steps).  From the next step on,
 * every mobile species is pushed by the Boris scheme: half kick by E_x at the
 * marker's position, rotation of v about B by the angle 2 atan(|t|),
 * t = (q/m)(dt/2) B, half kick, x += v_x dt; the force is q (E + v x B) in
 * the library's units (CGS users pass B / c).  B = (0, 0, 0) returns to the
 * field-free push.  A magnetized step pushes, re-sorts every marker by its
 * (v_y, v_z, v_x) dual rows into the other buffer and then deposits, so it
 * costs about three times a field-free step.  The stored state (markers, f,
 * rho, E) is not changed by the call.  Errors: AVL_EINVAL (nvdim 1, B NULL or
 * not finite). */
avl_status avl_set_bfield(avl_ctx* ctx, const double* B);

/* Reconstructed f of species s and, if n_opt is not NULL, the denominator of
 * Eq. 4 (sum of weights, the paper's "n" output, Sec. 3.4.3); FP64,
 * [x][v...] row-major.  Errors: AVL_EINVAL (species index out of range,
 * NULL f), AVL_ENOMEM (host reads stage through a scratch buffer). */
avl_status avl_get_f(avl_ctx* ctx, int32_t s, double* f, double* n_opt, int32_t on_device);

/* Net charge density rho (nx, FP64) of the current state (Eq. 14).
 * Errors: AVL_EINVAL (NULL rho, a batch: its runs hold the fields). */
avl_status avl_get_rho(avl_ctx* ctx, double* rho, int32_t on_device);

/* Electric field E (nx, FP64) of the current state (Eq. 6).
 * Errors: AVL_EINVAL (NULL E, a batch). */
avl_status avl_get_E(avl_ctx* ctx, double* E, int32_t on_device);

/* Velocity moments of species s of the current state (Sec. 3.4.2 outputs,
 * not used by the step; formed on demand from the stored f with the
 * midpoint rule of Eq. 14): out = (2 + nvdim) rows of nx FP64 values,
 * row-major: rho_s = q sum f dv, j_x = q sum v_x f dv, (1d3v: j_y, j_z),
 * M2 = q sum |v|^2 f dv (the trace of the second moment, q n <v^2>).
 * Errors: AVL_EINVAL (species index, NULL out). */
avl_status avl_get_moments(avl_ctx* ctx, int32_t s, double* out, int32_t on_device);

/* Residual charge of the field solve of the current state (Sec. 3.4.2):
 * drho_i = rho_i - (E_{i+1} - E_{i-1}) / (2 dx poisson_const), periodic,
 * nx FP64 values.  Nonzero even for an exact solve, from the centred
 * difference and the softening of Eq. 6.  Errors: AVL_EINVAL (NULL out, a
 * batch). */
avl_status avl_get_residual(avl_ctx* ctx, double* out, int32_t on_device);

/* Diagnostics of the current state (Sec. 3.4.1, FP64, host buffer of
 * 3 + 3 * nspecies values): W_E, W_kin, W_total, then W_kin of each species,
 * N (integral of f) of each species, entropy S of each species.
 * W_E = 1/(2 poisson_const) sum E^2 dx (Eq. 12); W_kin = m/2 sum v^2 f dx dv.
 * Returns AVL_ENUMERIC if any value is NaN or Inf, AVL_EINVAL for a NULL out
 * or a batch (its runs hold the rows). */
avl_status avl_get_diag(avl_ctx* ctx, double* out);

/* The same diagnostics row, copied to the host buffer out (3 + 3 * nspecies
 * FP64 values; page-locked host memory keeps the copy asynchronous) in
 * stream order behind the steps enqueued so far, without waiting: out holds
 * the row of the current state once the context's stream has drained
 * (avl_synchronize).  The caller keeps out valid until then and checks the
 * values itself (avl_synchronize reports AVL_ENUMERIC for a non-finite
 * field energy or species sum).  Errors: AVL_EINVAL (NULL out, a batch),
 * AVL_ECUDA. */
avl_status avl_get_diag_async(avl_ctx* ctx, double* out);

/* Counters (host buffer of 4 int64 per species): [0] 1d1v: runs of markers
 * that deposited through the out-of-window path in the last step; 1d3v:
 * markers whose v_x dual row had left their segment's in the last step;
 * [1] steps that re-sorted this species so far; [2] 1d1v: markers outside
 * their chunk's best window at the last decision, 1d3v: 0; [3] steps so
 * far.  Errors: AVL_EINVAL (NULL out). */
avl_status avl_get_stats(avl_ctx* ctx, int64_t* out);

/* Stand-alone spectral Poisson solve (Sec. 3.1, Eq. 5 / Eq. 6a-c): E from
 * rho on a periodic grid of nx cells over length L, k = 0 and Nyquist modes
 * removed.  rho and E are device pointers to nx FP64 values (E may not alias
 * rho); the work runs on cuda_stream (NULL: the legacy default stream).  The
 * transform tables live in scratch memory that the call allocates with
 * cudaMalloc and frees before returning; the call returns after the solve
 * has completed.  Errors (message via avl_last_error(NULL)): AVL_EINVAL for
 * nx outside [4, 65536] (or more shared memory than one block holds),
 * non-positive L or poisson_const, NULL pointers; AVL_ENOMEM; AVL_ECUDA. */
avl_status avl_field_solve(int32_t nx, double L, double poisson_const, int32_t softening,
                           const double* rho, double* E, void* cuda_stream);

/* Allocation-free variant of avl_field_solve; the paper has no counterpart.
 * For callers that cannot allocate device memory when they need a field
 * solve: their GPU memory is fully reserved by another allocator (a caching
 * allocator, a fixed budget), or they run a time-critical loop that must not
 * pay for cudaMalloc/cudaFree, which synchronise the device.  The transform
 * tables live in one file-scope device array of 250 KiB, sized for the
 * largest grid one block's shared memory can solve (nx <= 12798; power-of-two
 * grids up to 8192).  The call itself allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The CUDA runtime loads the
 * library's device code lazily: the array (and the solve's kernels) are
 * placed on a device by the first call there, which looks up the array's
 * device address (cudaGetSymbolAddress, with that device current).  Make
 * that first call on each device before reserving the rest of its memory
 * and before any stream capture; every later call finds them in place (the
 * address is looked up again on every call, which allocates nothing once
 * the code is loaded), and they stay until the process exits.  Same
 * arguments and result as avl_field_solve, but the work is only enqueued on
 * cuda_stream (the call does not wait for it).  Every call on a device
 * shares the array and rewrites the part it uses before reading it, so no
 * state carries over between calls; calls that overlap on the GPU (other
 * streams, other host threads) race on it.  Errors (message via
 * avl_last_error(NULL)): AVL_EINVAL for nx outside [4, 12798] and the
 * argument errors of avl_field_solve; AVL_ECUDA. */
avl_status avl_field_solve_noalloc(int32_t nx, double L, double poisson_const, int32_t softening,
                                   const double* rho, double* E, void* cuda_stream);

/* Gradient of the field energy at the final time (an extension beyond the
 * paper, which has no adjoint): J = 1/2 sum_i E_i(T)^2 dx after nsteps steps that
 * start from the markers each species got from its last avl_init_markers,
 * with the f0 of species s replaced by theta.  Outputs (host): *J,
 * dJ_damp[m] = dJ/d theta->amp[m] (theta->nmode values) and dJ_ddrift[b] =
 * dJ/d theta->beam_u[b][0] (theta->nbeam values).  The discrete adjoint of
 * the step (push, Eq. 4 reconstruction, Eq. 14 moment, Eq. 6 Poisson) runs
 * backwards over the step history, recomputed segment by segment from
 * checkpoints of the markers taken every ckpt_every steps; its device memory
 * (about (ckpt_every + 1) marker states and grids, plus one marker state per
 * checkpoint) is kept by the context for the next call.  The context's own
 * markers, f, rho and E are left untouched.  Blocks until done.  1d1v only.
 * Errors: AVL_EINVAL (nvdim 3, NULL pointers, nsteps < 0, ckpt_every < 1,
 * theta counts, FP64 with nx >= 2048: its positions are fixed-point counts
 * of 2^-52 cells), AVL_ESTATE (a species without lattice markers),
 * AVL_ENOMEM. */
avl_status avl_adjoint(avl_ctx* ctx, int32_t s, const avl_f0* theta, int32_t nsteps, int32_t ckpt_every,
                       double* dJ_damp, double* dJ_ddrift, double* J);

/* Batched ensemble (an extension beyond the paper, which runs one simulation
 * at a time): nrun independent 1d1v runs of any sizes, run r with domain doms[r]
 * and the nspecies[r] species that follow in sps (runs' species listed one
 * run after another).  All runs share one precision and the batch's stream
 * (cuda_stream, or one the batch creates).  avl_step on the batch advances
 * every run by one launch per kernel class (push + deposit, finalize,
 * field) for all runs together, recorded as one CUDA graph per step; all
 * other calls go to the runs, obtained with avl_batch_run (owned by the
 * batch: avl_destroy on a run does nothing, avl_destroy on the batch frees
 * every run).  avl_synchronize on the batch reports the first run's error.
 * Errors: AVL_EINVAL (nrun outside [1, 4096], nvdim 3, mixed precision, or
 * a run's own avl_create error, message prefixed with the run), AVL_ENOMEM. */
avl_status avl_create_batch(int32_t nrun, const avl_domain* doms, const avl_species* sps, const int32_t* nspecies,
                            void* cuda_stream, avl_ctx** out);

/* Run r of a batch (a context for every per-run call).  Errors: AVL_EINVAL
 * (NULL batch or run, r out of range). */
avl_status avl_batch_run(avl_ctx* batch, int32_t r, avl_ctx** run);

/* Chunk-size autotuner of the 1d1v path (a single context or a batch):
 * snapshots every marker set, times trial_steps steps (after two untimed
 * ones) for markers-per-chunk M in {heuristic, 1024, 2048, 4096, 8192,
 * 16384}, keeps the fastest and restores the snapshot, so the state is that
 * of the call (re-sorted, f, rho and E reconstructed; afterwards the markers
 * count as caller markers for avl_adjoint).  *chunk_out = the chosen M (0:
 * the heuristic).  Blocks until done.  Errors: AVL_EINVAL (trial_steps < 1,
 * 1d3v), AVL_ESTATE as avl_step, AVL_ENOMEM (snapshot: 24 B per marker). */
avl_status avl_autotune(avl_ctx* ctx, int32_t trial_steps, int32_t* chunk_out);

/* Per-kernel timing (the paper's time breakdown, Sec. 3.2): advance nsteps
 * steps exactly as avl_step does, but launched kernel by kernel with CUDA
 * events recorded on the context stream around each kernel; writes the summed
 * milliseconds of each kernel class into ms[0..3] = {1d1v: re-sort scatter,
 * 1d3v: pencil re-sort (with a magnetic field: Boris push + global
 * re-sort); push + deposit (deposit only in a magnetized 1d3v step);
 * finalize (f, moment, diagnostics); field (Poisson)}.  Blocks until done.
 * Errors: AVL_EINVAL (nkernels < 4 or ms NULL), AVL_ESTATE as avl_step. */
avl_status avl_profile_steps(avl_ctx* ctx, int32_t nsteps, double* ms, int32_t nkernels);

/* Block the host until the context's stream has drained; reports device-side
 * error flags (AVL_ETIMEOUT, AVL_ENUMERIC) raised by the work enqueued so far
 * and clears them, so that each flag is reported once.  On a batch: the
 * first run's error. */
avl_status avl_synchronize(avl_ctx* ctx);

/* Failure detection (an extension beyond the paper, which has no counterpart):
 * the deposit kernels stage marker fields and E with bulk copies (TMA) and
 * wait for them on an mbarrier at most `polls` polls (default 2^22, about a
 * second); a wait that gives up sets the AVL_ETIMEOUT flag, drains the copy
 * with the default limit (so no copy is left in flight) and the step goes
 * on.  polls = 0 makes every such wait give up at once, which forces the
 * failure path without any fault (a test of the host's error handling: the
 * step's results stay valid, the next avl_synchronize returns AVL_ETIMEOUT);
 * polls < 0 restores the default.  On a batch: every run.  Errors:
 * AVL_EINVAL (NULL ctx), AVL_ECUDA. */
avl_status avl_set_wait_limit(avl_ctx* ctx, int64_t polls);

#ifdef __cplusplus
}
#endif
#endif
