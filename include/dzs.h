/*
 * dzs.h -- C ABI of the GB300-native Dynamic Zoom Simulations TreePM step.
 *
 * Paper: Garaldi, Nori & Baldi, "Dynamic Zoom Simulations: a fast, adaptive
 * algorithm for simulating lightcones", arXiv 2005.05328.
 *
 * Problem statement (paper Sec. 1 footnote and Sec. 2.2.1): given initial
 * conditions, a cosmology, an observer at the box centre and the DZS
 * parameters (theta_dzs, buffer b, maximum node size l_max), evolve the
 * particles to z = 0 with TreePM gravity (Sec. 2.1), output every particle
 * once as the lightcone R_lc(a) sweeps it (Sec. 3.1.3), and de-refine the
 * particles outside R_lc + b by merging oct-tree nodes into centre-of-mass
 * particles (Sec. 2.2, Eq. 3).
 *
 * Conventions of every entry point
 *   - Positions are uint32 lattice coordinates u = floor(x / L * 2^32) per
 *     axis, stored SoA: u[0..n) is x, u[n..2n) is y, u[2n..3n) is z.  The
 *     observer sits at u = 2^31 on each axis.  Momenta p = a^2 dx/dt and
 *     accelerations g are SoA [3][n] in Mpc/h units with H0 = 1, always
 *     exchanged as double (converted on the device in DZS_FP32 mode).
 *   - Masses are uint32 multiplicities k of the base mass m0
 *     (4 pi G m0 = 1.5 Omega_m L^3 / N0, N0 = n1d^3).
 *   - Host pointers are caller-owned host memory; the context owns all device
 *     memory (one cudaMalloc'd arena per context) and its CUDA stream use.
 *   - Every call returns a dzs_status; errors never abort the process.
 *     DZS_EDEVICE / DZS_ETIMEOUT poison the context (only dzs_destroy is then
 *     valid).  dzs_last_error() gives a message for the last failure.
 *   - dzs_step enqueues on the context stream and returns; calls that return
 *     host data (drain, get_state, diagnostics, accel, ...) synchronise it.
 *   - One context is used by one host thread at a time.
 */
#ifndef DZS_H
#define DZS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DZS_API __attribute__((visibility("default")))
#else
#define DZS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dzs_ctx dzs_ctx;

typedef enum {
  DZS_OK = 0,
  DZS_EINVAL = 1,    /* invalid argument or parameter set */
  DZS_ENOMEM = 2,    /* device or host allocation failed */
  DZS_ECUDA = 3,     /* a CUDA runtime call failed (message in dzs_last_error) */
  DZS_EOVERFLOW = 4, /* a device buffer filled up (tree nodes, walk stack, lightcone ring) */
  DZS_ETIMEOUT = 5,  /* a bounded device wait gave up */
  DZS_ESTATE = 6,    /* call not valid in the context's current state */
  DZS_EDEVICE = 7    /* no usable CUDA device / unsupported architecture */
} dzs_status;

enum { DZS_RLC_SWEEP = 0, DZS_RLC_PHYSICAL = 1 };
enum { DZS_FP32 = 0, DZS_FP64 = 1 };
enum { DZS_CRIT_GEOMETRIC = 0, DZS_CRIT_DYNAMICAL = 1 };
enum { DZS_WALK_AUTO = 0, DZS_WALK_MASKED = 1, DZS_WALK_GUARDED = 2 };

/* flag bits of a particle */
enum { DZS_FL_CROSSED = 1, DZS_FL_MERGED = 2 };

/* stage bits for dzs_run_stages */
enum {
  DZS_STAGE_KICK_DRIFT = 1, /* opening kick, drift, crossing test, Morton keys, records */
  DZS_STAGE_SORT = 2,       /* stable radix sort of the keys + state permutation */
  DZS_STAGE_MERGE = 4,      /* DZS merge against R_lc(a_step+1) (only if dzs_on); the
                               dynamical criterion takes a_min from the kick-drift stage
                               of the same step (DZS_ESTATE if the state was sorted
                               since its accelerations were computed without one) */
  DZS_STAGE_FORCE = 8,      /* tree build, PM, tree walk: g of the current particles */
  DZS_STAGE_CLOSE = 16,     /* closing kick p += g K(a_step+1/2, a_step+1) */
  DZS_STAGE_ALL = 31
};

/* parts for dzs_accel */
enum { DZS_ACC_PM = 1, DZS_ACC_TREE = 2, DZS_ACC_ALL = 3 };

/* mesh selectors for dzs_get_mesh */
enum { DZS_MESH_DELTA = 0, DZS_MESH_PHI = 1 };

typedef struct {
  int32_t n1d;          /* particles per side at the start, N0 = n1d^3 (power of two, 8..512) */
  int32_t mesh;         /* PM mesh points per side M (power of two, 16..512) */
  double box;           /* L [Mpc/h] */
  double omega_m, omega_l, hubble, sigma8, ns;
  double z_init;        /* initial redshift (49) */
  int32_t nsteps;       /* global KDK steps, uniform in ln a to a = 1 */
  int32_t leaf_bucket;  /* B: leaf holds <= B particles (physics parameter) */
  int32_t walk_group;   /* G: walk group size bound, 32 (physics parameter) */
  int32_t dzs_on;       /* 1: DZS merge every step */
  int32_t merge_level;  /* l_max = 2^(merge_level-1) * L / n1d */
  int32_t rlc_mode;     /* DZS_RLC_SWEEP | DZS_RLC_PHYSICAL */
  double rs_cells;      /* PM split scale r_s in mesh cells (1.25) */
  double rcut_rs;       /* short-range cut r_cut / r_s (4.5) */
  double theta;         /* force-walk opening angle, Eq. 1 (0.5) */
  double soft_frac;     /* eps0 / (L / n1d) (1/40) */
  double theta_dzs;     /* DZS geometric merge angle, Sec. 2.2.1 (0.1) */
  double buffer_cells;  /* buffer b of Eq. 3 in mesh cells (2) */
  uint64_t seed;        /* IC white-noise seed */
  int32_t precision;    /* DZS_FP32 | DZS_FP64 force arithmetic */
  int32_t device;       /* CUDA device ordinal */
  uint64_t lc_capacity; /* lightcone ring records; 0 = N0 (never overflows); a smaller
                          ring makes dzs_step check each step's records first */
  int32_t dzs_criterion; /* DZS_CRIT_GEOMETRIC: l/D < theta_dzs (Sec. 2.2.1);
                           DZS_CRIT_DYNAMICAL: Eq. 2 with d -> D of Eq. 3 */
  int32_t walk_eval;     /* execution only (results identical): how the tree walk
                            evaluates its lists; DZS_WALK_AUTO (0), DZS_WALK_MASKED
                            (1: a range-test pass, then force arithmetic for the
                            pairs within r_cut), DZS_WALK_GUARDED (2: one pass, the
                            arithmetic guarded by the range test) */
  double alpha_dyn;      /* dynamical: merge iff D > 0 and G M l^2 / D^4 <
                            alpha_dyn a_min, a_min = smallest |g| (previous
                            step) of the particles not yet crossed; >= 0 */
  uint64_t capacity;     /* particle slots of the context, <= N0; 0 = N0.  dzs_ics
                            needs N0; a smaller context takes a restored or
                            injected state of up to `capacity` particles (the
                            re-allocation after a halt, dzs_step_until) */
} dzs_params;

/* one lightcone record: particle id and multiplicity, crossing expansion
 * factor a*, comoving position x* [Mpc/h] in [0, L) and momentum p (64 bytes) */
typedef struct {
  uint32_t id, k;
  double a_cross;
  double x[3];
  double p[3];
} dzs_lc_record;

/* Fill *p with the configuration-1 defaults of the paper's method
 * (32^3 particles in 64 Mpc/h, mesh 64, r_s = 1.25 cells, r_cut = 4.5 r_s,
 * theta = 0.5, eps0 = lambda/40, DZS on, merge level 2, theta_dzs = 0.1,
 * b = 2 cells, 96 steps from z = 49, FP32).  Returns DZS_EINVAL if p is NULL. */
DZS_API dzs_status dzs_params_default(dzs_params* p);

/* Device bytes a context with these parameters allocates (for admission by
 * memory budget).  DZS_EINVAL on an invalid parameter set. */
DZS_API dzs_status dzs_footprint_bytes(const dzs_params* p, size_t* bytes);

/* Validate p, compute the FP64 host tables (time integrals, R_lc), allocate
 * the device arena on p->device and bind cuda_stream (a cudaStream_t; NULL =
 * the legacy default stream).  On success *out owns everything; the particle
 * state is empty until dzs_ics or dzs_set_state. */
DZS_API dzs_status dzs_create(const dzs_params* p, void* cuda_stream, dzs_ctx** out);

/* Zel'dovich initial conditions at z_init from the seeded Gaussian field
 * (paper Fig. 1 caption: linear theory to z ~ 50), initial lightcone flags
 * (PHYSICAL mode), Morton sort and the first accelerations.  Step index 0. */
DZS_API dzs_status dzs_ics(dzs_ctx* c);

/* Enqueue up to nsteps full KDK steps (DZS_STAGE_ALL), stopping at a = 1.
 * *steps_done (nullable) receives the number enqueued.  With a lightcone ring
 * smaller than N0 (lc_capacity), each step first counts the records it will
 * write (a dry run of its kick, drift and crossing test; synchronises); if
 * they do not fit in the ring's room, the step is not started and
 * DZS_EOVERFLOW is returned (recoverable: drain, then call dzs_step again,
 * which resumes with that step; *steps_done counts the steps enqueued before
 * it).  With the default ring nothing is checked and no record is ever lost. */
DZS_API dzs_status dzs_step(dzs_ctx* c, int32_t nsteps, int32_t* steps_done);

/* Run the stages in stage_mask of the current step in stage order, without
 * advancing the step index unless DZS_STAGE_CLOSE is included.  Used for
 * per-stage parity tests and timing. */
DZS_API dzs_status dzs_run_stages(dzs_ctx* c, uint32_t stage_mask);

/* Copy the lightcone records written since the last drain (in step order,
 * within a step in the particle order at crossing) into host_buf, at most cap
 * of them; *n_out = number copied.  Remaining records stay for the next
 * drain.  Returns DZS_EOVERFLOW if records were dropped because the ring was
 * full (the count of kept records is still valid). */
DZS_API dzs_status dzs_lightcone_drain(dzs_ctx* c, dzs_lc_record* host_buf, size_t cap, size_t* n_out);

/* Pipelined per-step results (a serving convenience; Sec. 2.1 global steps,
 * Sec. 2.2 the conserved totals): with on != 0, every step dzs_step runs ends
 * by enqueueing its conservation diagnostics (as dzs_diagnostics), the
 * lightcone ring counters and the device error word into pinned host memory
 * the context owns, behind the step's kernels on the context stream, so that
 * the caller can read step s while step s + 1 runs.  The last 4 steps are
 * kept (a step's slot is reused 4 steps later, after its copies landed).
 * on = 0 waits for the stream and turns it off.  Errors as dzs_step. */
DZS_API dzs_status dzs_pipeline(dzs_ctx* c, int32_t on);

/* Result of step `step` (the number of steps completed, as dzs_get_count
 * reports after it): diag[8] as dzs_diagnostics, *lc_written = lightcone
 * records written up to that step.  Waits only for that step.  Returns
 * DZS_ESTATE if pipelining is off, DZS_EINVAL if that step's result is not
 * kept (not run yet, or more than 4 steps ago), DZS_EOVERFLOW if the device
 * flagged a buffer overflow by then. */
DZS_API dzs_status dzs_step_result(dzs_ctx* c, int32_t step, double diag[8], uint64_t* lc_written);

/* dzs_lightcone_drain up to the end of step `step` only (a kept step, see
 * dzs_step_result): the records written since the last drain and up to that
 * step, at most cap, copied on a copy stream of the context while later steps
 * keep running; same order, bookkeeping and DZS_EOVERFLOW as
 * dzs_lightcone_drain.  host_buf is caller-owned (pinned memory copies
 * fastest). */
DZS_API dzs_status dzs_lightcone_drain_step(dzs_ctx* c, int32_t step, dzs_lc_record* host_buf, size_t cap,
                                            size_t* n_out);

/* Free the context and its device memory.  NULL-safe. */
DZS_API dzs_status dzs_destroy(dzs_ctx* c);

/* Current particle count and step index (synchronises). */
DZS_API dzs_status dzs_get_count(dzs_ctx* c, size_t* n, int32_t* step);

/* Copy the state out (host arrays sized >= cap particles; SoA with stride n
 * for u, p, g).  Any pointer may be NULL to skip it.  *n = particle count. */
DZS_API dzs_status dzs_get_state(dzs_ctx* c, uint32_t* u, double* p, double* g, uint32_t* k,
                         uint32_t* id, uint8_t* fl, size_t cap, size_t* n);

/* Replace the state with n particles (n <= N0) at step index `step`.
 * g may be NULL (accelerations are then computed: DZS_STAGE_FORCE).  The
 * order is kept as given; dzs_run_stages(DZS_STAGE_SORT) sorts it. */
DZS_API dzs_status dzs_set_state(dzs_ctx* c, const uint32_t* u, const double* p, const double* g,
                         const uint32_t* k, const uint32_t* id, const uint8_t* fl, size_t n,
                         int32_t step);

/* Accelerations of the current particle set (PM and/or tree part), written
 * to g_out [3][n] in the current particle order.  The state is not modified. */
DZS_API dzs_status dzs_accel(dzs_ctx* c, int32_t parts, double* g_out);

/* Run the DZS merge alone (paper Sec. 2.2) on the current state, which must
 * be Morton-sorted, against the lattice lightcone radius rlat
 * (R_lc / L * 2^32).  With DZS_CRIT_DYNAMICAL, a_min is taken from the
 * state's accelerations g of the particles whose CROSSED flag is clear
 * (infinite when there is none). */
DZS_API dzs_status dzs_merge_only(dzs_ctx* c, uint64_t rlat);

/* Sum k, Sum k p[3], Sum k x[3] (Mpc/h), N (FP64; integer sums exact). */
DZS_API dzs_status dzs_diagnostics(dzs_ctx* c, double out[8]);

/* Checkpoint / restore (adapts the paper's halt-and-restart, Sec. 4.1.1: a run
 * stopped to re-allocate resources resumes from its output).  The
 * checkpoint holds the parameters, the step index, the particle state in the
 * context's own precision (raw, so a restored run continues bit for bit) and
 * the lightcone records not yet drained.  dzs_checkpoint_bytes gives the size;
 * dzs_checkpoint writes it to caller-owned host memory (DZS_EINVAL if cap is
 * too small); dzs_restore loads it into a context created with the same
 * parameters (device and lc_capacity may differ), DZS_EINVAL if the blob is
 * malformed or the parameters differ.  All three synchronise. */
DZS_API dzs_status dzs_checkpoint_bytes(dzs_ctx* c, size_t* bytes);
DZS_API dzs_status dzs_checkpoint(dzs_ctx* c, void* host_buf, size_t cap, size_t* written);
DZS_API dzs_status dzs_restore(dzs_ctx* c, const void* host_buf, size_t len);

/* The context's FP64 tables: a[nsteps+1], drift[nsteps], kick1[nsteps]
 * (a_n -> a_n+1/2), kick2[nsteps] (a_n+1/2 -> a_n+1), rlc[nsteps+1] (Mpc/h),
 * rlat[nsteps+1].  Any pointer may be NULL. */
/* Halt criteria (adapted from Sec. 4.1.1: the run stops for a re-allocation
 * of resources).  On one GPU the per-task workload balance has no
 * counterpart; the particle ratio R = N / N0 and the run-time rule do. */
typedef struct {
  double ratio_min;    /* halt once R < ratio_min (0: never) */
  double wall_limit_s; /* run-time limit of this call in seconds (0: none) */
  double horizon_s;    /* at the limit, halt for re-allocation if R, extrapolated
                          linearly in wall time, falls below ratio_min within
                          horizon_s after the restart */
} dzs_halt;

enum {
  DZS_HALT_NONE = 0,     /* max_steps done or a = 1 reached */
  DZS_HALT_RATIO = 1,    /* R < ratio_min */
  DZS_HALT_PREDICTED = 2, /* wall limit reached, R predicted below ratio_min within horizon_s */
  DZS_HALT_WALL = 3      /* wall limit reached, no re-allocation predicted */
};

/* Run up to max_steps full steps, checking the criteria after each step (one
 * synchronisation per step).  *reason gets a DZS_HALT_* value, *ratio the
 * last R.  A halted run resumes with dzs_step / dzs_step_until, or through
 * dzs_checkpoint and dzs_restore into a context created with a smaller
 * `capacity` (the freed memory goes back to the device). */
DZS_API dzs_status dzs_step_until(dzs_ctx* c, int32_t max_steps, const dzs_halt* h, int32_t* steps_done,
                                  int32_t* reason, double* ratio);

/* Lightcone observables (Sec. 3.1.2, Fig. 4: the lightcone mass projected on
 * an equal-area sky map and its angular power spectrum; Sec. 3.1.3, Fig. 5:
 * the 3D lightcone).  Once enabled, every lightcone record with
 * a_lo <= a_cross < a_hi adds its mass k (in units of m0) to
 *   - the pixel of its direction from the observer on the RING-ordered
 *     equal-area pixelisation of Górski et al. (2005), 12 nside^2 pixels
 *     (pixel index decided in FP64), and
 *   - the NGP cell floor(x* / L * mesh) per axis of a mesh^3 grid of the box
 *     ([i][j][l], l fastest),
 * as the step writes the record (also when the ring is full).  Counts are
 * exact uint64 sums.  Not part of a checkpoint. */
typedef struct {
  int32_t nside;  /* power of two, 1 .. 4096; 0: no sky map */
  int32_t mesh;   /* 1 .. 1024; 0: no 3D lightcone grid */
  double a_lo, a_hi;
} dzs_observe;

/* (Re)allocate and zero the observables; o == NULL or both sizes 0 turns them
 * off and frees them.  DZS_EINVAL for a bad size or a_lo > a_hi. */
DZS_API dzs_status dzs_observe_enable(dzs_ctx* c, const dzs_observe* o);
/* Bin n caller-owned host records (e.g. drained from another run) the same way. */
DZS_API dzs_status dzs_observe_add_records(dzs_ctx* c, const dzs_lc_record* rec, size_t n);
/* Copy the sky map (npix = 12 nside^2) / the 3D grid (ncell = mesh^3) to host
 * memory; DZS_EINVAL if the size differs or the observable is off. */
DZS_API dzs_status dzs_skymap_get(dzs_ctx* c, uint64_t* map, size_t npix);
DZS_API dzs_status dzs_lcdensity_get(dzs_ctx* c, uint64_t* grid, size_t ncell);
/* Harmonic analysis of the sky map (values = mass per pixel):
 * a_lm = (4 pi / npix) sum_p map_p conj(Y_lm(theta_p, phi_p)) at the pixel
 * centres, Y_lm orthonormal with the Condon-Shortley phase, 0 <= m <= l <=
 * lmax (lmax <= 4 nside); cl[lmax + 1] gets C_l = (|a_l0|^2 + 2 sum_m>0
 * |a_lm|^2) / (2l + 1); alm (may be NULL) gets (re, im) pairs at index
 * m (2 lmax + 1 - m) / 2 + l.  FP64, deterministic.  Synchronises. */
DZS_API dzs_status dzs_skymap_alm(dzs_ctx* c, int32_t lmax, double* cl, double* alm);

/* 3D power spectrum of the current particles (the time-slice P(k) compared
 * between DZS and standard runs): CIC deposit of the masses on the PM mesh,
 * delta = n / nbar - 1, forward FFT, P_mode = |delta_k|^2 L^3 / M^6 / W(k)^2
 * - P_shot with W = prod_i sinc^2(pi n_i / M) and P_shot = L^3 sum k^2 /
 * (sum k)^2; bin b = 1..nbins holds the modes with round(|n|) = b (|n| =
 * |k| L / 2 pi, rounding decided on integers); P_shot only with
 * DZS_PK_SHOT in flags.  k[b] = mean |k| [h/Mpc],
 * pk[b] = mean P_mode [(Mpc/h)^3], nmodes[b] = number of modes (k and nmodes
 * may be NULL).  1 <= nbins <= mesh / 2.  Arithmetic in the context's
 * precision, sums in FP64 in a fixed order.  Overwrites the meshes
 * dzs_get_mesh returns; the state and its order are unchanged.  Synchronises. */
DZS_API dzs_status dzs_power_spectrum(dzs_ctx* c, int32_t nbins, int32_t flags, double* k, double* pk,
                                      double* nmodes);
/* flags of dzs_power_spectrum: subtract P_shot (meant for Poisson-like sets;
 * merged particles, one per cell, and a displaced lattice are not) */
enum { DZS_PK_SHOT = 1 };

/* ---- Serving: continuous batching of independent lightcone mocks ----
 * No counterpart in the paper, which runs one simulation per MPI job; it
 * extends the paper's point that a DZS run needs less memory as it goes
 * (Sec. 4.1.1) to many mocks sharing one GPU.  Each request becomes a context
 * with its own non-blocking stream, admitted in arrival order once the sum of
 * the admitted footprints (dzs_footprint_bytes) fits hbm_budget_bytes (and
 * at most max_active run at once), advanced in slices of steps_per_slice
 * steps that overlap on the device, drained at a = 1 and destroyed (its
 * memory returns to the budget).  A mock's result does not depend on the mix
 * (separate state, deterministic reductions); record_hash (FNV-1a of the
 * drained records) lets a caller check that. */
typedef struct {
  double arrival_s; /* seconds after the start of dzs_serve */
  int32_t n1d;      /* particles per side */
  int32_t mesh;     /* PM mesh per side */
  double box;       /* L [Mpc/h] */
  double sigma8;
  uint64_t seed;
} dzs_request;

typedef struct {
  double admit_s, done_s; /* seconds after the start (latency = done_s - arrival_s) */
  uint64_t n_end;         /* particles left at a = 1 */
  uint64_t records;       /* lightcone records */
  uint64_t record_hash;   /* FNV-1a 64 of the records in drain order */
  double diag[8];         /* dzs_diagnostics at a = 1 */
  int32_t status;         /* dzs_status of this request */
  int32_t reserved_;
} dzs_request_result;

typedef struct {
  double hbm_budget_bytes;
  int32_t max_active;      /* 0: no limit besides the budget */
  int32_t steps_per_slice; /* >= 1 */
  int32_t host_threads;    /* host threads feeding the mocks; 0: min(8, hardware threads) */
  int32_t reserved_;
  dzs_params base;         /* everything but n1d, mesh, box, sigma8, seed (capacity ignored) */
} dzs_serve_config;

/* Batches (for many independent mocks on one GPU, batched or served; the
 * paper has one simulation per run): a batch steps several contexts
 * together.  dzs_batch_create keeps the n context pointers (it does not own
 * the contexts; they must outlive the batch) and uses host_threads worker
 * threads (0: min(8, hardware threads)).  dzs_batch_step enqueues up to
 * nsteps steps on every context, `slice` steps at a time round-robin over each
 * thread's share, so all streams get work early; it returns after enqueueing
 * (like dzs_step), with steps_done[i] (nullable, n entries) the steps
 * enqueued on context i, and the first failing status (the other contexts
 * still step).  Each context's results are exactly those of stepping it
 * alone.  dzs_batch_synchronize waits for every context's stream;
 * dzs_batch_destroy frees the batch (NULL-safe), not the contexts. */
typedef struct dzs_batch dzs_batch;
DZS_API dzs_status dzs_batch_create(dzs_ctx* const* ctxs, int32_t n, int32_t host_threads, dzs_batch** out);
DZS_API dzs_status dzs_batch_step(dzs_batch* b, int32_t nsteps, int32_t slice, int32_t* steps_done);
DZS_API dzs_status dzs_batch_synchronize(dzs_batch* b);
DZS_API dzs_status dzs_batch_destroy(dzs_batch* b);

/* Serve n requests (any order of arrival_s) to completion on base.device;
 * out[i] belongs to req[i].  Returns DZS_OK, or the first failing status (the
 * other requests still run); a request that alone exceeds the budget gets
 * DZS_ENOMEM.  *wall_s (may be NULL) = seconds from start to the last
 * completion.  The calling thread waits until every request is done; the
 * mocks are created, stepped, drained and destroyed by host_threads worker
 * threads (each admitted mock belongs to one of them; admission stays in
 * arrival order under the shared budget), so the kernel launches of many
 * small mocks are issued in parallel. */
DZS_API dzs_status dzs_serve(const dzs_serve_config* cfg, const dzs_request* req, size_t n,
                             dzs_request_result* out, double* wall_s);

/* Friends-of-friends haloes of the current particles (Sec. 3.1.1: the
 * lightcone halo mass function is built from FoF catalogues of frequent
 * outputs, keeping the haloes entirely inside the lightcone).  Two particles
 * are friends when their minimum-image lattice distance satisfies d^2 <=
 * floor((link 2^32 / n1d)^2), i.e. d <= link lambda, lambda = L / n1d (link
 * 0.2 is the usual choice); a halo is a connected component with >= nmin
 * particles.  Per halo: first = the smallest member index in the current
 * particle order (it labels the halo), count, mass = sum k (units of m0), the
 * centre of mass x = (u_first + S / K) L / 2^32 wrapped into [0, L) with S the
 * exact sum of k times the minimum-image lattice offsets from the first member
 * and K = mass, and rmax2 = the largest squared lattice distance of a member
 * from the observer (a halo is entirely inside the lightcone when rmax2 <
 * R_lat^2).  Haloes in increasing `first`; *nhalo = their number (only the
 * first `cap` are copied); label (may be NULL, n entries) = each particle's
 * halo `first` or -1.  Needs nmin >= 2 and 0 < link lambda < L / 4;
 * deterministic (the components are unique, every
 * sum is an integer sum).  The state is unchanged.  Synchronises. */
typedef struct {
  int64_t first;
  int64_t count;
  uint64_t mass;
  double x[3];
  uint64_t rmax2;
} dzs_halo;
DZS_API dzs_status dzs_fof(dzs_ctx* c, double link, int32_t nmin, dzs_halo* halos, size_t cap, size_t* nhalo,
                           int64_t* label);

DZS_API dzs_status dzs_get_tables(dzs_ctx* c, double* a, double* drift, double* kick1, double* kick2,
                          double* rlc, uint64_t* rlat);

/* Copy the PM density contrast or potential of the last force evaluation
 * ([M][M][M], iz fastest) as double. */
DZS_API dzs_status dzs_get_mesh(dzs_ctx* c, int32_t which, double* out);

/* Counters: [0] walk groups and [1] tree nodes of the last force evaluation,
 * [2] pair evaluations (interaction-list entries x group particles) summed
 * since the last dzs_ics / dzs_set_state / dzs_set_profiling, [3] device error
 * word, [4] kernels launched by this context so far, [5] lightcone records
  * written so far, [6] deepest tree-walk stack use (entries, of 512),
 * [7] tree-walk node tests and [8] traversal rounds summed like [2] ([6]-[8]
 * counted only with DZS_PROFILE_WALK, see dzs_set_profiling). */
DZS_API dzs_status dzs_get_counters(dzs_ctx* c, uint64_t out[9]);

/* Tree-walk work counters (Sec. 2.1 short-range force), summed like
 * dzs_get_counters' [2]: [0] listed pairs (interaction-list entries x group
 * particles, the same count as dzs_get_counters [2]), [1] pairs evaluated in
 * range (0 < r < r_cut: the pairs that carry force), [2] node tests, [3]
 * traversal rounds ([2] and [3] with DZS_PROFILE_WALK only), [4] group walks started from the window of deep frontier
 * cells around the group, [5] group walks that fell back to the shallow
 * frontier (a node between the two frontier depths might have been accepted).
 * Synchronises the context stream. */
DZS_API dzs_status dzs_get_walk_counters(dzs_ctx* c, uint64_t out[6]);

/* Interaction lists of the last tree walk, per walk group (Eq. 1 applied per
 * group: a node with <= walk_group particles whose parent holds more, or a
 * leaf): first particle (index in the current Morton order), particle count
 * and interaction-list length (accepted monopoles + particles of opened
 * leaves).  *ngroups receives the number of groups; any of first, count,
 * list_len may be NULL (all NULL: only the count); cap below the number of
 * groups is DZS_EINVAL.  Group order is the library's (by tree node).
 * Synchronises the context stream. */
DZS_API dzs_status dzs_walk_lists(dzs_ctx* c, int64_t* first, int64_t* count, int64_t* list_len, size_t cap,
                                  size_t* ngroups);

/* profile categories of dzs_get_profile */
enum {
  DZS_PROF_KICK_DRIFT = 0, /* opening kick, drift, crossing, record compaction */
  DZS_PROF_SORT = 1,       /* radix sort + permutation */
  DZS_PROF_MERGE = 2,      /* DZS merge */
  DZS_PROF_TREE = 3,       /* tree build + group list */
  DZS_PROF_PM = 4,         /* CIC deposit; four-point gradient + CIC interpolation */
  DZS_PROF_WALK = 5,       /* tree walk + closing kick */
  DZS_PROF_FFT = 6,        /* FFT Poisson solve (r2c, Green multiply, c2r) */
  DZS_PROF_N = 7
};

/* Profiling flags: DZS_PROFILE_STAGES (= 1) per-stage CUDA-event timing on
 * the context stream (two event records per stage, no synchronisation);
 * DZS_PROFILE_WALK (= 2) the tree walk's node-test, traversal-round and
 * deepest-stack counters (dzs_get_walk_counters [2] and [3],
 * dzs_get_counters [6]-[8]; 0 while off: counting costs ~1.5% of the
 * walk).  Any call resets the accumulators and the pair counters.  The pair
 * counts themselves (listed and in range) are always kept. */
enum { DZS_PROFILE_STAGES = 1, DZS_PROFILE_WALK = 2 };
DZS_API dzs_status dzs_set_profiling(dzs_ctx* c, int32_t enable);

/* Device milliseconds and call counts per category since the last
 * dzs_set_profiling (synchronises; either pointer may be NULL). */
DZS_API dzs_status dzs_get_profile(dzs_ctx* c, double ms[DZS_PROF_N], uint64_t calls[DZS_PROF_N]);

/* Largest n accepted by dzs_morton_sort_noalloc.  Its scratch is a static
 * device array of 24 * n + 4 * (257 * ceil(n / 2048) + 256) + 256 bytes,
 * about 6.4 MB, which every GPU that loads the library holds until exit. */
#define DZS_NOALLOC_SORT_MAX_N 262144

/* Allocation-free stable Morton sort of n <= DZS_NOALLOC_SORT_MAX_N lattice
 * positions.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- code inside a host framework whose
 * device memory belongs to that framework's own allocator, plugins given a
 * fixed memory budget, or paths that must not synchronise the device (an
 * allocation or free can).  It is the same radix sort as the step's Morton
 * sort (same keys, same stable order), but its scratch lives in one
 * file-scope static device array instead of a context arena.
 *   d_u     device, [3][n] uint32 lattice positions (x, then y, then z);
 *   d_perm  device, n uint32 output: sorted slot t holds input index d_perm[t];
 *   d_keys  device, n uint64 output of the sorted 63-bit keys, or NULL;
 *   stream  cudaStream_t the work is enqueued on (NULL = legacy stream).
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the process;
 * make that first call before any stream capture.  A cudaDeviceReset destroys
 * the array with the context that held it: do not call this entry point on
 * that device after a reset.  A CUDA error already pending on the calling
 * thread makes the call return DZS_ECUDA before it launches anything (the
 * error is left pending for its owner).  Every call shares the one array and leaves its contents behind
 * (each call writes every scratch word it reads before reading it), so calls
 * whose work overlaps on the GPU -- on two streams, or from two threads --
 * race and must be serialised by the caller.  Returns DZS_EINVAL for
 * n > DZS_NOALLOC_SORT_MAX_N or a NULL pointer with n > 0, DZS_EDEVICE when
 * no device is current, DZS_ECUDA when a CUDA call fails; asynchronous. */
DZS_API dzs_status dzs_morton_sort_noalloc(const uint32_t* d_u, size_t n, uint32_t* d_perm, uint64_t* d_keys,
                                           void* cuda_stream);

/* Measured FP32 arithmetic peaks of a device (the roofline denominators of the
 * tree walk, whose pair arithmetic of Sec. 2.1 runs on the FP32 FMA pipe and
 * the special-function unit): FMA-chain and reciprocal-square-root-chain
 * micro-benchmarks over every SM, timed with CUDA events, best of `reps`
 * launches after one warm-up.  *fma_tflops: FP32 TFLOP/s (an FFMA counts 2
 * flop); *sfu_gops: SFU operations per second / 1e9.  Either output may be
 * NULL (its kernel is then skipped), not both.  Allocates a few bytes of
 * device memory for the duration of the call and restores the current device.
 * Synchronous; DZS_EINVAL for reps < 1, DZS_EDEVICE / DZS_ECUDA on failure. */
DZS_API dzs_status dzs_measure_fp32_peaks(int32_t device, int32_t reps, double* fma_tflops, double* sfu_gops);

/* Twin-run integration accuracy (paper Sec. 3.2, the particle-by-particle
 * comparison of twin simulations with and without DZS): for the particles
 * inside the lightcone (not crossed) in both contexts a and b, matched by id,
 * the minimum-image distance of their positions divided by the softening
 * length h = L / n1d / 40, histogrammed by the nbins + 1 increasing edges
 * (host, in units of h): counts[k] (host, nbins) receives the pairs with
 * edges[k] <= dx / h < edges[k + 1]; *matched (nullable) the number of pairs,
 * *max_ratio (nullable) the largest dx / h.  FP64, correctly rounded, fixed
 * order: exact counts.  Both contexts on one device with the same n1d and box;
 * allocates a scratch of 4 n1d^3 bytes for the call; synchronises both streams.
 * DZS_EINVAL on bad arguments, DZS_ESTATE without particle states. */
DZS_API dzs_status dzs_twin_displacement(dzs_ctx* a, dzs_ctx* b, const double* edges, int32_t nbins,
                                         uint64_t* counts, uint64_t* matched, double* max_ratio);

/* Test hook (no counterpart in the paper): make the k-th device allocation
 * the library attempts from now on fail as if the device were out of memory
 * (k = 0 disables).  Host-side only: no GPU fault is involved.  The failing
 * call returns DZS_ENOMEM and frees what it had allocated. */
DZS_API void dzs_debug_fail_alloc(int32_t k);

/* Message of the last failure on this context (valid until the next call).
 * c may be NULL (then: the last dzs_create failure of this thread). */
DZS_API const char* dzs_last_error(const dzs_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* DZS_H */
