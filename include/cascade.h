/*
 * cascade.h -- C ABI of the GB300 pair-cascade particle-in-cell library.
 *
 * The library advances the 1D periodic electron-positron cascade of
 * Cruz, Grismayer & Silva, "Kinetic model of large-amplitude oscillations in
 * neutron star pair cascades" (arXiv:2012.05587), Section 3 setup, with the
 * simplified QED model of Section 2 (threshold emission, equal split of the
 * photon energy between the pair), on one CUDA device.
 *
 * Units (Section 3): c = 1, time in 1/omega_p, length in c/omega_p, E in
 * m c omega_p / e, momentum u = p / (m c), density in n0 (per species), with
 * omega_p^2 = 4 pi e^2 n0 / m.  Then du/dt = q E (q = -1 electrons, +1
 * positrons), dE/dt = -J (Ampere, Eq. 4 with 4 pi absorbed) and dE/dx = rho.
 *
 * Grid: nx cells of size dx, periodic.  Nodes x_i = i dx carry charge; edges
 * x_{i+1/2} carry E and J; arrays indexed by edge hold E_{i+1/2} at [i].
 * A particle is stored as an integer cell and an offset in [0, 1).
 *
 * Conventions for every entry point:
 *   - return CASCADE_OK (0) on success, a negative cascade_status otherwise;
 *   - all pointers named host_* / *_host / out are HOST memory owned by the
 *     caller; the library owns all device memory it allocates;
 *   - a failed call leaves the handle valid for cascade_diag, cascade_sync
 *     and cascade_destroy;
 *   - work is issued asynchronously on the CUDA stream given at creation
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream).
 */
#ifndef CASCADE_H
#define CASCADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CASCADE_OK = 0,
  CASCADE_ERR_INVALID_ARG = -1,     /* parameter outside the model's domain, bad pointer or size */
  CASCADE_ERR_OOM = -2,             /* device allocation failed */
  CASCADE_ERR_CAPACITY = -3,        /* particle_cap reached: pairs were dropped; results invalid */
  CASCADE_ERR_CUDA = -4,            /* a CUDA runtime call failed */
  CASCADE_ERR_TIMEOUT = -5,         /* a bounded device-side wait gave up */
  CASCADE_ERR_UNIMPLEMENTED = -6,
  CASCADE_ERR_PHOTON_CAPACITY = -7, /* photon ring full: photons were dropped; results invalid */
  CASCADE_ERR_BUSY = -8,            /* serving: no free slot or memory budget for the request */
  CASCADE_ERR_NONFINITE = -9        /* a lepton reached a non-finite energy: the run blew up */
} cascade_status;

/* CASCADE_FP64: every particle and grid quantity in FP64.
 * CASCADE_FP32_MIXED: int32 cell + FP32 offset and momentum (one FP32 word,
 *   or a compensated pair of two where one word cannot resolve the push at
 *   the threshold; see u_words); the per-CTA
 *   current is accumulated in int32 fixed point at a scale chosen per launch
 *   so no sum can overflow (resolution 2^-10 or finer per contribution at the
 *   largest sizes), then summed over CTAs, applied to E and reduced for the
 *   diagnostics in FP64; the threshold test of leptons above gamma = 1e6 is FP64.
 * CASCADE_FP32_MIXED_FINE: as FP32_MIXED with a two-word accumulator
 *   (resolution about 2^-20 per contribution, one more atomic each). */
typedef enum { CASCADE_FP64 = 0, CASCADE_FP32_MIXED = 1, CASCADE_FP32_MIXED_FINE = 2 } cascade_precision;

/* Parameters of one cascade, as Section 3 states them (plus the photon flight
 * length l_pp, which generalises the in-place pair creation of Section 2:
 * l_pp = 0 is the paper's model).
 * Validity (from the model's physics; otherwise CASCADE_ERR_INVALID_ARG):
 *   nx >= 2, ppc >= 1, 0 < dt < dx (so |dx per step| < one cell), n0 >= 0,
 *   u_spread >= 0, eps_gamma >= 2 (pair rest mass), gamma_thr - eps_gamma >= 1
 *   (the recoiled lepton stays physical), f = eps_gamma / gamma_thr < 2/3
 *   (the delay (1 - 3f/2) t_a of Eq. 1 is positive), l_pp >= 0. */
typedef struct {
  int32_t nx;            /* cells (periodic) */
  int32_t ppc;           /* seed macro-particles per cell per species */
  double dx, dt;         /* cell size, time step */
  double n0;             /* seed density per species; weight w = n0 dx / ppc */
  double u_spread;       /* seed momenta u ~ Normal(0, u_spread) */
  uint64_t seed;         /* Philox4x32-10 key for the seed momenta */
  double E0;             /* initial uniform field */
  double gamma_thr;      /* emission threshold */
  double eps_gamma;      /* photon energy in m c^2 (f = eps_gamma / gamma_thr) */
  double l_pp;           /* photon flight length before conversion */
  int64_t particle_cap;  /* capacity per species (particles) */
  int64_t photon_cap;    /* photons in flight; 0 = particle_cap rounded up to a power of 2 */
  int32_t precision;     /* cascade_precision */
  int32_t diag_ring;     /* per-step records kept on the device; 0 = 4096 */
  /* Co-rotating frame (Section 7, Eq. 25-26); all zero for the Section 3 model. */
  double j_m;            /* background current: dE/dt = -(J - j_m) */
  double rho_gj;         /* background charge: dE/dx = rho - rho_GJ (Gauss diagnostic) */
  int32_t open_bc;       /* 1: open boundaries -- the field beyond the outermost edges
                            equals the nearest edge, particles crossing x = 0 or x = L
                            deposit the path inside and are removed, photons that would
                            convert outside are not kept; 0: periodic */
  int32_t u_words;       /* FP32 modes: FP32 words per particle momentum.  0 = chosen at
                            creation: two when one word cannot resolve a push at the
                            threshold (cascade_momentum_words), else one; 1 = one
                            word (rejected where two are needed); 2 = two words, a
                            compensated hi + lo pair (4 B more per particle).
                            Ignored in CASCADE_FP64. */
} cascade_params;

/* One record per step, taken after the step (time t = step dt).  Energies are
 * per unit transverse area in n0 m c^2 (c/omega_p) units. */
typedef struct {
  int64_t step;
  double t;
  double E_mean;        /* mean of E over edges */
  double J_mean;        /* mean of J^{n+1/2} over edges */
  double E_absmax;      /* max |E| */
  double U_E;           /* sum E^2 / 2 dx */
  double U_K;           /* sum over leptons of w gamma (rest mass included) */
  double U_gamma;       /* photons in flight x w x eps_gamma */
  double gauss_resid;   /* max |E_{i+1/2} - E_{i-1/2} - dx rho_i|; NaN unless computed (cascade_gauss) */
  int64_t n_elec, n_posi;
  int64_t n_photon;     /* photons in flight */
  int64_t n_pairs_total;/* pairs created since the start */
  int64_t n_emit_multi; /* emissions of more than one photon in one step (dt too coarse) */
} cascade_diag_t;

typedef struct cascade cascade_t;

/* Device-memory hooks.  alloc returns a device pointer (256-byte aligned) or
 * NULL; free releases it.  Both receive the cascade's stream and ctx.  When
 * no hooks are set the library calls cudaMalloc / cudaFree.  The hooks are
 * global and apply to handles created after the call. */
typedef void* (*cascade_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cascade_free_fn)(void* ptr, void* stream, void* ctx);
int cascade_set_allocator(cascade_alloc_fn alloc_fn, cascade_free_fn free_fn, void* ctx);

/* Create a cascade in the Section 3 initial state: uniform E = E0 on every
 * edge and, in every cell, ppc co-located e-/e+ pairs (quiet start, rho = 0)
 * at offsets (k + 1/2)/ppc.  Pair j sits in cell j mod nx, k = j div nx; its
 * momenta are u_spread * (R cos A, R sin A) with R = sqrt(-2 ln U1),
 * A = 2 pi U2 (Box-Muller) from one Philox4x32-10 call with counter
 * (j, 0, 0, 0) and key (seed): U1, U2 are the two 64-bit halves of the
 * output reduced to 53-bit uniforms in (0, 1).  Electron j gets the cosine
 * branch, positron j the sine branch. */
int cascade_create(const cascade_params* params, void* cuda_stream, cascade_t** out);

/* Create a cascade from an explicit state (host arrays, copied): n_elec
 * electrons and n_posi positrons with cell in [0, nx), offset in [0, 1) and
 * momentum u; E_host (nx values) is the initial field or NULL for E0. */
int cascade_create_from_state(const cascade_params* params,
                              int64_t n_elec, const int32_t* cell_e, const double* off_e, const double* u_e,
                              int64_t n_posi, const int32_t* cell_p, const double* off_p, const double* u_p,
                              const double* E_host, void* cuda_stream, cascade_t** out);

/* As cascade_create_from_state, with FP32 host offsets and momenta: 12 B per
 * particle to upload instead of 20, for FP32 cascades (whose particles are
 * FP32 anyway; a two-word momentum gets a zero low word).  In CASCADE_FP64
 * the values are widened exactly. */
int cascade_create_from_state_f32(const cascade_params* params,
                                  int64_t n_elec, const int32_t* cell_e, const float* off_e, const float* u_e,
                                  int64_t n_posi, const int32_t* cell_p, const float* off_p, const float* u_p,
                                  const double* E_host, void* cuda_stream, cascade_t** out);

/* Advance nsteps steps (asynchronous).  One step n -> n+1 (Sections 2-3):
 *   1. photons due this step become e-/e+ pairs of gamma = eps_gamma/2 each,
 *      moving along the photon, at the conversion point x_emit +- l_pp;
 *   2. every lepton: gather E^n (linear between the two edges around it),
 *      push u += q dt E, move x += dt u / gamma, deposit the charge-conserving
 *      current of its linear (CIC) shape;
 *   3. Ampere: E^{n+1} = E^n - dt J^{n+1/2};
 *   4. every lepton with gamma >= gamma_thr emits k = 1 + floor((gamma -
 *      gamma_thr) / eps_gamma) photons and keeps its direction with gamma
 *      reduced by k eps_gamma; the photons convert n_pp = ceil(l_pp / dt)
 *      steps later (l_pp = 0: at the start of the next step, in place);
 *   5. the per-step record.
 * Errors of earlier asynchronous work (capacity) are reported by the next
 * cascade_sync / cascade_diag. */
int cascade_step(cascade_t* h, int32_t nsteps);

/* Wait for the cascade's stream; return the first device-side error seen. */
int cascade_sync(cascade_t* h);

/* Synchronise, then copy the newest min(max, kept) per-step records, oldest
 * first, into host_out and their number into n_out.  E_host / J_host (nx
 * values each, nullable) receive the current E^{n} and the last J^{n-1/2}. */
int cascade_diag(cascade_t* h, cascade_diag_t* host_out, int32_t max, int32_t* n_out,
                 double* E_host, double* J_host);

/* Per-step records without a wait (for a host loop that reads every step's
 * result while the next step runs).  cascade_record_enqueue queues, behind
 * the work queued on the cascade's stream so far, a copy of the newest
 * step's record (the one cascade_diag returns last) into pinned host memory
 * the library holds, and returns at once -- except when 64 copies are in
 * flight: it then waits for the oldest (so the host runs at most 64 steps
 * ahead of the device) and keeps that record for the poll.  Records are
 * kept until polled.  cascade_record_poll hands back up to max queued records, oldest
 * first, into host_out: with wait = 0 those that have landed (possibly none,
 * *n_out = 0), with wait != 0 it waits for each one it returns.  Returns the
 * cascade's sticky error status, like cascade_diag. */
int cascade_record_enqueue(cascade_t* h);
int cascade_record_poll(cascade_t* h, cascade_diag_t* host_out, int32_t max, int32_t wait, int32_t* n_out);
/* Bytes one queued copy moves to the host (the record with the step's
 * counters and error flag; no device needed). */
int32_t cascade_record_copy_bytes(void);

/* Synchronise and compute Gauss's-law residual max_i |E_{i+1/2} - E_{i-1/2} -
 * dx rho_i| of the current state (rho from the CIC shape); it is also stored
 * in the newest per-step record. */
int cascade_gauss(cascade_t* h, double* resid_out);

/* Per-step Gauss residual: with every > 0, each step whose index (after the
 * step) is a multiple of every also deposits the CIC charge of all leptons
 * and stores max_i |E_{i+1/2} - E_{i-1/2} - dx (rho_i - rho_GJ)| in that
 * step's record (gauss_resid; NaN in the other records).  A charge-conserving
 * step keeps the residual at round-off from one step to the next (Eq. 25,
 * Section 3 with rho_GJ = 0), so a growing value shows a broken invariant.
 * Cost: one more pass over the particles' cells and offsets (8 B in FP32)
 * with FP64 atomics, and two launches per step.  0 (the default) turns it
 * off.  The first call with every > 0 allocates nx + 1 doubles. */
int cascade_set_gauss_every(cascade_t* h, int32_t every);

/* Synchronise and copy particle counts, photons in flight and the step index. */
int cascade_counts(cascade_t* h, int64_t* n_elec, int64_t* n_posi, int64_t* n_photon, int64_t* step);

/* Phase-space histogram of one species (Fig. 2 and Eq. 8 of the paper show
 * these distributions): quantity 0 = momentum u, 1 = Lorentz factor gamma,
 * 2 = position x (in units of c/omega_p).  nbins (1 .. 65536) equal bins over
 * [lo, hi); values outside are not counted.  counts_host receives nbins
 * counts.  Synchronises the stream. */
int cascade_histogram(cascade_t* h, int32_t species, int32_t quantity, int32_t nbins, double lo, double hi,
                      int64_t* counts_host);

/* Synchronise and copy up to max particles of one species (0 = electrons,
 * 1 = positrons) in storage order into host arrays (nullable each); n_out
 * gets the number copied. */
int cascade_particles(cascade_t* h, int32_t species, int64_t max, int32_t* cell, double* off, double* u,
                      int64_t* n_out);

/* Kernel timing.  With timing on, cascade_step launches every step directly
 * (no graph replay) and records a CUDA event pair on the cascade's stream
 * around each launch of the particle kernel (gather/push/move/deposit/
 * emission).  cascade_timing synchronises and returns the summed duration
 * of those launches in milliseconds, their number, and the number of kernels
 * the library launched while timing was on; it then clears the counters. */
int cascade_set_timing(cascade_t* h, int32_t enable);
int cascade_timing(cascade_t* h, double* particle_kernel_ms, int64_t* particle_kernel_launches,
                   int64_t* kernels_launched);

/* ---------------------------------------------------------------------------
 * Batches: many independent cascades (uneven grids and particle counts)
 * advanced together.  One step is four launches for the whole batch: photon
 * conversion of every member, a plan that prices every member's particles
 * (plus a fixed share per member), one persistent particle kernel whose CTAs
 * each take an equal contiguous part of that cost, and one field kernel with
 * a CTA per member.  Steps are
 * replayed from a captured CUDA graph.  Each member keeps its own step
 * target; members that reach it stop.  All members share the batch's
 * precision (CASCADE_FP64 or one of the FP32 modes) and nx <= max_nx.
 * ------------------------------------------------------------------------- */
typedef struct cascade_batch cascade_batch_t;

/* Empty batch of max_slots slots.  hbm_budget caps the device bytes that
 * admitted members may hold (0 = no cap); max_nx sizes the shared-memory
 * stage of the particle kernel (members need nx <= max_nx). */
int cascade_batch_create_slots(int32_t max_slots, int32_t precision, int32_t max_nx, size_t hbm_budget,
                               void* cuda_stream, cascade_batch_t** out);

/* Batch of n members created from params[0..n-1] (all in the Section 3
 * initial state); max_nx is the largest member grid; every member starts
 * with zero steps to do.  Every member is checked on the host before any
 * device work: the single-cascade parameter domain, one precision class
 * for all, periodic grids; a failure returns CASCADE_ERR_INVALID_ARG and
 * cascade_last_error_message names the member. */
int cascade_batch_create(const cascade_params* params, int32_t n, size_t hbm_budget, void* cuda_stream,
                         cascade_batch_t** out);

/* Admit one cascade into a free slot with nsteps steps to run.  Its device
 * memory is allocated and seeded on a private stream, so admission does not
 * wait for the steps already queued.  CASCADE_ERR_BUSY: no free slot, or its
 * footprint (cascade_footprint) would exceed the budget. */
int cascade_batch_admit(cascade_batch_t* b, const cascade_params* params, int32_t nsteps, int32_t* slot_out);

/* Add nsteps_each[i] steps to member i (host array of max_slots entries;
 * empty slots ignore theirs) and run until every member is done.  Async. */
int cascade_batch_step(cascade_batch_t* b, const int32_t* nsteps_each);

/* Run up to nsteps batch steps (members with nothing left are skipped).
 * Async; queues a copy of the members' remaining step counts behind them. */
int cascade_batch_run(cascade_batch_t* b, int32_t nsteps);

/* Slots whose admitted run has finished and that were not reported before.
 * wait = 0: report only what the newest completed run shows (no blocking);
 * wait != 0: wait for all queued work first. */
int cascade_batch_poll(cascade_batch_t* b, int32_t* done_slots, int32_t max, int32_t* n_out, int32_t wait);

/* Per-step records of one member (as cascade_diag; waits for the batch). */
int cascade_batch_diag(cascade_batch_t* b, int32_t slot, cascade_diag_t* host_out, int32_t max, int32_t* n_out,
                       double* E_host, double* J_host);

/* Counts of one member (as cascade_counts; waits for the batch). */
int cascade_batch_counts(cascade_batch_t* b, int32_t slot, int64_t* n_elec, int64_t* n_posi, int64_t* n_photon,
                         int64_t* step);

/* Free a member's device memory and its slot (waits for the batch). */
int cascade_batch_release(cascade_batch_t* b, int32_t slot);

/* Number of slots, occupied slots and device bytes held by members. */
int cascade_batch_info(cascade_batch_t* b, int32_t* slots, int32_t* occupied, size_t* bytes_in_use);

/* Launch variant of the batched particle kernel.  All variants compute the
 * same step; they differ in speed, and in round-off through the fixed-point
 * scale of each CTA's share of the batch. */
typedef struct {
  int32_t shape;        /* threads per CTA and register budget: 0 = 2 x 512 threads (64
                           registers), 1 = 512 (128), 2 = 768 (80), 3 = 640 (96), all
                           persistent with the members' work split evenly over the CTAs;
                           4 = 1024 (64), a row of CTAs per member (grid members x CTAs,
                           each member's descriptor in the constant bank; FP32 batches that
                           hold a slice of the member table; the FP32 default) */
  int32_t stage;        /* 1: particles staged through shared memory with cp.async (FP32) */
  int32_t prefetch;     /* iterations ahead each warp prefetches its particles into L2 (0..8) */
  int32_t member_cost;  /* fixed work units per member in the partition (4-particle chunks) */
} cascade_batch_variant;

enum { CASCADE_VARIANT_DEFAULT = 0, CASCADE_VARIANT_CACHED = 1, CASCADE_VARIANT_TUNED = 2,
       CASCADE_VARIANT_FORCED = 3 };

/* Autotuning (the batches' launch shapes are picked by measurement).  A
 * batch tunes at every cascade_batch_step or cascade_batch_run that has work
 * and finds its size class (cascade_tune_key: grid, seed particles and
 * member count of the members present) changed since the variant in use was
 * picked -- at the first such call, and again as a server's occupancy moves
 * to another class.  It first looks the class up in the per-device cache
 * file (cascade_tune_cache_path); on a miss, after a warm-up
 * (cascade_batch_tune_warmup), it runs the
 * candidate variants -- the five shapes (four in FP64) with cp.async staging
 * (FP32) and without it (then an L2 prefetch) -- one batch step each, round after round
 * (4 rounds, or as many as the call's steps allow), times the particle
 * kernel with CUDA events, scores each variant by time per work unit of the
 * partition, keeps the fastest and stores it in the cache.  Tuning steps are
 * real steps of the members' work.  Setting any of CASCADE_BATCH_SHAPE,
 * CASCADE_BATCH_STAGE, CASCADE_BATCH_PREFETCH, CASCADE_BATCH_MEMBER_COST
 * before creation forces a variant (no tuning); CASCADE_BATCH_TUNE=0 keeps
 * the default variant.  CASCADE_BATCH_CTAS_PER_SM (1..64, default 8) sets how
 * many CTAs per SM and step shape 4 splits the members' work into.
 *   cascade_batch_set_variant  forces v (CASCADE_ERR_INVALID_ARG if it does not
 *                              fit this batch) and disarms tuning
 *   cascade_batch_get_variant  the variant in use, where it came from
 *                              (CASCADE_VARIANT_*) and, when tuned, its
 *                              measured ns per work unit (each nullable)
 *   cascade_batch_tune_next    (re)arms tuning for the next step or run
 *                              call: rounds of candidates (0 disarms);
 *                              use_cache = 0 makes that pass measure even
 *                              on a cache hit */
int cascade_batch_set_variant(cascade_batch_t* b, const cascade_batch_variant* v);
int cascade_batch_get_variant(cascade_batch_t* b, cascade_batch_variant* v, int32_t* source, double* ns_per_unit);
int cascade_batch_tune_next(cascade_batch_t* b, int32_t rounds, int32_t use_cache);
/* Steps a batch runs with its current variant before a tuning pass the
 * cache cannot answer (default 256; cascade_batch_step uses at most a
 * quarter of the steps it runs): the members then hold their grown particle
 * counts rather than their seeds. */
int cascade_batch_tune_warmup(cascade_batch_t* b, int64_t steps);
/* The candidates of the batch's last tuning pass and their measured ns per
 * work unit (up to max; *n_out = 0 before any pass). */
int cascade_batch_tuning_report(cascade_batch_t* b, cascade_batch_variant* cands, double* ns_per_unit, int32_t max,
                                int32_t* n_out);

/* The tuning cache.  Key of a size class: precision, ceil(log2) of the
 * largest member grid, the nearest log2 of the members' seed particles and
 * ceil(log2) of the number of members (key_len >= 64).  The file holds one
 * line per key: "<key>\t<shape> <stage> <prefetch> <member_cost>\t<ns per
 * unit>"; a store rewrites it whole through a temporary file and a rename.
 * Entries are also kept in memory for the process, so a path that cannot be
 * written (or NULL) still serves lookups of this process's own stores.
 * cascade_tune_cache_lookup sets *found to 1 and fills out on a hit.
 * cascade_tune_cache_path: $CASCADE_TUNE_CACHE if set (empty = memory only),
 * else $XDG_CACHE_HOME or $HOME/.cache, then
 * cascade-gb300/batch-tune-<device name>-sm<cc>.txt for the current device
 * (thread-local static storage). */
int cascade_tune_key(int32_t precision, int32_t max_nx, int64_t particles, int32_t members, char* key_out,
                     int32_t key_len);
int cascade_tune_cache_lookup(const char* path, const char* key, cascade_batch_variant* out, int32_t* found);
int cascade_tune_cache_store(const char* path, const char* key, const cascade_batch_variant* v, double ns_per_unit);
const char* cascade_tune_cache_path(void);

/* Kernel timing of a batch, as cascade_set_timing / cascade_timing: with
 * timing on, batch steps are launched directly (no graph replay) with a CUDA
 * event pair around each launch of the batched particle kernel;
 * cascade_batch_timing synchronises, returns the summed duration of those
 * launches (ms), their number and the kernels launched, and clears them. */
int cascade_batch_set_timing(cascade_batch_t* b, int32_t enable);
int cascade_batch_timing(cascade_batch_t* b, double* particle_kernel_ms, int64_t* particle_kernel_launches,
                         int64_t* kernels_launched);

/* Release everything (NULL is accepted). */
int cascade_batch_destroy(cascade_batch_t* b);

/* Largest grid cascade_gauss_noalloc accepts. */
#define CASCADE_NOALLOC_MAX_NX 65536

/* Gauss's-law residual max_i |E_{i+1/2} - E_{i-1/2} - dx (rho_i - rho_GJ)|
 * (Eq. 25; rho_GJ = 0 outside the co-rotating frame) of a state held by the
 * caller, computed without allocating any memory.  The paper has no
 * counterpart: this is a library service, the same check as cascade_gauss
 * but on the caller's buffers.  It exists for callers that cannot allocate
 * device memory: applications that reserve all device memory for their own
 * pool at start-up and forbid libraries to allocate, plug-ins whose host
 * program owns every allocation, and real-time loops where cudaMalloc (which
 * may synchronise the whole device) is not allowed.  Its scratch (charge per
 * node and the result: CASCADE_NOALLOC_MAX_NX + 32 doubles, 512.25 KiB) is a
 * static device array that every GPU which loads this library holds until
 * the process exits.
 *   nx          cells, 2 .. CASCADE_NOALLOC_MAX_NX (otherwise
 *               CASCADE_ERR_INVALID_ARG, with a message naming the limit)
 *   dx          cell size (> 0); the residual is in units of E
 *   w           macro-particle weight n0 dx / ppc
 *   rho_gj      background charge density (0 outside the co-rotating frame)
 *   open_bc     0: periodic (node nx is node 0); 1: open boundaries (the
 *               charge beyond node nx - 1 is not kept, node 0 is not checked)
 *   precision   CASCADE_FP64: offsets are double; CASCADE_FP32_MIXED and
 *               CASCADE_FP32_MIXED_FINE: offsets are float
 *   n_elec, cell_e, off_e / n_posi, cell_p, off_p
 *               particle counts and DEVICE arrays (cell int32 in [0, nx),
 *               offset in [0, 1); a cell outside the grid, such as the -1 of
 *               a departed particle, is skipped), read only
 *   E           DEVICE array of nx doubles, E_{i+1/2} at [i], read only
 *   resid_out   HOST double receiving the residual
 *   cuda_stream stream the work is issued on; the call synchronises it and
 *               copies the result to the host before returning
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call shares the one array and clears it first: calls that
 * overlap on the GPU (other streams or threads at the same time) race on it,
 * so serialise them.  No cudaMalloc, cudaFree or allocating library call is
 * made. */
int cascade_gauss_noalloc(int32_t nx, double dx, double w, double rho_gj, int32_t open_bc, int32_t precision,
                          int64_t n_elec, const int32_t* cell_e, const void* off_e,
                          int64_t n_posi, const int32_t* cell_p, const void* off_p,
                          const double* E, double* resid_out, void* cuda_stream);

/* Release all device memory of the handle (NULL is accepted). */
int cascade_destroy(cascade_t* h);

/* Photon-flight steps n_pp = ceil(l_pp / dt - 1e-9) and device bytes a
 * cascade with these parameters allocates (for admission by footprint). */
int cascade_footprint(const cascade_params* params, int32_t* n_pp_out, size_t* device_bytes_out);

/* FP32 words per particle momentum that cascade_create would use for these
 * parameters (1 or 2; 2 in CASCADE_FP64 stands for the FP64 word).  One FP32
 * word suffices when half its spacing at the threshold momentum
 * u_thr = sqrt(gamma_thr^2 - 1) is at most 2^-12 of the reference push
 * F dt, F = |E0|, or gamma_thr / (nx dx) when E0 = 0 (the weakest uniform
 * field that brings a lepton from rest to threshold across the domain).
 * Otherwise the push of a lepton near threshold would lose more than 2^-12 of
 * itself to rounding every step (at u = 7.3e7, the threshold Section 8
 * estimates, the FP32 spacing is 8: any push below 4 is lost entirely), so
 * the momentum is kept as a compensated pair of FP32 words whose sum carries
 * about 48 bits.  CASCADE_ERR_INVALID_ARG for parameters outside the domain,
 * or for u_words = 1 where two words are needed (the message names the
 * limit). */
int cascade_momentum_words(const cascade_params* params, int32_t* words_out);

/* Human-readable text of a status code (static storage). */
const char* cascade_status_string(int status);

/* Detail of the last failure on the calling thread (static, thread-local).
 * Every entry point except the destroy calls clears it on entry, so it
 * describes the most recent call only; it is empty when that call set no
 * detail. */
const char* cascade_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* CASCADE_H */
