/*
 * ddqmc.h -- C-ABI of libddqmc.so, a GB300 (sm_103a) implementation of one
 * step of driven-dissipative quantum Monte Carlo (DDQMC): real-time FCIQMC
 * sampling of the vectorised density matrix of an open spin-1/2 XYZ lattice
 * under the shifted Liouvillian (Nagy & Savona, arXiv:1802.05931).
 *
 * Conventions shared by every call
 *   - Return value: 0 (DDQMC_OK) on success, a negative DDQMC_ERR_* code
 *     otherwise.  Errors found on the device (capacity, int32 overflow,
 *     bounded-wait timeout) are sticky: once set, every later call on the run
 *     returns the same code.  No C++ exception crosses this interface.
 *   - Pointers named host_* or passed as plain arrays are HOST memory owned by
 *     the caller; the run owns all of its device memory.
 *   - A run is not thread-safe; separate runs may be driven from separate host
 *     threads.  All device work of a run is issued on its CUDA stream.
 *   - Basis: site k = x + Lx*y; bit k of a spin word is 1 when spin k is up.
 *     A configuration |i><j| is the pair (ket i, bra j).  Walker lists are in
 *     canonical order: by bra word, then by ket word.
 *   - Model (Sec. V): H = sum over nearest-neighbour bonds of
 *     Jx sx sx + Jy sy sy + Jz sz sz with Pauli matrices, and decay at rate
 *     gamma through sigma^- on every site (Lindblad equation, Sec. III.A).
 */
#ifndef DDQMC_H
#define DDQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDQMC_OK 0
#define DDQMC_ERR_INVALID_ARG (-1)   /* a parameter or pointer is invalid */
#define DDQMC_ERR_OOM (-2)           /* device or host allocation failed */
#define DDQMC_ERR_CAPACITY (-3)      /* walker list or spawn buffer capacity exceeded (sticky) */
#define DDQMC_ERR_OVERFLOW (-4)      /* a population left the int32 range (sticky) */
#define DDQMC_ERR_TIMEOUT (-5)       /* a bounded device wait gave up (sticky) */
#define DDQMC_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define DDQMC_ERR_UNSUPPORTED (-7)   /* valid parameters a call does not handle (see the call) */

#define DDQMC_MAX_SITES 64
#define DDQMC_MAX_BONDS 128

/* Lattice: Lx x Ly sites; periodic = 1 wraps both directions (then each
 * periodic extent must be 1 or >= 3, since L = 2 would repeat bonds). */
typedef struct {
    int32_t Lx, Ly, periodic;
} ddqmc_lattice;

/* Importance sampling (Sec. IV.B): the population on |i><j| represents
 * w_ij rho_ij and every off-diagonal rate is multiplied by w_child/w_parent.
 *   kind 0: none (w = 1);
 *   kind 1: uniform, w_ij = exp(-p) for every i != j, w_ii = 1 (the paper's
 *           single-parameter scheme);
 *   kind 2: site product, w_ij = prod over sites k where i and j differ of
 *           site_ratio[k] (N values in (0, 1]), w_ii = 1.  site_ratio is read
 *           during ddqmc_create only. */
typedef struct {
    int32_t kind;
    double p;
    const double *site_ratio;
} ddqmc_guide;

/* Options; fill with ddqmc_default_options() and override fields. */
typedef struct {
    uint64_t seed;             /* Philox key; default 1 */
    double damping;            /* delta of the shift update (Sec. III.C); default 0.05 */
    double shift0;             /* S before the target is reached; default -1.0 */
    int64_t n0;                /* initial real walkers on |down..down><down..down|; default 1000 */
    int32_t control;           /* 0: N_w = sum |Re rho_ii| (the paper's rule); 1: total sum |re|+|im| */
    int64_t t_eq;              /* steps after the shift switches on before estimates
                                  accumulate; < 0: ceil(10 / (gamma dt)) */
    int64_t capacity_entries;  /* walker-list capacity (entries); <= 0: 2*target (control 1)
                                  or 64*target (control 0), plus 65536 */
    int64_t capacity_spawns;   /* spawn-record capacity per step; <= 0: 4*target (control 1)
                                  or 64*target (control 0), plus 65536 */
    void *cuda_stream;         /* cudaStream_t to issue work on; NULL: the run creates its own */
    int32_t sm_limit;          /* > 0: size every kernel grid for at most this many SMs, so that
                                  several runs stepped on their own streams share the GPU;
                                  <= 0 (default): the whole GPU */
    double field_h;            /* in-plane field of Sec. V.B, H += h sum_k (cos t sx_k + sin t sy_k);
                                  default 0 (none) */
    int32_t field_axis;        /* direction t: 0 along x (t = 0), 1 along y (t = pi/2), 2 the
                                  angle field_theta; default 0 */
    int32_t wide_sort_bits;    /* lattices of more than 31 sites (two-word keys): the list and
                                  the spawn records are kept in the hashed order (stored bra
                                  word = bra ^ (64-bit hash of ket, low wide_sort_bits bits),
                                  then ket); a step sorts the spawn records on the stored bra
                                  word only and puts records that share it in ket order.
                                  0..64, default 64 (8 digit passes instead of up to 16);
                                  -1: plain (bra, ket) order on every key bit.  Results do not
                                  depend on it; fewer bits make equal stored words common (a
                                  test of their repair).  Import and export stay in (bra, ket)
                                  order and then need entries <= capacity_spawns (a batch: the
                                  exported run's entries).  A batch puts its run id above
                                  max(N, hash bits) in the bra word and sorts digit passes up
                                  to the run id's top bit; it hashes at most one digit byte
                                  more than its spin and run-id bits fill, and at most 64
                                  minus the run id's bits.  A 6x6 batch of up to 16 runs takes
                                  6 passes at the default, 10 in the plain order, and 5 with
                                  wide_sort_bits = 36, for small runs: D distinct keys spawned
                                  in a run then share stored bra words in about D^2 / 2^37
                                  pairs per step, and past 16,384 out-of-order neighbours in
                                  all runs the step stops with CAPACITY. */
    double field_theta;        /* field_axis 2: the angle t (radians); each site flip is then two
                                  moves, |h cos t| (the x part) and |h sin t| (the y part), so
                                  2B + 5N moves per configuration must fit the move table
                                  (UNSUPPORTED otherwise: up to 24 sites of a periodic lattice
                                  with one-word keys, 6x6 with two-word keys); default 0 */
} ddqmc_options;

typedef struct ddqmc_run ddqmc_run;

/* Steady-state estimates (ratios of time averages, Sec. III.A) with blocked
 * standard errors, over the steps t >= t_eq.  Without a field, sigma^x and
 * sigma^y are zero by the Z2 parity of the dynamics (every move flips an even
 * number of spins across ket and bra); with the in-plane field of Sec. V.B
 * they are reported per site and as the magnetisations mx, my. */
typedef struct {
    int64_t t;                 /* completed steps */
    double shift;              /* current S */
    int32_t variable;          /* 1 once the shift update is on */
    int64_t t_var, t_eq;       /* first variable-shift step; first accumulated step */
    int64_t n_samples;         /* steps accumulated */
    int64_t walkers;           /* sum |re|+|im| of the current list */
    int64_t entries;           /* occupied configurations */
    int64_t nw;                /* sum |Re rho_ii| of the current list */
    int64_t trace_re, trace_im;
    int32_t nsites, nbonds;
    double walker_steps;       /* sum over completed steps of the walkers stepped */
    double mz, mz_err;         /* M_z = (1/N) sum_k <sigma^z_k> (Sec. V.A) */
    double xx, xx_err, yy, yy_err, zz, zz_err;     /* bond averages of <s s> */
    double sz[DDQMC_MAX_SITES], sz_err[DDQMC_MAX_SITES];
    double bond_xx[DDQMC_MAX_BONDS], bond_yy[DDQMC_MAX_BONDS], bond_zz[DDQMC_MAX_BONDS];
    double mx, mx_err, my, my_err;   /* (1/N) sum_k <sigma^x_k>, <sigma^y_k>: non-zero only with a field */
    double sx[DDQMC_MAX_SITES], sy[DDQMC_MAX_SITES];
} ddqmc_estimates;

/* Scalar state of a run (for checkpoints and single-step comparisons). */
typedef struct {
    int64_t t;
    double shift;
    int32_t variable;
    int64_t q_prev;            /* controlled weight after the last step */
    int64_t t_var, t_eq;
    int64_t entries;
    int32_t status;            /* sticky device status (0 or a DDQMC_ERR_* code) */
    int32_t status_bits;       /* device status bits: 1 capacity, 2 int32 overflow, 4 timeout,
                                  8 walker-list capacity, 16 spawn-buffer capacity */
} ddqmc_state;

/* Defaults for every option field.  Returns DDQMC_OK, or INVALID_ARG for NULL. */
int ddqmc_default_options(ddqmc_options *opt);

/* Create a run (Sec. III.C problem statement: lattice, couplings, gamma, dt,
 * target population, initiator threshold I_limit = n_a (Sec. IV.A, 0 = none),
 * importance guide).  Allocates all device memory, writes the initial list
 * of opt->n0 real walkers on |down..down><down..down| and S = opt->shift0.
 * guide and opt may be NULL (no importance sampling / defaults).
 * Up to 31 sites, ket and bra pack into one 64-bit key (bra << N | ket) and
 * records are 16 bytes; from 32 to 64 sites (the 6x6 and 8x8 lattices) each
 * side is one 64-bit word and records are 24 bytes.
 * Errors: INVALID_ARG (N > 64, dt <= 0, gamma < 0, target <= 0, n_a < 0,
 * bad guide), OOM, CUDA.  *out is NULL on error. */
int ddqmc_create(const ddqmc_lattice *lattice, double Jx, double Jy, double Jz,
                 double gamma, double dt, int64_t target_walkers,
                 int32_t initiator_threshold, const ddqmc_guide *guide,
                 const ddqmc_options *opt, ddqmc_run **out);

/* Advance nsteps DDQMC steps (Sec. III.C, one step = spawn + death/clone,
 * annihilation under the initiator rule, estimators, shift update), issued
 * on the run's stream; waits for completion and returns the sticky device
 * status.  nsteps = 0 only reports the status.  Whole blocks of 32 steps are
 * replayed from a CUDA graph that the first such block captures on the run's
 * stream (one graph per starting list buffer; plain launches while
 * per-kernel timing is on, or if the stream cannot be captured); the results
 * are the same either way. */
int ddqmc_step(ddqmc_run *run, int64_t nsteps);

/* Same as ddqmc_step but does not wait: returns after enqueueing the work;
 * the device status is reported by the next waiting call. */
int ddqmc_step_async(ddqmc_run *run, int64_t nsteps);

/* Wait for the run's stream and return the sticky device status. */
int ddqmc_sync(ddqmc_run *run);

/* Steady-state estimates with blocked errors (waits for the stream). */
int ddqmc_estimators(ddqmc_run *run, ddqmc_estimates *out);

/* Integer estimator numerators of the current list (Sec. III.A):
 * [0] Tr Re, [1] Tr Im, [2] N_w, [3] sum |re|+|im|, [4] entries,
 * [5, 5+N) sum z_k Re rho_ii, then per bond zz, xx, yy numerators (B each),
 * then the sums over sites/bonds of those four blocks.  Writes
 * min(cap, nobs) values to host_out and nobs to *nobs. */
int ddqmc_raw_estimators(ddqmc_run *run, int64_t *host_out, int32_t cap, int32_t *nobs);

/* Exact integer blocking moments (Flyvbjerg-Petersen levels) of observable
 * k against the trace: for each level l < levels, n (blocks), sum X,
 * sum X^2, sum X*Y (Y = Tr Re block sums).  The 128-bit sums are returned as
 * (lo, hi) pairs of 64-bit words, two's complement.  Arrays hold `levels`
 * (resp. 2*levels) entries. */
int ddqmc_blocking_moments(ddqmc_run *run, int32_t k, int32_t levels, int64_t *host_n,
                           int64_t *host_sx, int64_t *host_sxx, int64_t *host_sxy);

/* Copy the current walker list (canonical order) to host arrays of capacity
 * cap; *n receives the list length (call with cap = 0 to query it).  The list
 * is unpacked into the four arrays on the device and each array crosses the
 * host link in one copy (at the link's speed when the host arrays are pinned,
 * e.g. from cudaMallocHost); device scratch of 24 bytes per entry is kept
 * by the run after the first call.  A run in the hashed order of two-word
 * keys (wide_sort_bits >= 0) is first sorted into the canonical order on
 * the device, in its spawn buffers: CAPACITY if the list has more entries
 * than capacity_spawns.  Waits for the run's stream. */
int ddqmc_export_walkers(ddqmc_run *run, uint64_t *ket, uint64_t *bra, int32_t *re,
                         int32_t *im, int64_t cap, int64_t *n);

/* Replace the walker list with n host entries (strictly increasing canonical
 * order, no all-zero entry, spin words within N bits) and set the step
 * counter t and shift S; the shift stays in its variable phase iff
 * variable != 0, with q_prev as the last controlled weight.  Clears the
 * accumulated estimates and any sticky error.  Each array crosses the host
 * link in one copy (pinned arrays at the link's speed); the entries are
 * checked and packed on the device into the run's spare list buffer, so a
 * list that fails a check (INVALID_ARG) leaves the run as it was.  A run in
 * the hashed order of two-word keys sorts the entries into it on the device,
 * in its spawn buffers (CAPACITY if n > capacity_spawns). */
int ddqmc_import_walkers(ddqmc_run *run, const uint64_t *ket, const uint64_t *bra,
                         const int32_t *re, const int32_t *im, int64_t n, int64_t t,
                         double S, int32_t variable, int64_t q_prev, int64_t t_var,
                         int64_t t_eq);

/* The walker list in the run's own record layout, for callers that stream it
 * through host memory every step: 16-byte records
 *     { uint64_t key = bra << N | ket; int32_t re; int32_t im; }
 * in canonical order (strictly increasing key), a third fewer bytes than the
 * four arrays above and no conversion on either side.  Single runs of at most
 * 31 sites (UNSUPPORTED otherwise).  host_records must be 8-byte aligned; the
 * copy runs at the link's speed when it is pinned. */

/* Copy the current list into host_records (capacity cap records); *n
 * receives the list length (cap = 0 queries it).  One copy over the link.
 * Waits for the run's stream. */
int ddqmc_export_records(ddqmc_run *run, void *host_records, int64_t cap, int64_t *n);

/* Replace the list with n host records and set the state as
 * ddqmc_import_walkers does (same checks: keys strictly increasing and within
 * 2N bits, no all-zero entry; INVALID_ARG leaves the run as it was).  One copy
 * over the link into the run's spare list buffer, checked there. */
int ddqmc_import_records(ddqmc_run *run, const void *host_records, int64_t n, int64_t t, double S,
                         int32_t variable, int64_t q_prev, int64_t t_var, int64_t t_eq);

/* The same for lattices of at most 16 sites (keys of at most 32 bits) in
 * 12-byte records { uint32_t key = bra << N | ket; int32_t re; int32_t im; }
 * (packed, 4-byte aligned), a quarter fewer bytes over the link than the
 * 16-byte records; packed and unpacked on the device (UNSUPPORTED for more
 * sites or a batch). */
int ddqmc_export_records32(ddqmc_run *run, void *host_records, int64_t cap, int64_t *n);
int ddqmc_import_records32(ddqmc_run *run, const void *host_records, int64_t n, int64_t t, double S,
                           int32_t variable, int64_t q_prev, int64_t t_var, int64_t t_eq);

/* Scalar state (waits for the stream). */
int ddqmc_get_state(ddqmc_run *run, ddqmc_state *out);

/* Last step's spawn-record count and the list/spawn capacities (diagnostics
 * and roofline accounting). */
int ddqmc_get_counts(ddqmc_run *run, int64_t *spawn_records, int64_t *capacity_entries,
                     int64_t *capacity_spawns);

/* Totals over all completed steps (device counters, exact): walkers stepped
 * (sum over steps of sum |re|+|im| of the list being stepped), configurations
 * stepped, spawn records written, and configurations of the merged lists.
 * They give the algorithmic bytes of each kernel.  Any pointer may be NULL. */
int ddqmc_get_totals(ddqmc_run *run, int64_t *walker_steps, int64_t *entry_steps,
                     int64_t *spawn_records, int64_t *merged_entries);

/* Per-kernel timing: with enable != 0 every later ddqmc_step brackets each
 * kernel class with CUDA events on the run's stream (classes: 0 spawn+death,
 * 1 radix passes, 2 merge partition, 3 merge+annihilation+estimators,
 * 4 finalize, 5 compaction of the merged list: tile-offset scan and copy)
 * and accumulates the elapsed times; enabling or disabling resets the sums.
 * ddqmc_step_async does not record events. */
int ddqmc_set_timing(ddqmc_run *run, int32_t enable);

/* Accumulated milliseconds and launch counts per kernel class (cap >= 6). */
int ddqmc_get_timing(ddqmc_run *run, double *ms, int64_t *launches, int32_t cap);

/* Launch shapes of a run's kernels (no counterpart in the paper: they change
 * how fast a step runs, never what it computes).  Blocks per SM of each
 * persistent kernel, the partition's blocks per SM, the walker count above
 * which a configuration takes the spawn kernel's warp-cooperative path, and
 * the radix tile of 8-byte packed records (12, 16 or 24 records per thread;
 * 0 for other record types).  step_ms_default and step_ms_tuned are filled
 * by ddqmc_tune: the kernel time of one step with the default shapes and with
 * the chosen ones, on the same list. */
typedef struct {
    int32_t spawn_blocks_per_sm, radix_blocks_per_sm, merge_blocks_per_sm;
    int32_t copy_blocks_per_sm, scan_blocks_per_sm, partition_blocks_per_sm;
    int32_t heavy_walkers;
    int32_t radix_records_per_thread;
    double step_ms_default, step_ms_tuned;
} ddqmc_tuning;

/* Autotune the launch shapes on the run's current walker list: the list and
 * every piece of device state are saved, each candidate shape is timed over
 * one step (CUDA events per kernel class), the state is restored after each
 * trial and at the end, and each kernel class gets its fastest shape (the
 * classes do not depend on each other's shapes).  The run then continues
 * exactly as if the call had not been made, with the chosen shapes, which are
 * also kept for later runs of the same lattice size, record type and batch
 * kind in this process.  Needs a non-empty list and no sticky error; takes
 * temporary device memory of one list and the blocking cells; waits for the
 * run's stream.  out may be NULL.  Errors: INVALID_ARG, OOM, CUDA, and the
 * run's sticky status. */
int ddqmc_tune(ddqmc_run *run, ddqmc_tuning *out);

/* Use the given launch shapes (each clamped to what its kernel can hold;
 * step_ms_* are ignored) or read the shapes in use. */
int ddqmc_set_tuning(ddqmc_run *run, const ddqmc_tuning *in);
int ddqmc_get_tuning(ddqmc_run *run, ddqmc_tuning *out);

/* ---- batches of runs in one walker store -------------------------------------
 * The paper averages many independent runs per parameter point (Sec. V: 21
 * runs per susceptibility point, several hundred per lattice size).  A batch
 * steps up to DDQMC_MAX_BATCH such runs of one lattice and one guide as a
 * single DDQMC step: one list sorted by (run, bra, ket) with the run id in
 * the key's high bits, one spawn + death/clone launch over all runs, one sort
 * and one merge, one finalize block per run.  Each run keeps its own
 * couplings, gamma, dt, target, initiator threshold, population control,
 * shift, seed, field, estimators and blocking accumulators, and its walker
 * list, estimates and step counts are the same as those of a ddqmc_create
 * run with the same parameters (every random draw is keyed by the run's
 * seed, the step and the walker's configuration).
 * ddqmc_step, ddqmc_step_async, ddqmc_sync, ddqmc_get_counts,
 * ddqmc_get_totals (sums over the runs), the timing calls and ddqmc_destroy
 * take a batch like a run; the per-run queries are the ddqmc_batch_* calls
 * below, and ddqmc_estimators, ddqmc_raw_estimators, ddqmc_blocking_moments,
 * ddqmc_export_walkers and ddqmc_get_state return INVALID_ARG for a batch
 * (ddqmc_import_walkers and ddqmc_annihilate: UNSUPPORTED). */
#define DDQMC_MAX_BATCH 64

/* Parameters of one run of a batch: the arguments of ddqmc_create and the
 * per-run fields of ddqmc_options, with the same meaning and checks. */
typedef struct {
    double Jx, Jy, Jz, gamma, dt;
    int64_t target_walkers;
    int32_t initiator_threshold;
    int32_t control;
    uint64_t seed;
    double damping;
    double shift0;
    int64_t n0;
    int64_t t_eq;
    double field_h;
    int32_t field_axis;
    int32_t reserved;          /* set to 0 */
    double field_theta;        /* as in ddqmc_options */
} ddqmc_run_spec;

/* Create a batch of nruns (1..DDQMC_MAX_BATCH) runs on one lattice and one
 * guide; runs[k] gives run k's parameters.  From opt only capacity_entries,
 * capacity_spawns (shared by all runs; <= 0: the sum of the per-run
 * defaults), cuda_stream, sm_limit and wide_sort_bits are read.  Key
 * layout: up to 31 sites one 64-bit key run << 2N | bra << N | ket (needs
 * 2N + ceil(log2 nruns) <= 63; 8-byte spawn records when it is <= 40), from
 * 32 to 63 sites the run id in the bra word above bit N, or above the hash
 * bits in the hashed order (needs N + ceil(log2 nruns) <= 64); 64 sites
 * need an extra key word and return UNSUPPORTED, as does a batch whose
 * per-block estimator sums (nruns x observables x 8 bytes) do not fit in
 * shared memory.  Errors: as ddqmc_create, UNSUPPORTED.  *out is NULL on
 * error. */
int ddqmc_create_batch(const ddqmc_lattice *lattice, int32_t nruns, const ddqmc_run_spec *runs,
                       const ddqmc_guide *guide, const ddqmc_options *opt, ddqmc_run **out);

/* Retire run `run` of a batch (no counterpart in the paper: it lets a
 * server stop paying for a run whose answer it already has).  From the next
 * step on, the run's configurations spawn nothing and the merge drops them,
 * so the run's list is empty after one step; the other runs of the batch are
 * unaffected (runs never interact).  Issued on the batch's stream, ordered
 * before the steps enqueued after it; not undone.  Errors: INVALID_ARG (not a
 * batch, or run out of range), CUDA. */
int ddqmc_batch_retire(ddqmc_run *batch, int32_t run);

/* Estimates of run `run` of a batch (as ddqmc_estimators). */
int ddqmc_batch_estimators(ddqmc_run *batch, int32_t run, ddqmc_estimates *out);

/* Estimator numerators of run `run` of a batch (as ddqmc_raw_estimators). */
int ddqmc_batch_raw_estimators(ddqmc_run *batch, int32_t run, int64_t *host_out, int32_t cap,
                               int32_t *nobs);

/* Walker list of run `run` of a batch, without the run id (as
 * ddqmc_export_walkers: *n receives that run's length). */
int ddqmc_batch_export_walkers(ddqmc_run *batch, int32_t run, uint64_t *ket, uint64_t *bra,
                               int32_t *re, int32_t *im, int64_t cap, int64_t *n);

/* Scalar state of run `run` of a batch (as ddqmc_get_state; entries counts
 * that run's configurations, status is the batch's). */
int ddqmc_batch_get_state(ddqmc_run *batch, int32_t run, ddqmc_state *out);

/* Annihilation stage on its own (Sec. III.C rule (iii) with the initiator
 * rule of Sec. IV.A): sort spawn records by configuration and merge them into
 * a sorted list.  Records are 16 bytes, { uint64 key; int32 re; int32 im; },
 * key = bra << N | ket; in spawn records bit 63 of the key is set when the
 * parent was an initiator.  One-word keys only: runs of more than 31 sites
 * return UNSUPPORTED.
 * Every record pointer must be 16-byte aligned (INVALID_ARG otherwise).
 *   d_list   m records, strictly increasing keys, no flag bit (device memory);
 *   d_spawns nsp records in any order (device memory, read only);
 *   d_out    room for out_cap records (device memory, must not overlap the
 *            inputs); receives the merged list, *m_out entries: every key keeps
 *            its list population plus its spawns, except that spawns of
 *            non-initiator parents count only on keys present in d_list or on
 *            the diagonal (or always when the run's threshold is 0); zero sums
 *            are dropped.
 * Uses the run's lattice and initiator threshold and the run's spawn buffers
 * as scratch (so it must not overlap a ddqmc_step_async of the same run);
 * issued on the run's stream and waited for.  Errors: INVALID_ARG (a null
 * or misaligned pointer, a negative size), CAPACITY (nsp above the run's spawn capacity, m above its list capacity,
 * or more than out_cap merged entries), OVERFLOW, TIMEOUT, UNSUPPORTED
 * (more than 31 sites), CUDA. */
int ddqmc_annihilate(ddqmc_run *run, const void *d_list, int64_t m, const void *d_spawns, int64_t nsp,
                     void *d_out, int64_t out_cap, int64_t *m_out);

/* The annihilation stage of ddqmc_annihilate for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a property
 * of the library, not of the method.  Some callers cannot call cudaMalloc:
 * their device memory is already reserved by another allocator's pool (a
 * serving engine or a framework's caching allocator that took it up front),
 * or they must stay off the driver's allocation path and its implicit
 * synchronisation.  This entry point allocates nothing and needs no run: its
 * scratch is a fixed array inside the library that every GPU loading the
 * library holds until the process exits (about 30 MB).
 *   lattice, initiator_threshold: as in ddqmc_create (key layout and rule;
 *     at most 31 sites, else UNSUPPORTED);
 *   d_list, m, d_spawns, nsp, d_out, out_cap, *m_out: as in ddqmc_annihilate,
 *     with m <= 1048576 list entries and nsp <= 262144 spawn records
 *     (larger sizes return DDQMC_ERR_CAPACITY before any work);
 *   cuda_stream: stream to issue on (NULL: the default stream); the call
 *     waits for it before returning.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current), so make that first call before any
 * stream capture.  Every call shares the array and leaves its contents
 * behind; calls that overlap on the GPU (from two streams or two host
 * threads at once) race on it and must be serialised by the caller. */
int ddqmc_annihilate_noalloc(const ddqmc_lattice *lattice, int32_t initiator_threshold,
                             const void *d_list, int64_t m, const void *d_spawns, int64_t nsp,
                             void *d_out, int64_t out_cap, int64_t *m_out, void *cuda_stream);

/* Failure-path check of the device waits (no counterpart in the paper: a
 * property of this library).  Every spin of a kernel on a status word written
 * by another block is bounded; when the bound runs out the kernel records a
 * timeout in the device status and returns, so the context stays usable and
 * the host call returns DDQMC_ERR_TIMEOUT.  This call spins one thread on a
 * word that nothing ever sets (about a second on a GB300) and returns what
 * the host sees: DDQMC_ERR_TIMEOUT when the bound works, CUDA on a launch or
 * copy error.  cuda_stream: stream to issue on (NULL: the default stream). */
int ddqmc_wait_selftest(void *cuda_stream);

/* Free every resource of the run (NULL is ignored). */
void ddqmc_destroy(ddqmc_run *run);

/* Static description of a status code. */
const char *ddqmc_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* DDQMC_H */
