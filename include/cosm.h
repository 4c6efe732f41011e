/*
 * cosm.h -- C ABI of the GB300 (sm_103a) implementation of Cosm,
 * Collective Switched Motion, a heuristic for sparse Ising / Max-Cut.
 *
 * Problem (eq. (1), Appendix A): a graph G = (V, E) with integer Max-Cut
 * weights w_ij = -J_ij and optional integer local fields h_i. Cosm relaxes each spin to a
 * phase on the circle, applies the finite-magnitude pair update of eq. (6)
 * one edge colour (matching) at a time (Section II-C, eqs. (9)-(12)),
 * perturbs with the dual window twist every DWT period sweeps (Section
 * II-D), anneals the step linearly from alpha_0 to 0 (Section II-B,
 * Table IX), and reads spins out with equally spaced bisectors, keeping the
 * best cut (Alg. 1; Appendix B). Many independent replicas (trials) run at
 * once.
 *
 * Conventions shared by every call
 *  - Status: every int-returning call returns COSM_OK (0) or a negative
 *    COSM_ERR_* code; cosm_last_error() gives a message for the calling
 *    thread's last failure. No C++ exception crosses this boundary.
 *  - Phases are exchanged in turns (1 turn = 360 degrees) in [0, 1).
 *  - Ownership: the library copies every input array it is given and owns
 *    all device memory it allocates; outputs go to caller-owned buffers.
 *  - Pointers documented "host or device" may be either (unified virtual
 *    addressing decides); all others are host pointers.
 *  - Streams are cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls that take a stream are asynchronous on it; results are
 *    valid after cosm_sync() or a later synchronising call on the handle.
 *  - Replica r of a run is an independent trial keyed by (seed, r): initial
 *    phases and DWT angles come from Philox4x32-10 with key = seed and
 *    counters (vertex/4, r, 0, 0) and (sweep, r, 0, 1).
 */
#ifndef COSM_H
#define COSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define COSM_OK 0
#define COSM_ERR_INVALID_ARG -1   /* bad size, pointer, parameter or graph   */
#define COSM_ERR_NOT_A_MATCHING -2 /* a colour class shares a vertex        */
#define COSM_ERR_PARTITION -3     /* a colour index outside [0, n_colors)    */
#define COSM_ERR_TOO_LARGE -4     /* does not fit the shared-memory layout   */
#define COSM_ERR_CUDA -5          /* a CUDA runtime call failed              */
#define COSM_ERR_TIMEOUT -6       /* a bounded device wait gave up           */
#define COSM_ERR_STATE -7         /* call out of order (e.g. no run yet)     */
#define COSM_ERR_NOMEM -8         /* host or device allocation failed        */
#define COSM_ERR_CHECK -9         /* a device-side index check failed (only the
                                   * checked build, libcosm_checked.so, has them) */

/* ---- phase storage ----------------------------------------------------- */
#define COSM_F32 0 /* binary32 phases, FP32 arithmetic                      */
#define COSM_F16 1 /* binary16 phases (half the shared memory), FP32 arithmetic */
#define COSM_Q16 2 /* fixed point: phases on the 2^-16-turn grid as u16,
                    * steps rounded to the grid, exact integer arithmetic   */
#define COSM_BF16 3 /* bfloat16 phases (8 significant bits; quantum 2^-9 turn
                     * near 1/2), FP32 arithmetic                           */

/* ---- variant flags ------------------------------------------------------ */
#define COSM_NO_DWT 1 /* no dual window twist (ablation, Table VII)         */
#define COSM_NO_SCS 2 /* simultaneous generalized-gradient step (eq. (8);
                       * ablation, Table VII)                               */
#define COSM_DWT_RANDOM_DIR 4 /* draw each twist's direction (Section II-D):
                       * -1 when the top bit of word 1 of the Philox draw
                       * that gives the twist angle is set, else +1         */
#define COSM_OPT_BISECTOR 8 /* final readout with the optimal bisector
                       * (Section II-B, after Burer, Monteiro and Zhang
                       * 2002): the best cut over every bisector position,
                       * not only the n_bisectors equally spaced ones; not
                       * with local fields                                  */

/* Sparse graph plus its edge partition (Alg. 1 line 1; Section II-C).
 *  n        number of vertices, 2 <= n <= 65536
 *  m        number of edges, 1 <= m; edges (src[e], dst[e]) with
 *           0 <= src < dst < n, no duplicates
 *  w        integer Max-Cut weight w = -J (Appendix A), 1 <= |w| <= 127
 *  n_colors number of colour classes C (1..64) when color != NULL
 *  color    colour of each edge in [0, C); each class must be a matching.
 *           NULL: the library colours the graph itself (regular lattice
 *           pattern when dims describes an even-sided torus, else greedy).
 *  dims     lattice hint {L1, L2, 0} for a 2D torus with v = r*L2 + c,
 *           {L1, L2, L3} for a 3D torus, {0, 0, 0} for a general graph.
 *           Every edge must be an edge of that torus (a subset is fine);
 *           the hint selects a shared-memory layout, and for the full 2D
 *           torus with +-1 weights and the regular colouring an
 *           implicit-index kernel. A hint that does not match is rejected.
 *  h        local fields h_i of eq. (1) (n entries, |h_i| <= 32767), or
 *           NULL for none. A field acts as a coupling J = h_i to a reference
 *           variable frozen at phase 0: one extra conflict-free sub-sweep
 *           after the colours, and the readout is the fixed half circle
 *           [-1/4, 1/4) turn around the reference (s_i = +1 there).
 *           Single instances only (cosm_create, cosm_solve). */
typedef struct cosm_graph_desc {
    int32_t n;
    int64_t m;
    const int32_t *src;
    const int32_t *dst;
    const int32_t *w;
    int32_t n_colors;
    const int32_t *color;
    int32_t dims[3];
    const int32_t *h;
} cosm_graph_desc;

/* Solver parameters (Tables IX-X; Appendix C).
 *  alpha0_deg   initial step alpha_0 in degrees (paper: 14; 25 for planted)
 *  dwt_ratio    DWT rotation as a multiple of the current alpha (0.5..1.5)
 *  dwt_period   sweeps between DWT events (3 or 6); 0 disables the DWT
 *  window_deg   width of each of the two DWT windows, (0, 180] (paper: 90)
 *  n_bisectors  bisectors over a semicircle at readout, 1..256 (paper: 100)
 *  storage      COSM_F32, COSM_F16, COSM_Q16 or COSM_BF16
 *  flags        COSM_NO_DWT | COSM_NO_SCS | COSM_DWT_RANDOM_DIR |
 *               COSM_OPT_BISECTOR
 *  track_period 0: one readout after the last sweep. T > 0: mid-anneal best
 *               tracking: a readout after every sweep s with s % T == 0 and
 *               after the last sweep, each replica keeping the readout of
 *               lowest energy (ties: the earlier) and its spins, and every
 *               readout's energy recorded (cosm_get_trace; the energy
 *               trajectories of Fig. 10 sample every 1000 sweeps). Single
 *               instances only.                                            */
typedef struct cosm_params {
    double alpha0_deg;
    double dwt_ratio;
    int32_t dwt_period;
    double window_deg;
    int32_t n_bisectors;
    int32_t storage;
    int32_t flags;
    int32_t track_period;
} cosm_params;

typedef struct cosm_handle cosm_handle;

/* Fills the paper's common Gset settings (Table IX; Table X for G72/G77/
 * G81): alpha0 14 deg, ratio 0.5, period 3, window 90 deg, 100 bisectors,
 * FP32 storage, no flags. */
void cosm_default_params(cosm_params *p);

/* Validates the graph and partition (every edge has a colour in range,
 * each colour class is a matching), builds the device layout and copies it
 * to the current CUDA device. Inputs are copied; the caller keeps them.
 * Errors: INVALID_ARG, NOT_A_MATCHING, PARTITION, TOO_LARGE, CUDA, NOMEM. */
int cosm_create(const cosm_graph_desc *g, const cosm_params *p, cosm_handle **out);

/* Releases the handle and its device memory. NULL is a no-op. */
void cosm_destroy(cosm_handle *h);

/* Runs one full trial (Alg. 1) for each of `replicas` replicas: random
 * phases, `sweeps` sweeps (each: C sub-sweeps in colour order, then the DWT
 * when sweep % dwt_period == 0, then the step update), then the bisector
 * readout with exact int64 cuts and best-state tracking. target_cut is the
 * success threshold of Appendix A's P_s: the run counts the replicas whose
 * kept cut is >= target_cut (cosm_get_success); INT64_MIN counts every
 * replica. Asynchronous on `stream`. sweeps in [1, 2^31), replicas in
 * [1, 2^24). Errors: INVALID_ARG, TOO_LARGE, CUDA, NOMEM. */
int cosm_run(cosm_handle *h, int64_t sweeps, int32_t replicas, uint64_t seed, int64_t target_cut,
             void *stream);

/* Part of a trial: sweeps s_from..s_to (1 <= s_from <= s_to <= sweeps) of
 * a `sweeps`-sweep trial, with the step schedule of the whole trial (Table
 * IX's linear ramp over `sweeps`). s_from == 1 starts the trial from the
 * seed's random phases, as cosm_run; s_from > 1 continues the current
 * state, which must have reached sweep s_from - 1 (by an earlier range or
 * cosm_import_state; else COSM_ERR_STATE) with the same replica count and
 * seed (else INVALID_ARG). The range that ends at s_to == sweeps reads out
 * as cosm_run does, with target_cut as there; earlier ranges only sweep.
 * Splitting a trial into ranges gives the same phases and cuts, bit for
 * bit, as one cosm_run. Asynchronous on `stream`. */
int cosm_run_range(cosm_handle *h, int64_t sweeps, int64_t s_from, int64_t s_to, int32_t replicas,
                   uint64_t seed, int64_t target_cut, void *stream);

/* Number of replicas of the last readout whose kept cut reached the run's
 * target_cut (Appendix A: P_s = count / replicas). Synchronises.
 * COSM_ERR_STATE before a readout. */
int cosm_get_success(cosm_handle *h, int64_t *count);

/* Waits for the handle's last launch and reports device-side errors
 * (COSM_ERR_TIMEOUT if a bounded wait between work segments gave up). */
int cosm_sync(cosm_handle *h);

/* Best replica of the last run or readout: lowest energy, ties to the
 * smallest replica index (without fields: the maximum cut); its cut, its
 * energy H = sum w s_i s_j - sum h s_i = W - 2 cut - sum h s_i (eq. (1));
 * spins (n entries of +1/-1, host or device) in original vertex order: the
 * rounding of that replica's phases at the kept readout's bisector (with
 * tracking, the spins saved when that readout was taken).
 * Any output pointer may be NULL. Synchronises. */
int cosm_get_best(cosm_handle *h, int64_t *cut, int64_t *energy, int32_t *replica, int8_t *spins);

/* Per-replica cut and bisector index of the kept readout of the last run
 * or readout (`replicas` entries each, host or device; either may be NULL).
 * The index is p of the bisector B_p = floor(p 2^31 / P) when the equally
 * spaced bisectors chose it, -1 for the fixed half circle (local fields)
 * and for the optimal bisector. */
int cosm_get_replica_cuts(cosm_handle *h, int64_t *cuts, int32_t *best_p);

/* Per-replica energy of eq. (1), fields included, of the kept readout
 * (`replicas` entries, host or device). Synchronises. */
int cosm_get_replica_energies(cosm_handle *h, int64_t *energies);

/* Per-replica position of the kept readout's bisector, in 2^-32 turn: spin
 * s_v = +1 iff ((floor(x_v 2^32) - B) mod 2^32) < 2^31 (`replicas`
 * entries, host or device). Synchronises. */
int cosm_get_replica_bisectors(cosm_handle *h, uint32_t *B);

/* Energy trace of the last run with track_period = T > 0: row-major
 * [replica][k], k = 0 .. ceil(sweeps / T) - 1, the energy of readout k
 * (after sweep min((k + 1) T, sweeps)); `count` must equal replicas times
 * that number (host or device). COSM_ERR_STATE without tracking. */
int cosm_get_trace(cosm_handle *h, int64_t *trace, int64_t count);

/* Exports all replicas' phases as FP64 turns in [0, 1), row-major
 * [replica][vertex] in original vertex order (host or device pointer).
 * The conversion from the stored FP32/FP16 value is exact. */
int cosm_get_state(cosm_handle *h, double *phases);

/* Replaces the state with `replicas` x n phases (FP64 turns, [replica]
 * [vertex], host or device), rounded to nearest into the storage type, and
 * sets the seed used by cosm_step for DWT angles (sweep index 0). Used to
 * replay states. */
int cosm_set_state(cosm_handle *h, const double *phases, int32_t replicas, uint64_t seed);

/* Checkpoint of the state in its own storage type (no counterpart in the
 * paper; the state of Alg. 1 between sweeps). Export writes replicas x n
 * elements [replica][vertex] in original vertex order to `phases` (host or
 * device): float for COSM_F32, the 16-bit words of binary16 / bfloat16 /
 * the 2^-16-turn fixed point otherwise; `storage` must be the handle's
 * (else INVALID_ARG). *sweep_idx (may be NULL) gets the number of sweeps of
 * the current trial the state has had. Binary32 phases are exported as
 * stored: a representative of the turn that may lie outside [0, 1).
 * Import replaces the state with such a checkpoint, with its replica
 * count, seed (for the remaining DWT angles) and sweep index; a
 * cosm_run_range from sweep_idx + 1 then continues the trial. On a handle
 * created from the same graph and parameters the continuation equals the
 * uninterrupted trial bit for bit. The checkpoint holds the phases only:
 * with track_period > 0 the readouts kept before it are not carried over
 * to another handle. Export synchronises. */
int cosm_export_state(cosm_handle *h, void *phases, int32_t storage, int64_t *sweep_idx);
int cosm_import_state(cosm_handle *h, const void *phases, int32_t storage, int32_t replicas, uint64_t seed,
                      int64_t sweep_idx);

/* Failure detection (no counterpart in the paper). A trial split between
 * two CTAs hands its state over through global memory; the CTA running the
 * tail waits for the head's ready flag for at most `seconds` (default: the
 * environment variable COSM_WAIT_LIMIT_S, else 20 s), then gives up on that
 * tile, sets the handle's error word and returns; cosm_sync then reports
 * COSM_ERR_TIMEOUT and the handle stays usable. INVALID_ARG outside
 * (0, 3600]. */
int cosm_set_wait_limit(cosm_handle *h, double seconds);

/* Host-side fault injection for testing the bounded waits: with
 * COSM_FAULT_DROP_SIGNAL the next run's split tiles do not publish their
 * ready flags, so every tail's wait runs out (COSM_ERR_TIMEOUT at
 * cosm_sync, after the wait limit); the run after that is normal. 0 clears
 * it. Nothing faults on the device: the kernel only stops waiting. */
#define COSM_FAULT_DROP_SIGNAL 1
int cosm_inject_fault(cosm_handle *h, int32_t kind);

/* Applies exactly one sweep with index `sweep` (1-based; the DWT fires when
 * sweep % dwt_period == 0) and step `alpha` (turns, FP32) to every replica
 * of the current state. The DWT rotation is dwt_ratio * alpha. With
 * COSM_Q16 both are rounded to the nearest 2^-16-turn quantum. */
int cosm_step(cosm_handle *h, int64_t sweep, float alpha, void *stream);

/* Readout of the current state without sweeping (Alg. 1 final loop: the
 * equally spaced bisectors, the optimal bisector with COSM_OPT_BISECTOR,
 * the fixed half circle with local fields), for replayed-state checks;
 * results via cosm_get_best and cosm_get_replica_*. */
int cosm_readout(cosm_handle *h, void *stream);

/* One-shot call for host-resident inputs and outputs: create, run, read
 * the best result and per-replica cuts, destroy. replica_cuts may be NULL;
 * spins may be NULL. Synchronous. */
int cosm_solve(const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps, int32_t replicas,
               uint64_t seed, int64_t *best_cut, int64_t *energy, int8_t *spins,
               int64_t *replica_cuts);

/* ---- ragged batches: many instances of uneven size in one run ---------- */
typedef struct cosm_batch cosm_batch;

/* Creates `count` instances, each exactly as cosm_create would (graphs[i];
 * params[i], or params[0] for all when shared_params != 0). Inputs are
 * copied. Local fields, tracking and COSM_OPT_BISECTOR are single-instance
 * features (COSM_ERR_INVALID_ARG here). Errors as cosm_create, with the
 * failing instance in the message. */
int cosm_batch_create(int32_t count, const cosm_graph_desc *graphs, const cosm_params *params,
                      int32_t shared_params, cosm_batch **out);

/* Runs one trial (Alg. 1) per replica of every instance i: sweeps[i] sweeps,
 * replicas[i] replicas, seed seeds[i] (host arrays of `count`). Replica
 * tiles of all instances are work units; units of one class (storage, tile
 * width, kernel, threads per CTA, CTAs per SM) share one persistent launch
 * draining a queue ordered by decreasing cost; class launches overlap on
 * forked streams; the run is
 * captured into a CUDA graph once and replayed while its layout holds.
 * Per instance, results equal those of cosm_run with the same arguments.
 * Asynchronous: ordered after earlier work on `stream`, and later work on
 * `stream` is ordered after it. */
int cosm_batch_run(cosm_batch *b, const int64_t *sweeps, const int32_t *replicas, const uint64_t *seeds,
                   void *stream);

/* Waits for the batch's last run. */
int cosm_batch_sync(cosm_batch *b);

/* Results of instance i of the last run, as cosm_get_best /
 * cosm_get_replica_cuts / cosm_get_state for that instance. */
int cosm_batch_get_best(cosm_batch *b, int32_t i, int64_t *cut, int64_t *energy, int32_t *replica,
                        int8_t *spins);
int cosm_batch_get_replica_cuts(cosm_batch *b, int32_t i, int64_t *cuts, int32_t *best_p);
int cosm_batch_get_state(cosm_batch *b, int32_t i, double *phases);

/* Autotuner: times a short run (probe_sweeps sweeps per instance, the given
 * replica counts) of eight layouts and keeps the fastest for later runs:
 * the tile policies -- per instance the tile that keeps the most replicas
 * resident per SM when the GPU is full (ties to the wider tile), the
 * narrowest tile, the single-instance rule for the instance's own replica
 * count, or the first rule with ties to the narrower tile -- each with the
 * per-instance thread rule, the first policy with 128, 256 or 512 threads
 * per CTA forced, and the last with 256. Instances of one
 * kernel, thread count and occupancy form a class: one persistent launch.
 * With the environment variable COSM_TUNE_CACHE naming a file, a choice for
 * the same batch shape is read from it, and new choices are appended. */
int cosm_batch_tune(cosm_batch *b, const int32_t *replicas, int64_t probe_sweeps, void *stream);

/* out[0] instances, out[1] classes, out[2] units, out[3] kernel launches
 * per run, out[4] graphs built, out[5] tile policy (0 full-GPU rule, 1
 * narrowest tile, 2 single-instance rule, 3 full-GPU rule with ties to the
 * narrower tile), out[6] forced threads (0 = rule), out[7] CTAs over all
 * classes. */
int cosm_batch_info(cosm_batch *b, int64_t out[8]);

/* Layout of instance i in the last run, as cosm_layout gives it for a
 * single instance (out[0] replicas per tile, out[1] threads per CTA, out[2]
 * shared bytes per CTA, ...). COSM_ERR_STATE before a run. */
int cosm_batch_layout(cosm_batch *b, int32_t i, int32_t out[8]);

/* Releases the batch and all its instances. NULL is a no-op. */
void cosm_batch_destroy(cosm_batch *b);

/* ---- serving: continuous batching of requests ------------------------- */
typedef struct cosm_server cosm_server;

/* memory_budget: device bytes the admitted requests may hold together (a
 * request's graph, phases of all its replicas, outputs, step table);
 * max_active: requests on the device at once; chunk_sweeps: sweeps each
 * active request advances per launch; threads: threads per CTA (0 = rule). */
typedef struct cosm_server_config {
    int64_t memory_budget;
    int32_t max_active;
    int32_t chunk_sweeps;
    int32_t threads;
    int32_t reserved;
} cosm_server_config;

/* status: 0 queued, 1 running, 2 target reached, 3 trials used up without
 * reaching it, < 0 a COSM_ERR_* code. Times are seconds on the server's
 * steady clock; ttt = time from submission to the end of the first trial
 * whose best cut reached the target (< 0 if none). updates: edge-replica
 * updates spent. best_* refer to the best trial so far. */
typedef struct cosm_request_result {
    int32_t status;
    int32_t trials;
    int64_t best_cut;
    int64_t energy;
    int32_t best_trial;
    int32_t best_replica;
    double t_submit;
    double t_admit;
    double t_done;
    double ttt;
    int64_t updates;
} cosm_request_result;

/* Defaults: 8 GiB budget, 64 active requests, 500-sweep chunks. */
void cosm_server_default_config(cosm_server_config *c);

/* Starts a server on the current device with its own worker thread. A
 * request, once admitted (in arrival order, when a slot is free and its
 * footprint fits the budget), keeps its phases on the device; all active
 * requests advance together, one chunk of sweeps per launch; a request
 * retires when a trial's best cut reaches its target or after max_trials
 * trials, freeing its slot and memory. Trial t uses the seed
 * seed + t * 0x9E3779B97F4A7C15, so a request's result is the same alone
 * and in any mix. No paper counterpart (the paper runs batches of trials,
 * Section III-B). */
int cosm_server_create(const cosm_server_config *cfg, cosm_server **out);

/* Queues a request (the graph is copied): trials of `sweeps` sweeps and
 * `replicas` replicas each (Alg. 1 per replica), until a trial's best cut
 * >= target_cut or max_trials trials. Returns at once with *id.
 * COSM_ERR_TOO_LARGE if its footprint exceeds the whole budget;
 * COSM_ERR_INVALID_ARG for local fields, tracking or COSM_OPT_BISECTOR
 * (single-instance features). */
int cosm_server_submit(cosm_server *s, const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps,
                       int32_t replicas, uint64_t seed, int64_t target_cut, int32_t max_trials,
                       int64_t *id);

/* Current state of a request (non-blocking). */
int cosm_server_poll(cosm_server *s, int64_t id, cosm_request_result *out);

/* Waits up to timeout_s seconds for a request to retire; COSM_ERR_TIMEOUT
 * if it has not (out still receives its current state). */
int cosm_server_wait(cosm_server *s, int64_t id, double timeout_s, cosm_request_result *out);

/* Spins (+1/-1, n entries, original order) of a retired request's best trial. */
int cosm_server_get_spins(cosm_server *s, int64_t id, int8_t *spins);

/* out[0] queued, out[1] active, out[2] retired, out[3] chunks run, out[4]
 * kernel launches, out[5] most requests active at once, out[6] peak
 * admitted footprint (bytes), out[7] current footprint. */
int cosm_server_stats(cosm_server *s, int64_t out[8]);

/* Stops the worker after its current chunk and releases everything. */
void cosm_server_destroy(cosm_server *s);

/* Kernel layout chosen by cosm_create / cosm_run, for inspection:
 * out[0] replicas per CTA, out[1] threads per CTA, out[2] dynamic shared
 * bytes per CTA, out[3] resident CTAs per SM, out[4] lattice layout (1/0),
 * out[5] CTAs in the last launch, out[6] kernel launches in the last run. */
int cosm_layout(cosm_handle *h, int32_t out[8]);

/* ---- edge colourings (host only; Alg. 1 line 1) ------------------------ */

/* Greedy colouring of Section II-B: edges in the given order each take the
 * lowest colour free at both endpoints. Writes color[m] and *n_colors. */
int cosm_color_greedy(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                      int32_t *color, int32_t *n_colors);

/* Misra-Gries edge colouring with at most Delta + 1 colours (Vizing bound;
 * J. Misra and D. Gries, Inf. Proc. Letters 41, 1992). */
int cosm_color_misra_gries(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           int32_t *color, int32_t *n_colors);

/* Regular lattice patterns (Section II-B, Appendix B). 2D torus, 4 colours
 * in the order: horizontal edges leaving an even column, vertical edges
 * leaving an even row, horizontal from an odd column, vertical from an odd
 * row (each consecutive pair acts inside disjoint 2x2 blocks). 3D torus, 6
 * colours: 3 * parity + axis. Sides must be even and >= 4. */
int cosm_color_torus2d(int32_t L1, int32_t L2, int64_t m, const int32_t *src, const int32_t *dst,
                       int32_t *color);
int cosm_color_torus3d(int32_t L1, int32_t L2, int32_t L3, int64_t m, const int32_t *src,
                       const int32_t *dst, int32_t *color);

/* Partition check: COSM_OK, COSM_ERR_PARTITION (colour out of range) or
 * COSM_ERR_NOT_A_MATCHING (a class shares a vertex). */
int cosm_validate_partition(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            int32_t n_colors, const int32_t *color);

/* QUBO input (the general Ising form of eq. (1)): minimise
 * f(x) = sum_k qv[k] x_qi[k] x_qj[k] over x in {0,1}^n, given as nnz
 * triplets (duplicates add up; i == j is a linear term). With
 * x_i = (1 + s_i) / 2 it becomes 4 f(x) = H(s) + offset, H of eq. (1) with
 * Max-Cut weights w_ij = c_ij = Q_ij + Q_ji (i < j) and fields
 * h_i = -(sum_j c_ij + 2 Q_ii), offset = sum c_ij + 2 sum Q_ii. Host code,
 * no device work. src, dst, w: room for nnz edges (caller-owned, host);
 * *m gets the edge count (pairs with c_ij != 0, sorted by (src, dst));
 * h: n entries. Errors: INVALID_ARG (an index outside [0, n)), TOO_LARGE
 * (a weight above 127 or a field above 32767 in magnitude). */
int cosm_qubo_to_ising(int32_t n, int64_t nnz, const int32_t *qi, const int32_t *qj, const int64_t *qv,
                       int32_t *src, int32_t *dst, int32_t *w, int64_t *m, int32_t *h, int64_t *offset);

/* Measurement support (no counterpart in the paper): shared-memory read
 * bandwidth of the current device, for the roofline of the sweep kernel.
 * Two CTAs of 1024 threads per SM stream conflict-free 16-byte words
 * `iters` x 8 times; outputs bytes per SM clock (per SM) and GB/s (whole
 * device, at the clock the probe ran at). Allocates 12 bytes of device
 * memory and synchronises the device. */
int cosm_probe_smem(int32_t iters, double *bytes_per_clk_per_sm, double *gbps);

/* Measurement support (no counterpart in the paper): the FP32 arithmetic
 * issue rate of the current device, for the arithmetic roofline of the
 * sweep kernels. Two CTAs of 1024 threads per SM run 8 independent chains
 * of fused multiply-adds per thread, iters x 8 per chain: scalar
 * fma.rn.f32 (one operation per lane) and packed fma.rn.f32x2 (two
 * operations per lane). Outputs FP32 operations per SM clock per SM for
 * each form (either pointer may be NULL). Allocates 12 bytes of device
 * memory and synchronises the device. Errors: INVALID_ARG (iters < 1),
 * CUDA, NOMEM. */
int cosm_probe_fp32(int32_t iters, double *ops_per_clk_per_sm, double *ops_per_clk_per_sm_packed);

/* No-allocation run, for callers that cannot allocate device memory (code
 * inside a host application that owns every device allocation, a plugin
 * with no allocator, a process whose device memory is already committed).
 * The paper has no counterpart; it is the edge-list sweep of cosm_run for
 * one trial per replica, with the kernel's scratch -- packed edge records,
 * weights, the step table, the work list and an error word -- held in a
 * fixed static device array of COSM_STATIC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits. It needs
 *   5 m + 4 n + 8 sweeps + 28 ceil(replicas / tile) + 4 (C + 1) + 8 bytes
 * (C colours; tile = 1 replica for COSM_F32, 2 for COSM_F16), in eight
 * parts -- records 4 m, weights m, vertex ids 4 n, step table 8 sweeps,
 * work list 24 and offsets 4 per tile plus 4, error word 4, colour offsets
 * 4 (C + 1) -- each rounded up to 256 bytes; larger problems fail with
 * COSM_ERR_TOO_LARGE before any device work. It calls no cudaMalloc or
 * cudaFree. Inputs are host arrays as for cosm_create (the lattice hint is
 * ignored; color may be NULL for the greedy colouring; no local fields,
 * COSM_F32 or COSM_F16 storage, flags COSM_NO_DWT | COSM_NO_SCS only,
 * track_period 0, else COSM_ERR_INVALID_ARG); outputs are
 * caller-owned DEVICE buffers of `replicas` entries: each replica's best
 * cut and best bisector index, the same values cosm_run + cosm_get_replica_cuts
 * give for that graph without a lattice hint. Both must be device (or
 * managed) memory of the current device, else COSM_ERR_INVALID_ARG before
 * any device work. Asynchronous on `stream`; a stream that is capturing is
 * refused with COSM_ERR_INVALID_ARG (the scratch is filled from host
 * tables that are released when the call returns).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. All calls share the array and it keeps the last call's contents:
 * calls on one stream are ordered, but calls that may overlap on the GPU
 * (other streams, other host threads) race and must not be issued. */
#define COSM_STATIC_SCRATCH_BYTES (8u << 20)
int cosm_solve_static(const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps, int32_t replicas,
                      uint64_t seed, int64_t *replica_cuts, int32_t *best_p, void *stream);

/* Message for the calling thread's last failed call ("" if none). */
const char *cosm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* COSM_H */
