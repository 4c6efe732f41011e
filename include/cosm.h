/*
 * cosm.h -- C ABI of the GB300 (sm_103a) implementation of Cosm,
 * Collective Switched Motion, a heuristic for sparse Ising / Max-Cut.
 *
 * Problem (eq. (1), Appendix A): a graph G = (V, E) with integer Max-Cut
 * weights w_ij = -J_ij and no local fields. Cosm relaxes each spin to a
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

/* ---- phase storage (arithmetic is FP32 in both) ------------------------ */
#define COSM_F32 0 /* binary32 phases                                       */
#define COSM_F16 1 /* binary16 phases: half the shared memory per replica   */

/* ---- variant flags (ablations of Table VII) ---------------------------- */
#define COSM_NO_DWT 1 /* no dual window twist                              */
#define COSM_NO_SCS 2 /* simultaneous generalized-gradient step (eq. (8))  */

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
 *           The hint only selects a faster shared-memory layout; it is
 *           checked against the edges and rejected if it does not match. */
typedef struct cosm_graph_desc {
    int32_t n;
    int64_t m;
    const int32_t *src;
    const int32_t *dst;
    const int32_t *w;
    int32_t n_colors;
    const int32_t *color;
    int32_t dims[3];
} cosm_graph_desc;

/* Solver parameters (Tables IX-X; Appendix C).
 *  alpha0_deg   initial step alpha_0 in degrees (paper: 14; 25 for planted)
 *  dwt_ratio    DWT rotation as a multiple of the current alpha (0.5..1.5)
 *  dwt_period   sweeps between DWT events (3 or 6); 0 disables the DWT
 *  window_deg   width of each of the two DWT windows, (0, 180] (paper: 90)
 *  n_bisectors  bisectors over a semicircle at readout, 1..256 (paper: 100)
 *  storage      COSM_F32 or COSM_F16
 *  flags        COSM_NO_DWT | COSM_NO_SCS                                  */
typedef struct cosm_params {
    double alpha0_deg;
    double dwt_ratio;
    int32_t dwt_period;
    double window_deg;
    int32_t n_bisectors;
    int32_t storage;
    int32_t flags;
    int32_t reserved;
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
 * readout with exact int64 cuts and best-state tracking. Asynchronous on
 * `stream`. sweeps in [1, 2^31), replicas in [1, 2^24).
 * Errors: INVALID_ARG, TOO_LARGE, CUDA, NOMEM. */
int cosm_run(cosm_handle *h, int64_t sweeps, int32_t replicas, uint64_t seed, void *stream);

/* Waits for the handle's last launch and reports device-side errors
 * (COSM_ERR_TIMEOUT if a bounded wait between work segments gave up). */
int cosm_sync(cosm_handle *h);

/* Best replica of the last run or readout: maximum cut, ties to the
 * smallest replica index; energy H = sum w s_i s_j = W - 2 cut (eq. (1),
 * h = 0); spins (n entries of +1/-1, host or device) in original vertex
 * order, the rounding of that replica's phases at its best bisector.
 * Any output pointer may be NULL. Synchronises. */
int cosm_get_best(cosm_handle *h, int64_t *cut, int64_t *energy, int32_t *replica, int8_t *spins);

/* Per-replica best cut and best bisector index of the last run or readout
 * (`replicas` entries each, host or device; either may be NULL). */
int cosm_get_replica_cuts(cosm_handle *h, int64_t *cuts, int32_t *best_p);

/* Exports all replicas' phases as FP64 turns in [0, 1), row-major
 * [replica][vertex] in original vertex order (host or device pointer).
 * The conversion from the stored FP32/FP16 value is exact. */
int cosm_get_state(cosm_handle *h, double *phases);

/* Replaces the state with `replicas` x n phases (FP64 turns, [replica]
 * [vertex], host or device), rounded to nearest into the storage type, and
 * sets the seed used by cosm_step for DWT angles. Used to replay states. */
int cosm_set_state(cosm_handle *h, const double *phases, int32_t replicas, uint64_t seed);

/* Applies exactly one sweep with index `sweep` (1-based; the DWT fires when
 * sweep % dwt_period == 0) and step `alpha` (turns, FP32) to every replica
 * of the current state. The DWT rotation is dwt_ratio * alpha. */
int cosm_step(cosm_handle *h, int64_t sweep, float alpha, void *stream);

/* Bisector readout of the current state without sweeping (Alg. 1 final
 * loop), for replayed-state checks; results via cosm_get_best and
 * cosm_get_replica_cuts. */
int cosm_readout(cosm_handle *h, void *stream);

/* One-shot call for host-resident inputs and outputs: create, run, read
 * the best result and per-replica cuts, destroy. replica_cuts may be NULL;
 * spins may be NULL. Synchronous. */
int cosm_solve(const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps, int32_t replicas,
               uint64_t seed, int64_t *best_cut, int64_t *energy, int8_t *spins,
               int64_t *replica_cuts);

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

/* Measurement support (no counterpart in the paper): shared-memory read
 * bandwidth of the current device, for the roofline of the sweep kernel.
 * Two CTAs of 1024 threads per SM stream conflict-free 16-byte words
 * `iters` x 8 times; outputs bytes per SM clock (per SM) and GB/s (whole
 * device, at the clock the probe ran at). Allocates 12 bytes of device
 * memory and synchronises the device. */
int cosm_probe_smem(int32_t iters, double *bytes_per_clk_per_sm, double *gbps);

/* No-allocation run, for callers that cannot allocate device memory (code
 * inside a host application that owns every device allocation, a plugin
 * with no allocator, a process whose device memory is already committed).
 * The paper has no counterpart; it is the edge-list sweep of cosm_run for
 * one trial per replica, with the kernel's scratch -- packed edge records,
 * weights, the step table, the work list and an error word -- held in a
 * fixed static device array of COSM_STATIC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits. It needs
 *   5 m + 4 n + 8 sweeps + 28 ceil(replicas / tile) bytes
 * (each part rounded up to 256 bytes); larger problems fail with
 * COSM_ERR_TOO_LARGE before any device work. It calls no cudaMalloc or
 * cudaFree. Inputs are host arrays as for cosm_create (the lattice hint is
 * ignored; color may be NULL for the greedy colouring); outputs are
 * caller-owned DEVICE buffers of `replicas` entries: each replica's best
 * cut and best bisector index, the same values cosm_run + cosm_get_replica_cuts
 * give for that graph without a lattice hint. Asynchronous on `stream`.
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
