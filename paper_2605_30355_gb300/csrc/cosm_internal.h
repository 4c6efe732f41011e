// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <stdint.h>
#include <vector_types.h>

#include <string>
#include <vector>

namespace cosm {

constexpr int kMaxColors = 64;
constexpr int kMaxBisectors = 256;
constexpr int kMaxVertices = 65536;

// Work segment of one CTA: sweeps [s_begin, s_end] (1-based, inclusive) of
// one replica tile. A CTA runs its segments in order.
enum SegFlags : int32_t {
    SEG_INIT = 1,     // draw initial phases (Philox) instead of loading state
    SEG_LOAD = 2,     // load the tile's state from global memory
    SEG_WAIT = 4,     // wait until ready[tile] >= s_begin - 1 before loading
    SEG_STORE = 8,    // store the tile's state to global memory at the end
    SEG_SIGNAL = 16,  // publish ready[tile] = s_end after storing
    SEG_READOUT = 32  // bisector readout after the last sweep
};

struct Segment {
    int32_t tile;
    int32_t flags;
    int64_t s_begin;
    int64_t s_end;
};

// Everything a work segment of one instance touches.
struct InstView {
    int32_t n;            // vertices (slots)
    int32_t C;            // colours
    const int32_t *off;   // device: colour offsets into ij / w (C + 1)
    const uint32_t *ij;   // edge records: slot(src) | slot(dst) << 16, colour-major
    const int8_t *w;      // Max-Cut weights, colour-major
    // the same records for +-1 weights on at most 2^15 slots with the weight
    // in bit 0 ([w = -1] | slot(src) << 1 | slot(dst) << 16), so the
    // binary32 edge-list sweep loads one word per edge; nullptr otherwise
    const uint32_t *ijs;
    const int32_t *orig_of;  // slot -> original vertex id (Philox init key)
    // 2D lattice mode: Q = n/4 slots per sublattice, Wd = L2/2 columns;
    // wnib[pass * Q + f] holds the weight bits of the four edges of 2x2
    // block f in that pass (bit set: w = -1)
    const uint8_t *wnib;
    int32_t Q;
    int32_t Wd;
    const float2 *alpha_tab;    // (alpha_s, dwt_step_s) for s = alpha_base ..
    int64_t alpha_base;
    int64_t S;            // sweeps of the trial (readout after sweep S)
    uint64_t seed;
    int32_t replicas;     // valid replicas
    int32_t dwt_period;   // 0 = off
    float window;         // DWT window width in turns
    int32_t flags;        // COSM_NO_DWT | COSM_NO_SCS
    int32_t P;            // bisectors
    int32_t mode;         // KernelMode of this instance
    int32_t K;            // replicas per tile
    uint32_t qwin;        // DWT window width in 2^-32 turns (fixed point)
    void *state;          // [tiles][n_pad][K] phases in the storage type
    int64_t state_tile_stride;  // elements of the storage type per tile
    int64_t *cut;         // [replicas] cut of the kept readout
    int32_t *bestp;       // [replicas] its bisector index (-1: not an equally spaced one)
    // local fields and readout bookkeeping (nullptr / 0 where unused)
    const int32_t *hv;    // [n] local field per slot (eq. (1)), nullptr = none
    int64_t W;            // total Max-Cut weight
    int64_t *energy;      // [replicas] energy (eq. (1)) of the kept readout
    uint32_t *bisB;       // [replicas] position of its bisector (2^-32 turn)
    int32_t track;        // readout period in sweeps, 0 = last sweep only
    int32_t n_trace;      // readouts per trial with tracking
    int64_t *trace;       // [replicas][n_trace] readout energies
    uint32_t *bits;       // [replicas][words] spins of the kept readout (slot order)
    int32_t words;        // (n + 31) / 32
    int32_t paired;       // binary32 lattice tiles: packed f32x2 passes (0 scalar, 1 single blocks, 2 block pairs in the even pass)
    int32_t wrap_p;       // binary32 lattice phases: wrapped on sweeps s with s % wrap_p == 0
    // binary32 edge lists: bytes of the record and weight parts of each of
    // the two shared-memory staging buffers after the tile (0: records are
    // read from global memory)
    int32_t stage_ij;
    int32_t stage_w;
    int32_t *check;       // error word for the checked build's device checks (nullptr: none)
};

// Bytes of the record and weight parts of one staging buffer for colours of
// at most max_ec edges (16-byte chunks covering the colour's range).
inline int32_t stage_ij_bytes(int max_ec) { return (int32_t)(((size_t)(max_ec + 8) * 4 + 15) & ~(size_t)15); }
inline int32_t stage_w_bytes(int max_ec) { return (int32_t)(((size_t)max_ec + 32 + 15) & ~(size_t)15); }

// Single-instance launch: the instance plus the CTAs' segment lists.
struct KernelArgs {
    InstView v;
    const Segment *segs;     // all segments
    const int32_t *seg_off;  // CTA b runs segs[seg_off[b] .. seg_off[b+1])
    int32_t *ready;          // per tile: last sweep whose state is published
    int32_t *err;            // device error word (1 = wait timeout)
    uint64_t wait_limit_ns;
};

// Queue launch: CTAs take units (instance, tile, sweep range, SegFlags)
// from a queue; a whole trial is (1, S, INIT | READOUT | STORE).
struct BatchUnit {
    int32_t inst;
    int32_t tile;
    int32_t flags;
    int32_t pad_;
    int64_t s_begin;
    int64_t s_end;
};
struct BatchArgs {
    const InstView *insts;
    const BatchUnit *units;  // in decreasing cost order
    int32_t n_units;
    int32_t *counter;        // next unit (zeroed before the launch)
};

enum KernelMode { MODE_GENERAL_ = 0, MODE_ACCUM_ = 1, MODE_LATTICE2D_ = 2 };

// Sweeps between wraps of binary32 phases (InstView::wrap_p). One sweep moves
// a phase by at most alpha0 * wbound (wbound: the smaller of the sum over
// colours of the largest |w| in the colour, as a vertex meets at most one
// edge per colour, plus the largest |h|, and the largest sum of |w| over a
// vertex's own edges plus its |h|), and by the twist on the DWT sweeps. 2D lattice: the
// largest P <= 4 for which P sweeps keep a phase wrapped to [-1/2, 1/2] inside
// |g| < 1; edge lists: the largest P <= 12 (preferring a multiple of the
// twist period, whose pass takes the wrap along) that keeps it inside
// |g| < 2, or 0 (every update is wrapped) when one sweep could leave that
// range; 1 for the other modes and storages.
int32_t wrap_period(double alpha0_deg, double dwt_ratio, int dwt_period, int flags, int mode, int storage,
                    int64_t wbound);
// wbound of a colour-major weight array (off: C + 1 colour offsets) and the
// local fields h (nullptr: none).
int64_t colour_weight_bound(const int32_t *off, int C, const int8_t *w, const int32_t *h, int32_t n);
// The largest sum of |w| over one vertex's edges plus its |h| (h may be nullptr).
int64_t vertex_weight_bound(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
                            const int32_t *h);

struct LaunchCfg {
    int mode;      // KernelMode
    int storage;   // 0 f32, 1 f16
    int K;         // replicas per tile
    int threads;   // threads per CTA
    int grid;      // CTAs
    size_t smem;   // dynamic shared bytes
    bool cooperative;
};

// Shared-memory bytes for a tile and the resident CTAs per SM for a config.
// mode: general edge lists, simultaneous update (NO_SCS, per-vertex
// accumulators in shared memory) or the implicit-index 2D lattice.
size_t sweep_smem_bytes(int storage, int K, int n, int P, int mode);
int sweep_occupancy(int storage, int K, int mode, int threads, size_t smem);
int sweep_launch(const LaunchCfg &cfg, const KernelArgs &a, void *stream);

// Batch kernels, one per (storage, K, mode) class.
int batch_occupancy(int storage, int K, int mode, int threads, size_t smem);
int batch_launch(int storage, int K, int mode, int grid, int threads, size_t smem, const BatchArgs &b,
                 void *stream);
// Per-instance finalisation of a batch: CTA i handles instance i.
struct BatchFinal {
    int64_t W;
    int8_t *spins;        // n, original vertex order
    int64_t *best;        // [0] cut, [1] energy, [2] replica, [3] replicas with cut >= target
    int32_t storage;      // 0 f32, 1 f16
    int32_t pad_;
};
int batch_finalize_launch(int count, const InstView *insts, const BatchFinal *fin, void *stream);

// Finalisation: best replica (max cut, ties -> lowest index), energy, spins.
struct FinalArgs {
    int32_t n;
    int32_t replicas;
    int32_t K;
    int32_t storage;
    int32_t P;
    int64_t W;            // total weight
    const void *state;
    int64_t state_tile_stride;
    const int32_t *orig_of;
    const int64_t *cut;
    const int32_t *bestp;
    const int64_t *energy;  // nullptr: select by cut
    const uint32_t *bisB;   // nullptr: bisector from bestp
    const uint32_t *bits;   // nullptr: spins from the phases
    int32_t words;
    int64_t *best;        // [0] cut, [1] energy, [2] replica, [3] replicas with cut >= target
    int8_t *spins;        // n, original vertex order
    int64_t target;       // success threshold (INT64_MIN: every replica counts)
};
int finalize_launch(const FinalArgs &a, void *stream);

// Optimal-bisector readout (Section II-B; Burer, Monteiro and Zhang 2002):
// per replica, the best cut over every bisector position, from the stored
// phases; one CTA per replica at a time, scratch in global memory.
struct OptArgs {
    InstView v;           // graph, state, outputs
    uint32_t *qbuf;       // [grid][n] phase positions of the current replica
    int32_t *delta;       // [grid][n] cut change at each vertex's position
    uint64_t *items;      // [grid][npow2] (position << 32 | delta), sorted
    int32_t npow2;        // power of two >= n
    int32_t keep_better;  // 1: replace the kept readout only if strictly lower in energy
    int32_t storage;      // 0 f32, 1 f16, 2 u16 fixed point
    int32_t pad_;
};
int opt_readout_launch(const OptArgs &a, int grid, void *stream);

// Records the message that cosm_last_error() returns on this thread.
void set_last_error(const std::string &msg);

// Host-side graph tools (cosm_graph.cpp).
struct Graph {
    int32_t n = 0;
    int64_t m = 0;
    std::vector<int32_t> src, dst, w, color;
    int32_t C = 0;
    int32_t dims[3] = {0, 0, 0};
};

int validate_graph(const Graph &g, std::string &why);
int validate_partition(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t C,
                       const int32_t *color, std::string &why);
int color_greedy(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *color,
                 int32_t *C);
int color_misra_gries(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *color,
                      int32_t *C);
int color_torus2d(int32_t L1, int32_t L2, int64_t m, const int32_t *src, const int32_t *dst,
                  int32_t *color);
int color_torus3d(int32_t L1, int32_t L2, int32_t L3, int64_t m, const int32_t *src,
                  const int32_t *dst, int32_t *color);
// Vertex -> slot relabel for shared-memory locality (lattice sublattices).
bool lattice_relabel(const Graph &g, std::vector<int32_t> &slot_of, std::string &why);

}  // namespace cosm
