// Host-side state of one instance and the runtime helpers shared by the
// single-instance, batch and serving code.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_internal.h"

#include <nvtx3/nvToolsExt.h>

namespace cosm {

// Records msg for cosm_last_error() and returns code.
int fail(int code, const std::string &msg);

// An NVTX range over the scope of one ABI call (host side: create, run,
// readout, batch and server steps), visible to profilers that attach an
// NVTX tool and free otherwise.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace cosm

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(COSM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace cosm {

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;  // elements
    int ensure(size_t count)
    {
        if (count <= cap && p) return COSM_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc((void **)&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return fail(COSM_ERR_NOMEM, "cudaMalloc failed");
        }
        cap = std::max<size_t>(count, 1);
        return COSM_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

}  // namespace cosm

struct cosm_handle {
    using Graph = cosm::Graph;
    template <typename T> using DevBuf = cosm::DevBuf<T>;
    Graph g;                        // host copy, original vertex ids
    cosm_params prm;
    int device = 0;
    int num_sms = 0;
    bool lattice = false;
    int64_t W = 0;                  // total weight
    int64_t wbound = 0;             // sum over colours of the largest |w|, plus the largest |h|
    std::vector<int32_t> slot_of;   // original id -> slot
    std::vector<int32_t> orig_of;   // slot -> original id
    int32_t off[cosm::kMaxColors + 1] = {0};
    int32_t C = 0;
    DevBuf<uint32_t> d_ij;
    DevBuf<int8_t> d_w;
    DevBuf<uint32_t> d_ijs;         // +-1 weights on <= 2^15 slots: records with the sign in bit 31
    DevBuf<int32_t> d_orig;
    DevBuf<int32_t> d_off;          // colour offsets
    int mode = cosm::MODE_GENERAL_;       // kernel variant
    int32_t Q = 0, Wd = 0;          // 2D lattice geometry
    DevBuf<uint8_t> d_wnib;         // 2D lattice block weight bits
    bool fields = false;            // local fields given
    DevBuf<int32_t> d_h;            // local field per slot
    // per run
    DevBuf<unsigned char> d_state;
    DevBuf<int64_t> d_cut;
    DevBuf<int32_t> d_bestp;
    DevBuf<float2> d_alpha;
    DevBuf<cosm::Segment> d_segs;
    DevBuf<int32_t> d_segoff;
    DevBuf<int32_t> d_ready;
    DevBuf<int32_t> d_err;
    DevBuf<int64_t> d_best;
    DevBuf<int8_t> d_spins;
    DevBuf<int64_t> d_energy;       // per replica: energy of the kept readout
    DevBuf<uint32_t> d_bisB;        // per replica: its bisector position
    DevBuf<int64_t> d_trace;        // tracking: [replica][readout] energies
    DevBuf<uint32_t> d_bits;        // tracking: [replica][words] kept spins
    DevBuf<uint32_t> d_qbuf;        // optimal bisector scratch
    DevBuf<int32_t> d_delta;
    DevBuf<uint64_t> d_items;
    int32_t n_trace = 0;            // readouts per trial of the last tracked run
    bool have_trace = false;
    bool bits_valid = false;        // d_bits holds the kept spins of the last run
    // cached host tables
    int64_t alpha_S = -1;
    double alpha_a0 = -1, alpha_ratio = -1;
    std::vector<cosm::Segment> h_segs;
    std::vector<int32_t> h_segoff;
    int64_t sched_tiles = -1, sched_S = -1, sched_G = -1, sched_s0 = -1, sched_s1 = -1;
    bool segs_uploaded = false;
    // state of the last launch
    int replicas = 0;
    int K = 0, threads = 0, occupancy = 0, grid = 0;
    bool block_pairs = false;  // binary32 lattice tiles of two replicas: two 2x2 blocks per thread (even pass)
    bool staged = false;       // binary32 edge lists: colour records staged in shared memory
    size_t smem = 0;
    int64_t tile_stride = 0;  // storage elements per tile
    uint64_t seed = 0;
    int64_t sweep_idx = 0;          // sweeps of the current trial applied to the state
    int64_t target = INT64_MIN;     // success threshold of the last run's cuts
    uint64_t wait_limit_ns = 0;     // bounded waits between segments (0: environment / 20 s)
    int32_t fault = 0;              // host-side fault injection for the next run (COSM_FAULT_*)
    bool have_state = false, have_result = false;
    cudaStream_t stream = nullptr;
    int launches = 0;
};

namespace cosm {

int env_int(const char *name, int dflt);
// narrow_ties: among tiles keeping as many replicas resident, the narrower
// one (more CTAs per SM) instead of the wider one on a full GPU.
int choose_layout(cosm_handle *h, int replicas, bool narrow_ties = false);
int ensure_run_buffers(cosm_handle *h, int replicas);
InstView inst_view(cosm_handle *h);
int upload_alpha(cosm_handle *h, int64_t S, cudaStream_t st);
int launch_finalize(cosm_handle *h, cudaStream_t st);
int launch_opt_readout(cosm_handle *h, bool keep_better, cudaStream_t st);
int single_only(const cosm_graph_desc *g, const cosm_params *p);

}  // namespace cosm
