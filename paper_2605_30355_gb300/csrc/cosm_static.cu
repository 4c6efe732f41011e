// cosm_solve_static: a run of the edge-list sweep kernel that allocates no
// device memory. Some callers cannot call cudaMalloc -- code running inside
// a memory-pool-less runtime, a plugin whose host owns every device
// allocation, or a process whose allocator is already exhausted -- yet they
// can pass device buffers for the results. For them the kernel's scratch
// (packed edge records, weights, the step table, the work-segment list and
// the error word) lives in the fixed array below, which is part of the
// library image and is held by every GPU that loads the library until the
// process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_internal.h"

using namespace cosm;

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB, see COSM_STATIC_SCRATCH_BYTES
static_assert(kScratchBytes == COSM_STATIC_SCRATCH_BYTES, "header and library disagree");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device with that device
// current. In host code the symbol names a host-side stand-in, so only this
// address may be handed to kernels.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

int fail(int code, const std::string &msg)
{
    set_last_error(msg);  // reported by cosm_last_error()
    return code;
}

int scratch_address(unsigned char **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(COSM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(COSM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return COSM_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int cosm_solve_static(const cosm_graph_desc *gd, const cosm_params *p, int64_t sweeps,
                                 int32_t replicas, uint64_t seed, int64_t *replica_cuts,
                                 int32_t *best_p, void *stream)
{
    if (!gd || !p || !replica_cuts || !best_p) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!gd->src || !gd->dst || !gd->w) return fail(COSM_ERR_INVALID_ARG, "NULL edge arrays");
    if (sweeps < 1 || sweeps >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "sweeps must be in [1, 2^31)");
    if (replicas < 1 || replicas >= (1 << 24)) return fail(COSM_ERR_INVALID_ARG, "replicas must be in [1, 2^24)");
    if (!(p->alpha0_deg >= 0.0 && p->alpha0_deg < 180.0) || !(p->dwt_ratio >= 0.0 && p->dwt_ratio <= 16.0) ||
        p->dwt_period < 0 || !(p->window_deg > 0.0 && p->window_deg <= 180.0) || p->n_bisectors < 1 ||
        p->n_bisectors > kMaxBisectors || (p->storage != COSM_F32 && p->storage != COSM_F16) ||
        (p->flags & ~(COSM_NO_DWT | COSM_NO_SCS)) || p->track_period != 0)
        return fail(COSM_ERR_INVALID_ARG, "invalid parameters");
    if (gd->h) return fail(COSM_ERR_INVALID_ARG, "local fields are not supported without allocation");
    if (gd->n < 2 || gd->n > kMaxVertices || gd->m < 1 || gd->m > ((int64_t)1 << 26))
        return fail(COSM_ERR_INVALID_ARG, "n must be in [2, 65536] and m in [1, 2^26]");
    // the outputs must be device memory of the current device: a host
    // address handed to the kernel would fault or write the wrong memory
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(COSM_ERR_CUDA, "cudaGetDevice failed");
    for (const void *q : {(const void *)replica_cuts, (const void *)best_p}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
            cudaGetLastError();
            return fail(COSM_ERR_INVALID_ARG, "an output buffer is not a CUDA allocation");
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return fail(COSM_ERR_INVALID_ARG, "the output buffers must be device memory of the current device");
    }
    // the scratch is filled from host tables released on return, which a
    // stream capture would record by address: capturing streams are refused
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
            cudaGetLastError();
            return fail(COSM_ERR_INVALID_ARG, "invalid stream");
        }
        if (cs != cudaStreamCaptureStatusNone)
            return fail(COSM_ERR_INVALID_ARG, "cosm_solve_static cannot be called on a capturing stream");
    }

    // graph checks and partition, as cosm_create does (host memory only)
    Graph g;
    g.n = gd->n;
    g.m = gd->m;
    g.src.assign(gd->src, gd->src + gd->m);
    g.dst.assign(gd->dst, gd->dst + gd->m);
    g.w.assign(gd->w, gd->w + gd->m);
    std::string why;
    int rc = validate_graph(g, why);
    if (rc) return fail(rc, why);
    g.color.assign((size_t)g.m, 0);
    if (gd->color) {
        g.color.assign(gd->color, gd->color + gd->m);
        g.C = gd->n_colors;
    } else {
        color_greedy(g.n, g.m, g.src.data(), g.dst.data(), g.color.data(), &g.C);
    }
    rc = validate_partition(g.n, g.m, g.src.data(), g.dst.data(), g.C, g.color.data(), why);
    if (rc) return fail(rc, why);

    // layout: the smallest replica tile of the storage type, one tile per CTA
    const int mode = (p->flags & COSM_NO_SCS) ? MODE_ACCUM_ : MODE_GENERAL_;
    const int K = p->storage == COSM_F32 ? 1 : 2;
    const int threads = 256;
    const size_t smem = sweep_smem_bytes(p->storage, K, g.n, p->n_bisectors, mode);
    if (smem > 227 * 1024 || sweep_occupancy(p->storage, K, mode, threads, smem) < 1)
        return fail(COSM_ERR_TOO_LARGE, "a replica does not fit in shared memory");
    const int64_t tiles = (replicas + K - 1) / K;
    if (tiles > (1 << 30)) return fail(COSM_ERR_INVALID_ARG, "too many replicas");

    // scratch layout and its size limit
    const size_t o_ij = 0;
    const size_t o_w = align256(o_ij + (size_t)g.m * 4);
    const size_t o_orig = align256(o_w + (size_t)g.m);
    const size_t o_alpha = align256(o_orig + (size_t)g.n * 4);
    const size_t o_segs = align256(o_alpha + (size_t)sweeps * sizeof(float2));
    const size_t o_segoff = align256(o_segs + (size_t)tiles * sizeof(Segment));
    const size_t o_err = align256(o_segoff + (size_t)(tiles + 1) * 4);
    const size_t o_off = align256(o_err + 4);
    const size_t total = align256(o_off + (size_t)(g.C + 1) * 4);
    if (total > kScratchBytes)
        return fail(COSM_ERR_TOO_LARGE,
                    "graph, step table and work list need " + std::to_string(total) +
                        " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
                        " (5 m + 4 n + 8 sweeps + 28 ceil(replicas / tile) + 4 (colours + 1) + 8 bytes, each of its eight"
                        " parts rounded up to 256 bytes)");
    unsigned char *base = nullptr;
    if ((rc = scratch_address(&base))) return rc;

    // host tables: colour-major records (src | dst << 16), weights, offsets
    std::vector<int64_t> count((size_t)g.C + 1, 0);
    for (int64_t e = 0; e < g.m; ++e) count[(size_t)g.color[(size_t)e] + 1]++;
    for (int c = 0; c < g.C; ++c) count[(size_t)c + 1] += count[(size_t)c];
    std::vector<int64_t> pos(count.begin(), count.end() - 1);
    std::vector<uint32_t> ij((size_t)g.m);
    std::vector<int8_t> wv((size_t)g.m);
    for (int64_t e = 0; e < g.m; ++e) {
        const int64_t k = pos[(size_t)g.color[(size_t)e]]++;
        ij[(size_t)k] = (uint32_t)g.src[(size_t)e] | ((uint32_t)g.dst[(size_t)e] << 16);
        wv[(size_t)k] = (int8_t)g.w[(size_t)e];
    }
    std::vector<int32_t> offc((size_t)g.C + 1);
    for (int c = 0; c <= g.C; ++c) offc[(size_t)c] = (int32_t)count[(size_t)c];
    const int64_t wbound = std::min(colour_weight_bound(offc.data(), g.C, wv.data(), nullptr, g.n),
                                    vertex_weight_bound(g.n, g.m, g.src.data(), g.dst.data(), g.w.data(), nullptr));
    std::vector<int32_t> orig((size_t)g.n);
    for (int32_t v = 0; v < g.n; ++v) orig[(size_t)v] = v;
    const double a0 = p->alpha0_deg / 360.0;
    std::vector<float2> tab((size_t)sweeps);
    for (int64_t s = 1; s <= sweeps; ++s) {
        const double a = (sweeps <= 1) ? a0 : a0 * (double)(sweeps - s) / (double)(sweeps - 1);
        tab[(size_t)(s - 1)] = make_float2((float)a, (float)(p->dwt_ratio * a));
    }
    std::vector<Segment> segs((size_t)tiles);
    std::vector<int32_t> segoff((size_t)tiles + 1);
    for (int64_t t = 0; t < tiles; ++t) {
        segs[(size_t)t] = Segment{(int32_t)t, SEG_INIT | SEG_READOUT, 1, sweeps};
        segoff[(size_t)t] = (int32_t)t;
    }
    segoff[(size_t)tiles] = (int32_t)tiles;

    // copies into the scratch, ordered after earlier work on the stream, so
    // calls on one stream never overlap (the host tables are staged before
    // each copy call returns)
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    struct Piece { size_t off; const void *src; size_t bytes; };
    const Piece pieces[] = {{o_ij, ij.data(), ij.size() * 4}, {o_w, wv.data(), wv.size()},
                            {o_orig, orig.data(), orig.size() * 4}, {o_alpha, tab.data(), tab.size() * sizeof(float2)},
                            {o_segs, segs.data(), segs.size() * sizeof(Segment)},
                            {o_segoff, segoff.data(), segoff.size() * 4}};
    std::vector<int32_t> offs((size_t)g.C + 1);
    for (int c = 0; c <= g.C; ++c) offs[(size_t)c] = (int32_t)count[(size_t)c];
    for (const Piece &pc : pieces) {
        cudaError_t e = cudaMemcpyAsync(base + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("copy to scratch: ") + cudaGetErrorString(e));
    }
    {
        cudaError_t e = cudaMemcpyAsync(base + o_off, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("copy to scratch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMemsetAsync(base + o_err, 0, 4, st);  // the error word starts at zero
    if (e != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

    KernelArgs a;
    std::memset(&a, 0, sizeof(a));
    InstView &v = a.v;
    v.n = g.n;
    v.C = g.C;
    v.off = reinterpret_cast<const int32_t *>(base + o_off);
    v.ij = reinterpret_cast<const uint32_t *>(base + o_ij);
    v.w = reinterpret_cast<const int8_t *>(base + o_w);
    v.orig_of = reinterpret_cast<const int32_t *>(base + o_orig);
    v.state = base;  // no segment loads or stores the state
    v.state_tile_stride = 0;
    v.alpha_tab = reinterpret_cast<const float2 *>(base + o_alpha);
    v.alpha_base = 1;
    v.S = sweeps;
    v.seed = seed;
    v.replicas = replicas;
    v.dwt_period = (p->flags & COSM_NO_DWT) ? 0 : p->dwt_period;
    v.wrap_p = wrap_period(p->alpha0_deg, p->dwt_ratio, p->dwt_period, p->flags, mode, p->storage, wbound);
    v.window = (float)(p->window_deg / 360.0);
    v.flags = p->flags;
    v.P = p->n_bisectors;
    v.mode = mode;
    v.K = K;
    v.cut = replica_cuts;
    v.bestp = best_p;
    a.segs = reinterpret_cast<const Segment *>(base + o_segs);
    a.seg_off = reinterpret_cast<const int32_t *>(base + o_segoff);
    a.ready = reinterpret_cast<int32_t *>(base + o_err);  // no segment waits or signals
    a.err = reinterpret_cast<int32_t *>(base + o_err);
    a.wait_limit_ns = 0;
    LaunchCfg cfg{mode, p->storage, K, threads, (int)tiles, smem, false};
    if (sweep_launch(cfg, a, st))
        return fail(COSM_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString(cudaGetLastError()));
    return COSM_OK;
}
