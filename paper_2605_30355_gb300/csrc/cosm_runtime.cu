// Host runtime behind the C ABI of include/cosm.h: handles, device layout,
// the work schedule of replica tiles over resident CTAs, and launches.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_internal.h"

using namespace cosm;

static thread_local std::string g_err;

static int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(COSM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

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

struct cosm_handle {
    Graph g;                        // host copy, original vertex ids
    cosm_params prm;
    int device = 0;
    int num_sms = 0;
    bool lattice = false;
    int64_t W = 0;                  // total weight
    std::vector<int32_t> slot_of;   // original id -> slot
    std::vector<int32_t> orig_of;   // slot -> original id
    int32_t off[kMaxColors + 1] = {0};
    int32_t C = 0;
    DevBuf<uint32_t> d_ij;
    DevBuf<int8_t> d_w;
    DevBuf<int32_t> d_orig;
    int mode = MODE_GENERAL_;       // kernel variant
    int32_t Q = 0, Wd = 0;          // 2D lattice geometry
    DevBuf<uint8_t> d_wnib;         // 2D lattice block weight bits
    // per run
    DevBuf<unsigned char> d_state;
    DevBuf<int64_t> d_cut;
    DevBuf<int32_t> d_bestp;
    DevBuf<float2> d_alpha;
    DevBuf<Segment> d_segs;
    DevBuf<int32_t> d_segoff;
    DevBuf<int32_t> d_ready;
    DevBuf<int32_t> d_err;
    DevBuf<int64_t> d_best;
    DevBuf<int8_t> d_spins;
    // cached host tables
    int64_t alpha_S = -1;
    double alpha_a0 = -1, alpha_ratio = -1;
    std::vector<Segment> h_segs;
    std::vector<int32_t> h_segoff;
    int64_t sched_tiles = -1, sched_S = -1, sched_G = -1;
    bool segs_uploaded = false;
    // state of the last launch
    int replicas = 0;
    int K = 0, threads = 0, occupancy = 0, grid = 0;
    size_t smem = 0;
    int64_t tile_stride = 0;  // storage elements per tile
    uint64_t seed = 0;
    bool have_state = false, have_result = false;
    cudaStream_t stream = nullptr;
    int launches = 0;
};

extern "C" const char *cosm_last_error(void) { return g_err.c_str(); }

void cosm::set_last_error(const std::string &msg) { g_err = msg; }

extern "C" void cosm_default_params(cosm_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->alpha0_deg = 14.0;
    p->dwt_ratio = 0.5;
    p->dwt_period = 3;
    p->window_deg = 90.0;
    p->n_bisectors = 100;
    p->storage = COSM_F32;
    p->flags = 0;
}

static int check_params(const cosm_params *p)
{
    if (!p) return fail(COSM_ERR_INVALID_ARG, "params is NULL");
    if (!(p->alpha0_deg >= 0.0 && p->alpha0_deg < 180.0))
        return fail(COSM_ERR_INVALID_ARG, "alpha0_deg must be in [0, 180)");
    if (!(p->dwt_ratio >= 0.0 && p->dwt_ratio <= 16.0))
        return fail(COSM_ERR_INVALID_ARG, "dwt_ratio must be in [0, 16]");
    if (p->dwt_period < 0) return fail(COSM_ERR_INVALID_ARG, "dwt_period must be >= 0");
    if (!(p->window_deg > 0.0 && p->window_deg <= 180.0))
        return fail(COSM_ERR_INVALID_ARG, "window_deg must be in (0, 180]");
    if (p->n_bisectors < 1 || p->n_bisectors > kMaxBisectors)
        return fail(COSM_ERR_INVALID_ARG, "n_bisectors must be in [1, 256]");
    if (p->storage != COSM_F32 && p->storage != COSM_F16)
        return fail(COSM_ERR_INVALID_ARG, "storage must be COSM_F32 or COSM_F16");
    if (p->flags & ~(COSM_NO_DWT | COSM_NO_SCS)) return fail(COSM_ERR_INVALID_ARG, "unknown flags");
    return COSM_OK;
}

extern "C" int cosm_validate_partition(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                       int32_t n_colors, const int32_t *color)
{
    if (!src || !dst || !color || n < 1 || m < 0) return fail(COSM_ERR_INVALID_ARG, "bad arguments");
    std::string why;
    int rc = validate_partition(n, m, src, dst, n_colors, color, why);
    if (rc) return fail(rc, why);
    return COSM_OK;
}

extern "C" int cosm_color_greedy(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 int32_t *color, int32_t *n_colors)
{
    if (!src || !dst || !color || !n_colors || n < 1 || m < 0)
        return fail(COSM_ERR_INVALID_ARG, "bad arguments");
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || src[e] == dst[e])
            return fail(COSM_ERR_INVALID_ARG, "edge endpoint out of range or loop");
    return color_greedy(n, m, src, dst, color, n_colors);
}

extern "C" int cosm_color_misra_gries(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                      int32_t *color, int32_t *n_colors)
{
    if (!src || !dst || !color || !n_colors || n < 1 || m < 0)
        return fail(COSM_ERR_INVALID_ARG, "bad arguments");
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || src[e] == dst[e])
            return fail(COSM_ERR_INVALID_ARG, "edge endpoint out of range or loop");
    int rc = color_misra_gries(n, m, src, dst, color, n_colors);
    if (rc) return fail(rc, "Misra-Gries colouring failed (multigraph?)");
    return COSM_OK;
}

extern "C" int cosm_color_torus2d(int32_t L1, int32_t L2, int64_t m, const int32_t *src,
                                  const int32_t *dst, int32_t *color)
{
    if (!src || !dst || !color) return fail(COSM_ERR_INVALID_ARG, "bad arguments");
    int rc = color_torus2d(L1, L2, m, src, dst, color);
    if (rc) return fail(rc, "not an even-sided 2D torus edge list");
    return COSM_OK;
}

extern "C" int cosm_color_torus3d(int32_t L1, int32_t L2, int32_t L3, int64_t m, const int32_t *src,
                                  const int32_t *dst, int32_t *color)
{
    if (!src || !dst || !color) return fail(COSM_ERR_INVALID_ARG, "bad arguments");
    int rc = color_torus3d(L1, L2, L3, m, src, dst, color);
    if (rc) return fail(rc, "not an even-sided 3D torus edge list");
    return COSM_OK;
}

// ------------------------------------------------------------------ create

extern "C" void cosm_destroy(cosm_handle *h)
{
    if (!h) return;
    if (h->stream || h->have_state) cudaStreamSynchronize(h->stream);
    h->d_ij.release(); h->d_w.release(); h->d_orig.release(); h->d_state.release();
    h->d_cut.release(); h->d_bestp.release(); h->d_alpha.release(); h->d_segs.release();
    h->d_segoff.release(); h->d_ready.release(); h->d_err.release(); h->d_best.release();
    h->d_spins.release();
    h->d_wnib.release();
    delete h;
}

// The implicit-index 2D lattice kernel applies when the graph is an
// even-sided torus given with the regular 4-colour pattern, all weights are
// +-1 and the update is the sequential one. It walks 2x2 blocks in two
// passes; this builds each block's four weight bits from the edge list, in
// the kernel's edge order (even pass: A-B, C-D, A-C, B-D; odd pass: D-C,
// B-A, D-B, C-A over the shifted block).
static int setup_lattice2d(cosm_handle *h)
{
    const Graph &g = h->g;
    h->mode = (h->prm.flags & COSM_NO_SCS) ? MODE_ACCUM_ : MODE_GENERAL_;
    if (std::getenv("COSM_NO_LATTICE")) return COSM_OK;
    if (!h->lattice || g.dims[2] != 0 || h->mode != MODE_GENERAL_ || h->C != 4) return COSM_OK;
    for (int64_t e = 0; e < g.m; ++e)
        if (g.w[(size_t)e] != 1 && g.w[(size_t)e] != -1) return COSM_OK;
    std::vector<int32_t> pat((size_t)g.m);
    if (color_torus2d(g.dims[0], g.dims[1], g.m, g.src.data(), g.dst.data(), pat.data()) != 0)
        return COSM_OK;
    if (pat != g.color) return COSM_OK;  // another colour order changes the dynamics
    const int32_t Q = g.n / 4, Wd = g.dims[1] / 2;
    std::unordered_map<int64_t, int32_t> wmap;
    wmap.reserve((size_t)g.m * 2);
    for (int64_t e = 0; e < g.m; ++e)
        wmap[(int64_t)g.src[(size_t)e] * g.n + g.dst[(size_t)e]] = g.w[(size_t)e];
    auto weight = [&](int32_t slot_a, int32_t slot_b) {
        const int32_t a = h->orig_of[(size_t)slot_a], b = h->orig_of[(size_t)slot_b];
        auto it = wmap.find((int64_t)std::min(a, b) * g.n + std::max(a, b));
        return it == wmap.end() ? 0 : it->second;
    };
    std::vector<uint8_t> nib((size_t)2 * Q, 0);
    for (int32_t f = 0; f < Q; ++f) {
        const int32_t A = f, B = Q + f, Cc = 2 * Q + f, D = 3 * Q + f;
        const int32_t even[4][2] = {{A, B}, {Cc, D}, {A, Cc}, {B, D}};
        const int32_t gcol = (f % Wd == Wd - 1) ? f + 1 - Wd : f + 1;
        const int32_t hrow = (f + Wd) % Q, gh = (gcol + Wd) % Q;
        const int32_t odd[4][2] = {{D, 2 * Q + gcol}, {Q + hrow, gh}, {D, Q + hrow}, {2 * Q + gcol, gh}};
        for (int k = 0; k < 4; ++k) {
            const int32_t we = weight(even[k][0], even[k][1]), wo = weight(odd[k][0], odd[k][1]);
            if (we == 0 || wo == 0) return fail(COSM_ERR_INVALID_ARG, "lattice block edge missing");
            if (we == -1) nib[(size_t)f] |= (uint8_t)(1u << k);
            if (wo == -1) nib[(size_t)Q + f] |= (uint8_t)(1u << k);
        }
    }
    int rc = h->d_wnib.ensure(nib.size());
    if (rc) return rc;
    CK(cudaMemcpy(h->d_wnib.p, nib.data(), nib.size(), cudaMemcpyHostToDevice));
    h->Q = Q;
    h->Wd = Wd;
    h->mode = MODE_LATTICE2D_;
    return COSM_OK;
}

extern "C" int cosm_create(const cosm_graph_desc *gd, const cosm_params *p, cosm_handle **out)
{
    if (!gd || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if (!gd->src || !gd->dst || !gd->w) return fail(COSM_ERR_INVALID_ARG, "NULL edge arrays");
    if (gd->n < 2 || gd->n > kMaxVertices) return fail(COSM_ERR_INVALID_ARG, "n must be in [2, 65536]");
    if (gd->m < 1 || gd->m > ((int64_t)1 << 26)) return fail(COSM_ERR_INVALID_ARG, "m must be in [1, 2^26]");
    cosm_handle *h = new (std::nothrow) cosm_handle();
    if (!h) return fail(COSM_ERR_NOMEM, "host allocation failed");
    h->prm = *p;
    Graph &g = h->g;
    g.n = gd->n;
    g.m = gd->m;
    g.src.assign(gd->src, gd->src + gd->m);
    g.dst.assign(gd->dst, gd->dst + gd->m);
    g.w.assign(gd->w, gd->w + gd->m);
    for (int k = 0; k < 3; ++k) g.dims[k] = gd->dims[k];
    std::string why;
    rc = validate_graph(g, why);
    if (rc) { delete h; return fail(rc, why); }
    // partition: given, or coloured here (lattice pattern, else greedy)
    g.color.assign((size_t)g.m, 0);
    if (gd->color) {
        g.color.assign(gd->color, gd->color + gd->m);
        g.C = gd->n_colors;
    } else if (g.dims[0] > 0 && g.dims[2] == 0 &&
               color_torus2d(g.dims[0], g.dims[1], g.m, g.src.data(), g.dst.data(), g.color.data()) == 0) {
        g.C = 4;
    } else if (g.dims[0] > 0 && g.dims[2] > 0 &&
               color_torus3d(g.dims[0], g.dims[1], g.dims[2], g.m, g.src.data(), g.dst.data(),
                             g.color.data()) == 0) {
        g.C = 6;
    } else {
        color_greedy(g.n, g.m, g.src.data(), g.dst.data(), g.color.data(), &g.C);
    }
    rc = validate_partition(g.n, g.m, g.src.data(), g.dst.data(), g.C, g.color.data(), why);
    if (rc) { delete h; return fail(rc, why); }
    h->C = g.C;
    // shared-memory layout: lattice sublattices when the hint matches
    h->slot_of.resize((size_t)g.n);
    if (g.dims[0] > 0) {
        if (!lattice_relabel(g, h->slot_of, why)) { delete h; return fail(COSM_ERR_INVALID_ARG, why); }
        h->lattice = true;
    } else {
        for (int32_t v = 0; v < g.n; ++v) h->slot_of[(size_t)v] = v;
    }
    h->orig_of.assign((size_t)g.n, 0);
    for (int32_t v = 0; v < g.n; ++v) h->orig_of[(size_t)h->slot_of[(size_t)v]] = v;
    // colour-major edge records, each colour sorted by the slot of src
    std::vector<int64_t> order((size_t)g.m);
    for (int64_t e = 0; e < g.m; ++e) order[(size_t)e] = e;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        if (g.color[(size_t)a] != g.color[(size_t)b]) return g.color[(size_t)a] < g.color[(size_t)b];
        return h->slot_of[(size_t)g.src[(size_t)a]] < h->slot_of[(size_t)g.src[(size_t)b]];
    });
    std::vector<uint32_t> ij((size_t)g.m);
    std::vector<int8_t> wv((size_t)g.m);
    std::memset(h->off, 0, sizeof(h->off));
    for (int64_t k = 0; k < g.m; ++k) {
        const int64_t e = order[(size_t)k];
        ij[(size_t)k] = (uint32_t)h->slot_of[(size_t)g.src[(size_t)e]] |
                        ((uint32_t)h->slot_of[(size_t)g.dst[(size_t)e]] << 16);
        wv[(size_t)k] = (int8_t)g.w[(size_t)e];
        h->off[g.color[(size_t)e] + 1]++;
        h->W += g.w[(size_t)e];
    }
    for (int c = 0; c < h->C; ++c) h->off[c + 1] += h->off[c];
    // device copies
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if ((rc = h->d_ij.ensure((size_t)g.m)) || (rc = h->d_w.ensure((size_t)g.m)) ||
        (rc = h->d_orig.ensure((size_t)g.n)) || (rc = h->d_err.ensure(1)) ||
        (rc = h->d_best.ensure(4)) || (rc = h->d_spins.ensure((size_t)g.n))) {
        cosm_destroy(h);
        return rc;
    }
    if (cudaMemcpy(h->d_ij.p, ij.data(), ij.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_w.p, wv.data(), wv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_orig.p, h->orig_of.data(), (size_t)g.n * 4, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cosm_destroy(h);
        return fail(COSM_ERR_CUDA, "copying the graph to the device failed");
    }
    if ((rc = setup_lattice2d(h))) {
        cosm_destroy(h);
        return rc;
    }
    *out = h;
    return COSM_OK;
}

// ------------------------------------------------------------------ layout

static int env_int(const char *name, int dflt)
{
    const char *s = std::getenv(name);
    return (s && *s) ? std::atoi(s) : dflt;
}

// Replicas per CTA (K) and threads per CTA: maximise resident replicas per
// SM (COSM_K / COSM_THREADS override for experiments).
static int choose_layout(cosm_handle *h, int replicas)
{
    const cosm_params &p = h->prm;
    const int mode = h->mode;
    const int P = p.n_bisectors;
    int max_ec = 0;
    for (int c = 0; c < h->C; ++c) max_ec = std::max(max_ec, h->off[c + 1] - h->off[c]);
    const int Ks_f32[3] = {1, 2, 4}, Ks_f16[3] = {2, 4, 8};
    const int *Ks = p.storage == COSM_F32 ? Ks_f32 : Ks_f16;
    int forceK = env_int("COSM_K", 0), forceT = env_int("COSM_THREADS", 0);
    int bestK = 0, bestT = 0, bestOcc = 0;
    long bestScore = -1;
    for (int k = 0; k < 3; ++k) {
        const int K = Ks[k];
        if (forceK && K != forceK) continue;
        const size_t smem = sweep_smem_bytes(p.storage, K, h->g.n, P, mode);
        if (smem > 227 * 1024) continue;
        int T = forceT ? forceT : std::min(1024, std::max(64, ((max_ec + 1) / 2 + 31) / 32 * 32));
        if (!forceT && T > 512) T = 512;
        if (mode == MODE_LATTICE2D_ && !forceT) T = std::min(512, std::max(64, (h->Q + 31) / 32 * 32));
        int occ = sweep_occupancy(p.storage, K, mode, T, smem);
        while (occ == 0 && T > 64 && !forceT) {
            T /= 2;
            occ = sweep_occupancy(p.storage, K, mode, T, smem);
        }
        if (occ == 0) continue;
        const long tiles = (replicas + K - 1) / K;
        // resident replicas per SM, capped by what the run can fill; on a tie
        // a larger tile amortises per-edge work when the run fills every CTA
        // slot, a smaller one spreads a small run over more SMs
        const long resident = std::min<long>((long)occ * K, std::max<long>(1, tiles * K / h->num_sms));
        const bool full = tiles >= (long)occ * h->num_sms;
        const long score = resident * 1000 + (full ? K : -K);
        if (score > bestScore) {
            bestScore = score;
            bestK = K;
            bestT = T;
            bestOcc = occ;
        }
    }
    if (!bestK) return fail(COSM_ERR_TOO_LARGE, "no replica tile fits in shared memory");
    h->K = bestK;
    h->threads = bestT;
    h->occupancy = bestOcc;
    h->smem = sweep_smem_bytes(p.storage, bestK, h->g.n, P, mode);
    const size_t esz = p.storage == COSM_F32 ? 4 : 2;
    h->tile_stride = (int64_t)(((size_t)h->g.n * bestK * esz + 15) / 16 * 16 / esz);
    return COSM_OK;
}

static int ensure_run_buffers(cosm_handle *h, int replicas)
{
    const size_t esz = h->prm.storage == COSM_F32 ? 4 : 2;
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    int rc;
    if ((rc = h->d_state.ensure((size_t)tiles * (size_t)h->tile_stride * esz)) ||
        (rc = h->d_cut.ensure((size_t)replicas)) || (rc = h->d_bestp.ensure((size_t)replicas)) ||
        (rc = h->d_ready.ensure((size_t)tiles)))
        return rc;
    return COSM_OK;
}

static KernelArgs base_args(cosm_handle *h)
{
    KernelArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = h->g.n;
    a.C = h->C;
    std::memcpy(a.off, h->off, sizeof(a.off));
    a.ij = h->d_ij.p;
    a.w = h->d_w.p;
    a.orig_of = h->d_orig.p;
    a.state = h->d_state.p;
    a.state_tile_stride = h->tile_stride;
    a.seed = h->seed;
    a.replicas = h->replicas;
    a.dwt_period = (h->prm.flags & COSM_NO_DWT) ? 0 : h->prm.dwt_period;
    a.window = (float)(h->prm.window_deg / 360.0);
    a.flags = h->prm.flags;
    a.P = h->prm.n_bisectors;
    a.ready = h->d_ready.p;
    a.err = h->d_err.p;
    a.wait_limit_ns = (uint64_t)env_int("COSM_WAIT_LIMIT_S", 20) * 1000000000ull;
    a.cut = h->d_cut.p;
    a.bestp = h->d_bestp.p;
    a.wnib = h->d_wnib.p;
    a.Q = h->Q;
    a.Wd = h->Wd;
    return a;
}

static int upload_segments(cosm_handle *h, cudaStream_t st)
{
    if (h->segs_uploaded) return COSM_OK;
    int rc;
    if ((rc = h->d_segs.ensure(h->h_segs.size())) || (rc = h->d_segoff.ensure(h->h_segoff.size())))
        return rc;
    CK(cudaMemcpyAsync(h->d_segs.p, h->h_segs.data(), h->h_segs.size() * sizeof(Segment),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->d_segoff.p, h->h_segoff.data(), h->h_segoff.size() * 4,
                       cudaMemcpyHostToDevice, st));
    h->segs_uploaded = true;
    return COSM_OK;
}

// Work schedule for `tiles` tiles of S sweeps each on at most G resident
// CTAs. With tiles <= G every CTA runs one whole trial. Otherwise the
// wrap-around rule of McNaughton (1959) gives every CTA an equal share of
// tiles * S sweeps: a tile split between CTA b and b+1 runs its head first
// on b and its tail last on b+1 (the share exceeds S, so the two never
// overlap), and b+1 waits for the head's published state before the tail.
static void build_schedule(cosm_handle *h, int64_t tiles, int64_t S, int64_t G)
{
    if (h->sched_tiles == tiles && h->sched_S == S && h->sched_G == G) return;
    h->h_segs.clear();
    h->h_segoff.assign(1, 0);
    h->segs_uploaded = false;
    if (tiles <= G) {
        for (int64_t t = 0; t < tiles; ++t) {
            h->h_segs.push_back(Segment{(int32_t)t, SEG_INIT | SEG_READOUT | SEG_STORE, 1, S});
            h->h_segoff.push_back((int32_t)h->h_segs.size());
        }
    } else {
        const __int128 L = (__int128)tiles * S;
        for (int64_t b = 0; b < G; ++b) {
            const int64_t lo = (int64_t)(L * b / G), hi = (int64_t)(L * (b + 1) / G);
            std::vector<Segment> pieces;
            for (int64_t j = lo / S; j <= (hi - 1) / S && j < tiles; ++j) {
                const int64_t a0 = std::max<int64_t>(lo, j * S) - j * S;
                const int64_t z = std::min<int64_t>(hi, (j + 1) * S) - j * S;
                if (z <= a0) continue;
                Segment sg{(int32_t)j, 0, a0 + 1, z};
                sg.flags = (a0 == 0) ? SEG_INIT : (SEG_LOAD | SEG_WAIT);
                sg.flags |= (z == S) ? (SEG_READOUT | SEG_STORE) : (SEG_STORE | SEG_SIGNAL);
                pieces.push_back(sg);
            }
            // execution order: head of the tile continuing on b+1 first, the
            // tail of the tile started on b-1 last
            std::vector<Segment> ordered;
            if (!pieces.empty() && pieces.back().s_begin == 1 && pieces.back().s_end < S) {
                ordered.push_back(pieces.back());
                pieces.pop_back();
            }
            Segment tail{};
            bool has_tail = false;
            if (!pieces.empty() && pieces.front().s_begin > 1) {
                tail = pieces.front();
                has_tail = true;
                pieces.erase(pieces.begin());
            }
            for (auto &sg : pieces) ordered.push_back(sg);
            if (has_tail) ordered.push_back(tail);
            for (auto &sg : ordered) h->h_segs.push_back(sg);
            h->h_segoff.push_back((int32_t)h->h_segs.size());
        }
    }
    h->sched_tiles = tiles;
    h->sched_S = S;
    h->sched_G = G;
}

static int upload_alpha(cosm_handle *h, int64_t S, cudaStream_t st)
{
    const double a0 = h->prm.alpha0_deg / 360.0, ratio = h->prm.dwt_ratio;
    if (h->alpha_S == S && h->alpha_a0 == a0 && h->alpha_ratio == ratio) return COSM_OK;
    std::vector<float2> tab((size_t)S);
    for (int64_t s = 1; s <= S; ++s) {
        // linear ramp alpha_0 -> 0 (Table IX), FP64 rounded once to FP32
        const double a = (S <= 1) ? a0 : a0 * (double)(S - s) / (double)(S - 1);
        tab[(size_t)(s - 1)] = make_float2((float)a, (float)(ratio * a));
    }
    int rc = h->d_alpha.ensure((size_t)S);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_alpha.p, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // the host table is released here
    h->alpha_S = S;
    h->alpha_a0 = a0;
    h->alpha_ratio = ratio;
    return COSM_OK;
}

static int launch_finalize(cosm_handle *h, cudaStream_t st)
{
    FinalArgs f;
    f.n = h->g.n;
    f.replicas = h->replicas;
    f.K = h->K;
    f.storage = h->prm.storage;
    f.P = h->prm.n_bisectors;
    f.W = h->W;
    f.state = h->d_state.p;
    f.state_tile_stride = h->tile_stride;
    f.orig_of = h->d_orig.p;
    f.cut = h->d_cut.p;
    f.bestp = h->d_bestp.p;
    f.best = h->d_best.p;
    f.spins = h->d_spins.p;
    if (finalize_launch(f, st)) return fail(COSM_ERR_CUDA, std::string("finalize launch: ") +
                                                          cudaGetErrorString(cudaGetLastError()));
    return COSM_OK;
}

extern "C" int cosm_run(cosm_handle *h, int64_t sweeps, int32_t replicas, uint64_t seed, void *stream)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (sweeps < 1 || sweeps >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "sweeps must be in [1, 2^31)");
    if (replicas < 1 || replicas >= (1 << 24)) return fail(COSM_ERR_INVALID_ARG, "replicas must be in [1, 2^24)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc;
    if (!h->K || replicas != h->replicas) {
        if ((rc = choose_layout(h, replicas))) return rc;
    }
    h->replicas = replicas;
    h->seed = seed;
    if ((rc = ensure_run_buffers(h, replicas))) return rc;
    if ((rc = upload_alpha(h, sweeps, st))) return rc;
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    int64_t cap = (int64_t)h->occupancy * h->num_sms;
    const int cap_env = env_int("COSM_GRID_CAP", 0);  // test hook: fewer resident CTAs
    if (cap_env > 0) cap = std::min<int64_t>(cap, cap_env);
    build_schedule(h, tiles, sweeps, cap);
    if ((rc = upload_segments(h, st))) return rc;
    const bool waits = tiles > cap;
    if (waits) CK(cudaMemsetAsync(h->d_ready.p, 0, (size_t)tiles * 4, st));
    CK(cudaMemsetAsync(h->d_err.p, 0, 4, st));
    KernelArgs a = base_args(h);
    a.alpha_tab = h->d_alpha.p;
    a.alpha_base = 1;
    a.S = sweeps;
    a.segs = h->d_segs.p;
    a.seg_off = h->d_segoff.p;
    LaunchCfg cfg{h->mode, h->prm.storage, h->K, h->threads, (int)(h->h_segoff.size() - 1), h->smem, waits};
    h->grid = cfg.grid;
    if (sweep_launch(cfg, a, st))
        return fail(COSM_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString(cudaGetLastError()));
    if ((rc = launch_finalize(h, st))) return rc;
    h->stream = st;
    h->have_state = true;
    h->have_result = true;
    h->launches = 2;
    return COSM_OK;
}

extern "C" int cosm_sync(cosm_handle *h)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    int err = 0;
    CK(cudaMemcpy(&err, h->d_err.p, 4, cudaMemcpyDeviceToHost));
    if (err) return fail(COSM_ERR_TIMEOUT, "a bounded wait between work segments gave up");
    return COSM_OK;
}

extern "C" int cosm_get_best(cosm_handle *h, int64_t *cut, int64_t *energy, int32_t *replica, int8_t *spins)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_result) return fail(COSM_ERR_STATE, "no run or readout yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    int64_t best[3];
    CK(cudaMemcpy(best, h->d_best.p, sizeof(best), cudaMemcpyDeviceToHost));
    if (cut) *cut = best[0];
    if (energy) *energy = best[1];
    if (replica) *replica = (int32_t)best[2];
    if (spins) CK(cudaMemcpy(spins, h->d_spins.p, (size_t)h->g.n, cudaMemcpyDefault));
    return COSM_OK;
}

extern "C" int cosm_get_replica_cuts(cosm_handle *h, int64_t *cuts, int32_t *best_p)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_result) return fail(COSM_ERR_STATE, "no run or readout yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    if (cuts) CK(cudaMemcpy(cuts, h->d_cut.p, (size_t)h->replicas * 8, cudaMemcpyDefault));
    if (best_p) CK(cudaMemcpy(best_p, h->d_bestp.p, (size_t)h->replicas * 4, cudaMemcpyDefault));
    return COSM_OK;
}

// Stored value (FP32 or FP16, representative in [-1/2, 1/2]) -> turn in [0, 1).
static inline double to_turn(double g)
{
    double x = g < 0.0 ? g + 1.0 : g;
    return x >= 1.0 ? 0.0 : x;
}

extern "C" int cosm_get_state(cosm_handle *h, double *phases)
{
    if (!h || !phases) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    const int64_t tiles = (h->replicas + h->K - 1) / h->K;
    const size_t esz = h->prm.storage == COSM_F32 ? 4 : 2;
    std::vector<unsigned char> raw((size_t)tiles * (size_t)h->tile_stride * esz);
    CK(cudaMemcpy(raw.data(), h->d_state.p, raw.size(), cudaMemcpyDeviceToHost));
    std::vector<double> out((size_t)h->replicas * h->g.n);
    for (int32_t r = 0; r < h->replicas; ++r) {
        const size_t base = (size_t)(r / h->K) * (size_t)h->tile_stride;
        for (int32_t v = 0; v < h->g.n; ++v) {
            const size_t idx = base + (size_t)h->slot_of[(size_t)v] * h->K + (size_t)(r % h->K);
            double g;
            if (esz == 4) {
                float f;
                std::memcpy(&f, raw.data() + idx * 4, 4);
                g = f;
            } else {
                __half hv;
                std::memcpy(&hv, raw.data() + idx * 2, 2);
                g = (double)__half2float(hv);
            }
            out[(size_t)r * h->g.n + v] = to_turn(g);
        }
    }
    CK(cudaMemcpy(phases, out.data(), out.size() * 8, cudaMemcpyDefault));
    return COSM_OK;
}

extern "C" int cosm_set_state(cosm_handle *h, const double *phases, int32_t replicas, uint64_t seed)
{
    if (!h || !phases) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (replicas < 1 || replicas >= (1 << 24)) return fail(COSM_ERR_INVALID_ARG, "bad replica count");
    int rc;
    if (h->stream) CK(cudaStreamSynchronize(h->stream));
    if (!h->K || replicas != h->replicas) {
        if ((rc = choose_layout(h, replicas))) return rc;
    }
    h->replicas = replicas;
    h->seed = seed;
    if ((rc = ensure_run_buffers(h, replicas))) return rc;
    std::vector<double> in((size_t)replicas * h->g.n);
    CK(cudaMemcpy(in.data(), phases, in.size() * 8, cudaMemcpyDefault));
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    const size_t esz = h->prm.storage == COSM_F32 ? 4 : 2;
    std::vector<unsigned char> raw((size_t)tiles * (size_t)h->tile_stride * esz, 0);
    for (int32_t r = 0; r < replicas; ++r) {
        const size_t base = (size_t)(r / h->K) * (size_t)h->tile_stride;
        for (int32_t v = 0; v < h->g.n; ++v) {
            double x = in[(size_t)r * h->g.n + v];
            if (!(x >= 0.0 && x < 1.0)) return fail(COSM_ERR_INVALID_ARG, "phases must be in [0, 1)");
            const double g = x >= 0.5 ? x - 1.0 : x;
            const size_t idx = base + (size_t)h->slot_of[(size_t)v] * h->K + (size_t)(r % h->K);
            if (esz == 4) {
                const float f = (float)g;
                std::memcpy(raw.data() + idx * 4, &f, 4);
            } else {
                const __half hv = __float2half_rn((float)g);
                std::memcpy(raw.data() + idx * 2, &hv, 2);
            }
        }
    }
    CK(cudaMemcpy(h->d_state.p, raw.data(), raw.size(), cudaMemcpyHostToDevice));
    h->have_state = true;
    h->have_result = false;
    return COSM_OK;
}

// One launch over all tiles of the current state with per-tile segments of
// the given flags and sweep range.
static int launch_on_state(cosm_handle *h, int32_t flags, int64_t s0, int64_t s1, const float2 *tab,
                           int64_t base, cudaStream_t st)
{
    const int64_t tiles = (h->replicas + h->K - 1) / h->K;
    h->h_segs.clear();
    h->h_segoff.assign(1, 0);
    for (int64_t t = 0; t < tiles; ++t) {
        h->h_segs.push_back(Segment{(int32_t)t, flags, s0, s1});
        h->h_segoff.push_back((int32_t)h->h_segs.size());
    }
    h->sched_tiles = -1;  // invalidate the cached run schedule
    h->segs_uploaded = false;
    int rc = upload_segments(h, st);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->d_err.p, 0, 4, st));
    KernelArgs a = base_args(h);
    a.alpha_tab = tab;
    a.alpha_base = base;
    a.S = s1;
    a.segs = h->d_segs.p;
    a.seg_off = h->d_segoff.p;
    LaunchCfg cfg{h->mode, h->prm.storage, h->K, h->threads, (int)tiles, h->smem, false};
    h->grid = cfg.grid;
    if (sweep_launch(cfg, a, st))
        return fail(COSM_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString(cudaGetLastError()));
    h->stream = st;
    return COSM_OK;
}

extern "C" int cosm_step(cosm_handle *h, int64_t sweep, float alpha, void *stream)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    if (sweep < 1 || sweep >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "bad sweep index");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc;
    DevBuf<float2> tab;  // one-entry step table for this sweep
    if ((rc = tab.ensure(1))) return rc;
    const float2 v = make_float2(alpha, (float)(h->prm.dwt_ratio * (double)alpha));
    if (h->stream) CK(cudaStreamSynchronize(h->stream));
    if (cudaMemcpy(tab.p, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess) {
        tab.release();
        return fail(COSM_ERR_CUDA, "alpha upload failed");
    }
    rc = launch_on_state(h, SEG_LOAD | SEG_STORE, sweep, sweep, tab.p, sweep, st);
    if (!rc) rc = cudaStreamSynchronize(st) == cudaSuccess ? COSM_OK : fail(COSM_ERR_CUDA, "step failed");
    tab.release();
    h->have_result = false;
    h->launches = 1;
    return rc;
}

extern "C" int cosm_readout(cosm_handle *h, void *stream)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = launch_on_state(h, SEG_LOAD | SEG_READOUT, 1, 0, h->d_alpha.p, 1, st);
    if (rc) return rc;
    if ((rc = launch_finalize(h, st))) return rc;
    h->have_result = true;
    h->launches = 2;
    return COSM_OK;
}

extern "C" int cosm_layout(cosm_handle *h, int32_t out[8])
{
    if (!h || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    out[0] = h->K;
    out[1] = h->threads;
    out[2] = (int32_t)h->smem;
    out[3] = h->occupancy;
    out[4] = h->mode == MODE_LATTICE2D_ ? 2 : (h->lattice ? 1 : 0);
    out[5] = h->grid;
    out[6] = h->launches;
    out[7] = h->C;
    return COSM_OK;
}

extern "C" int cosm_solve(const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps, int32_t replicas,
                          uint64_t seed, int64_t *best_cut, int64_t *energy, int8_t *spins,
                          int64_t *replica_cuts)
{
    cosm_handle *h = nullptr;
    int rc = cosm_create(g, p, &h);
    if (rc) return rc;
    rc = cosm_run(h, sweeps, replicas, seed, nullptr);
    if (!rc) rc = cosm_get_best(h, best_cut, energy, nullptr, spins);
    if (!rc && replica_cuts) rc = cosm_get_replica_cuts(h, replica_cuts, nullptr);
    cosm_destroy(h);
    return rc;
}
