// Host runtime behind the C ABI of include/cosm.h: handles, device layout,
// the work schedule of replica tiles over resident CTAs, and launches.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_handle.h"
#include "cosm_internal.h"

using namespace cosm;

static thread_local std::string g_err;

int cosm::fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

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
    if (p->storage != COSM_F32 && p->storage != COSM_F16 && p->storage != COSM_Q16 && p->storage != COSM_BF16)
        return fail(COSM_ERR_INVALID_ARG, "storage must be COSM_F32, COSM_F16, COSM_Q16 or COSM_BF16");
    if (p->flags & ~(COSM_NO_DWT | COSM_NO_SCS | COSM_DWT_RANDOM_DIR | COSM_OPT_BISECTOR))
        return fail(COSM_ERR_INVALID_ARG, "unknown flags");
    if (p->track_period < 0) return fail(COSM_ERR_INVALID_ARG, "track_period must be >= 0");
    return COSM_OK;
}

// Features of single-instance runs only (local fields, tracking, optimal
// bisector): the batch and serving paths reject them up front.
int cosm::single_only(const cosm_graph_desc *g, const cosm_params *p)
{
    if (g && g->h) return fail(COSM_ERR_INVALID_ARG, "local fields are supported by single instances only");
    if (p && p->track_period > 0)
        return fail(COSM_ERR_INVALID_ARG, "mid-anneal tracking is supported by single instances only");
    if (p && (p->flags & COSM_OPT_BISECTOR))
        return fail(COSM_ERR_INVALID_ARG, "the optimal bisector is supported by single instances only");
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
    h->d_ij.release(); h->d_w.release(); h->d_ijs.release(); h->d_orig.release(); h->d_off.release(); h->d_state.release();
    h->d_cut.release(); h->d_bestp.release(); h->d_alpha.release(); h->d_segs.release();
    h->d_segoff.release(); h->d_ready.release(); h->d_err.release(); h->d_best.release();
    h->d_spins.release();
    h->d_wnib.release();
    h->d_h.release(); h->d_energy.release(); h->d_bisB.release(); h->d_trace.release();
    h->d_bits.release(); h->d_qbuf.release(); h->d_delta.release(); h->d_items.release();
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
    if (std::getenv("COSM_NO_LATTICE") || h->fields) return COSM_OK;
    // the full torus only (every block needs its four edges)
    if (!h->lattice || g.dims[2] != 0 || h->mode != MODE_GENERAL_ || h->C != 4 || g.m != 2 * (int64_t)g.n)
        return COSM_OK;
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

// Order of one colour class's edges for the edge-list kernel. A warp takes
// 32 consecutive edges; with two binary32 replicas per slot (8 bytes) a
// half-warp's 16 loads of source phases, and its 16 loads of destination
// phases, are each conflict-free in shared memory when their slots are
// distinct modulo 16. Edges are grouped accordingly: the class is read as a
// bipartite multigraph between source residues and destination residues
// (slot mod 16), properly edge-coloured with its maximum degree of colours
// by Konig's alternating-path method, and each colour class (at most one
// edge per residue on either side) becomes a run of consecutive edges,
// largest first, in source-residue order. Edges of one colour share no
// vertex, so their order changes no result; it only changes which phases a
// half-warp touches together.
static void balance_banks(int64_t *e, int64_t cnt, const std::vector<int32_t> &ss,
                          const std::vector<int32_t> &ds)
{
    constexpr int R = 16;
    if (cnt < 32 || cnt > ((int64_t)1 << 20)) return;
    std::vector<int32_t> A((size_t)cnt), B((size_t)cnt);
    int deg[2 * R] = {0};
    for (int64_t k = 0; k < cnt; ++k) {
        A[(size_t)k] = ss[(size_t)e[k]] & (R - 1);
        B[(size_t)k] = R + (ds[(size_t)e[k]] & (R - 1));
        ++deg[A[(size_t)k]];
        ++deg[B[(size_t)k]];
    }
    int D = 0;
    for (int v = 0; v < 2 * R; ++v) D = std::max(D, deg[v]);
    const int Wd = (D + 63) / 64;
    std::vector<int32_t> at((size_t)2 * R * D, -1);  // at[v D + c]: edge of colour c at residue v
    std::vector<uint64_t> freeb((size_t)2 * R * Wd, ~0ull);
    std::vector<int32_t> color((size_t)cnt, -1);
    auto mark = [&](int v, int c, bool used) {
        uint64_t &w = freeb[(size_t)v * Wd + c / 64];
        if (used) w &= ~(1ull << (c % 64));
        else w |= 1ull << (c % 64);
    };
    auto first_free = [&](int v, int u) {  // first colour free at v (and at u when u >= 0)
        for (int w = 0; w < Wd; ++w) {
            uint64_t f = freeb[(size_t)v * Wd + w];
            if (u >= 0) f &= freeb[(size_t)u * Wd + w];
            if (w == Wd - 1 && D % 64) f &= (1ull << (D % 64)) - 1;
            if (f) return w * 64 + __builtin_ctzll(f);
        }
        return -1;
    };
    auto put = [&](int32_t k, int c) {
        color[(size_t)k] = c;
        at[(size_t)A[(size_t)k] * D + c] = k;
        at[(size_t)B[(size_t)k] * D + c] = k;
        mark(A[(size_t)k], c, true);
        mark(B[(size_t)k], c, true);
    };
    auto take = [&](int32_t k) {
        const int c = color[(size_t)k];
        at[(size_t)A[(size_t)k] * D + c] = -1;
        at[(size_t)B[(size_t)k] * D + c] = -1;
        mark(A[(size_t)k], c, false);
        mark(B[(size_t)k], c, false);
    };
    std::vector<int32_t> path;
    for (int32_t k = 0; k < (int32_t)cnt; ++k) {
        const int a = A[(size_t)k], b = B[(size_t)k];
        int c = first_free(a, b);
        if (c < 0) {
            // colour al free at a, be free at b; swap al/be along the
            // alternating path that starts at b with its al-edge (it never
            // reaches a), after which al is free at both ends
            const int al = first_free(a, -1), be = first_free(b, -1);
            path.clear();
            int v = b, cur = al;
            for (;;) {
                const int32_t k2 = at[(size_t)v * D + cur];
                if (k2 < 0) break;
                path.push_back(k2);
                v = (B[(size_t)k2] == v) ? A[(size_t)k2] : B[(size_t)k2];
                cur = (cur == al) ? be : al;
            }
            std::vector<int> old(path.size());
            for (size_t i = 0; i < path.size(); ++i) {
                old[i] = color[(size_t)path[i]];
                take(path[i]);
            }
            for (size_t i = 0; i < path.size(); ++i) put(path[i], old[i] == al ? be : al);
            c = al;
        }
        put(k, c);
    }
    std::vector<std::vector<int32_t>> groups((size_t)D);
    for (int32_t k = 0; k < (int32_t)cnt; ++k) groups[(size_t)color[(size_t)k]].push_back(k);
    std::stable_sort(groups.begin(), groups.end(),
                     [](const std::vector<int32_t> &x, const std::vector<int32_t> &y) { return x.size() > y.size(); });
    std::vector<int64_t> out;
    out.reserve((size_t)cnt);
    for (auto &g : groups) {
        std::sort(g.begin(), g.end(), [&](int32_t x, int32_t y) { return A[(size_t)x] < A[(size_t)y]; });
        for (int32_t k : g) out.push_back(e[k]);
    }
    std::copy(out.begin(), out.end(), e);
}

extern "C" int cosm_create(const cosm_graph_desc *gd, const cosm_params *p, cosm_handle **out)
{
    NvtxRange range("cosm_create");
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
    if (gd->h) {
        if (p->flags & COSM_OPT_BISECTOR) {
            delete h;
            return fail(COSM_ERR_INVALID_ARG, "local fields fix the readout; COSM_OPT_BISECTOR does not apply");
        }
        int64_t mag = 0;
        for (int64_t e = 0; e < g.m; ++e) mag += std::abs(g.w[(size_t)e]);
        for (int32_t v = 0; v < g.n; ++v) {
            if (gd->h[v] > 32767 || gd->h[v] < -32767) {
                delete h;
                return fail(COSM_ERR_INVALID_ARG, "local field " + std::to_string(v) + " exceeds 32767 in magnitude");
            }
            mag += std::abs(gd->h[v]);
        }
        if (mag >= ((int64_t)1 << 31)) {
            delete h;
            return fail(COSM_ERR_INVALID_ARG, "sum of |w| and |h| must be below 2^31");
        }
        h->fields = true;
    }
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
    {
        std::vector<int32_t> ss((size_t)g.m), ds((size_t)g.m);
        for (int64_t e = 0; e < g.m; ++e) {
            ss[(size_t)e] = h->slot_of[(size_t)g.src[(size_t)e]];
            ds[(size_t)e] = h->slot_of[(size_t)g.dst[(size_t)e]];
        }
        int64_t a = 0;
        while (a < g.m) {
            int64_t z = a;
            while (z < g.m && g.color[(size_t)order[(size_t)z]] == g.color[(size_t)order[(size_t)a]]) ++z;
            if (!std::getenv("COSM_SRC_ORDER")) balance_banks(order.data() + a, z - a, ss, ds);
            a = z;
        }
    }
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
    h->wbound = std::min(colour_weight_bound(h->off, h->C, wv.data(), gd->h, g.n),
                         vertex_weight_bound(g.n, g.m, g.src.data(), g.dst.data(), g.w.data(), gd->h));
    // device copies
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    // records and weights padded with zeros past a multiple of 16 edges: the
    // staged edge-list sweep copies whole 16-byte chunks around each colour
    const size_t m_pad = (((size_t)g.m + 15) & ~(size_t)15) + 16;
    ij.resize(m_pad, 0u);
    wv.resize(m_pad, 0);
    if ((rc = h->d_ij.ensure(m_pad)) || (rc = h->d_w.ensure(m_pad)) ||
        (rc = h->d_orig.ensure((size_t)g.n)) || (rc = h->d_off.ensure((size_t)h->C + 1)) ||
        (rc = h->d_err.ensure(1)) ||
        (rc = h->d_best.ensure(4)) || (rc = h->d_spins.ensure((size_t)g.n))) {
        cosm_destroy(h);
        return rc;
    }
    if (cudaMemcpy(h->d_ij.p, ij.data(), ij.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_w.p, wv.data(), wv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_orig.p, h->orig_of.data(), (size_t)g.n * 4, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(h->d_off.p, h->off, ((size_t)h->C + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d_err.p, 0, 4) != cudaSuccess) {
        cosm_destroy(h);
        return fail(COSM_ERR_CUDA, "copying the graph to the device failed");
    }
    // +-1 weights on at most 2^15 slots: the weight folded into the record
    bool unit = g.n <= (1 << 15);
    for (int64_t k = 0; unit && k < g.m; ++k) unit = wv[(size_t)k] == 1 || wv[(size_t)k] == -1;
    if (unit) {
        std::vector<uint32_t> ijs(m_pad, 0u);
        for (int64_t k = 0; k < g.m; ++k)
            ijs[(size_t)k] = ((ij[(size_t)k] & 0xFFFFu) << 1) | (ij[(size_t)k] & 0xFFFF0000u) | (wv[(size_t)k] < 0 ? 1u : 0u);
        if ((rc = h->d_ijs.ensure(m_pad))) {
            cosm_destroy(h);
            return rc;
        }
        if (cudaMemcpy(h->d_ijs.p, ijs.data(), ijs.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cosm_destroy(h);
            return fail(COSM_ERR_CUDA, "copying the graph to the device failed");
        }
    }
    if (h->fields) {
        std::vector<int32_t> hs((size_t)g.n);
        for (int32_t v = 0; v < g.n; ++v) hs[(size_t)h->slot_of[(size_t)v]] = gd->h[v];
        if ((rc = h->d_h.ensure((size_t)g.n))) {
            cosm_destroy(h);
            return rc;
        }
        if (cudaMemcpy(h->d_h.p, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cosm_destroy(h);
            return fail(COSM_ERR_CUDA, "copying the local fields to the device failed");
        }
    }
    if ((rc = setup_lattice2d(h))) {
        cosm_destroy(h);
        return rc;
    }
    *out = h;
    return COSM_OK;
}

// ------------------------------------------------------------------ layout

int cosm::env_int(const char *name, int dflt)
{
    const char *s = std::getenv(name);
    return (s && *s) ? std::atoi(s) : dflt;
}

// Replicas per CTA (K) and threads per CTA: maximise resident replicas per
// SM (COSM_K / COSM_THREADS override for experiments).
int cosm::choose_layout(cosm_handle *h, int replicas, bool narrow_ties)
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
    // binary32 lattice tiles of two replicas on an even number of block
    // columns take two adjacent 2x2 blocks per thread in the even pass
    // (COSM_SCALAR_F32 and COSM_SINGLE_BLOCKS keep the other passes
    // available as cross-checks)
    const bool pairs_ok = mode == MODE_LATTICE2D_ && p.storage == COSM_F32 && h->Wd % 2 == 0 &&
                          !std::getenv("COSM_SCALAR_F32") && !std::getenv("COSM_SINGLE_BLOCKS");
    long bestScore = -1;
    for (int k = 0; k < 3; ++k) {
        const int K = Ks[k];
        if (forceK && K != forceK) continue;
        const size_t smem = sweep_smem_bytes(p.storage, K, h->g.n, P, mode);
        if (smem > 227 * 1024) continue;
        // thread counts to try: edge-list kernels half a colour class's edges
        // (at most 512, or 1,024 for tiles of two or four replicas and for
        // fixed-point tiles of eight); lattice kernels the 2x2 blocks of a
        // sublattice, up to 512 or, for tiles of at most 4 replicas, 1024
        // threads
        int cand[2] = {0, 0};
        if (forceT) {
            cand[0] = forceT;
        } else if (mode == MODE_LATTICE2D_) {
            for (int c = 0; c < (K <= 4 ? 2 : 1); ++c) {
                int T = std::min(c ? 1024 : 512, std::max(64, (h->Q + 31) / 32 * 32));
                // a multiple of the block-row width fixes each thread's column
                if (h->Wd <= T && (T / h->Wd) * h->Wd >= T / 2) T = (T / h->Wd) * h->Wd;
                cand[c] = T;
            }
            if (cand[1] == cand[0]) cand[1] = 0;
        } else {
            cand[0] = std::min(512, std::max(64, ((max_ec + 1) / 2 + 31) / 32 * 32));
            // tiles of two or four replicas (and fixed-point tiles of eight)
            // may also take 1,024 threads
            if (mode == MODE_GENERAL_ && (K == 2 || K == 4 || p.storage == COSM_Q16))
                cand[1] = std::min(1024, std::max(64, ((max_ec + 1) / 2 + 31) / 32 * 32));
            if (cand[1] == cand[0]) cand[1] = 0;
        }
        for (int c = 0; c < 2 && cand[c]; ++c) {
            int T = cand[c];
            int occ = sweep_occupancy(p.storage, K, mode, T, smem);
            while (occ == 0 && T > 64 && !forceT) {
                T /= 2;
                occ = sweep_occupancy(p.storage, K, mode, T, smem);
            }
            if (occ == 0) continue;
            const long tiles = (replicas + K - 1) / K;
            // resident replicas per SM, capped by what the run can fill; on a
            // tie a larger tile amortises per-edge work when the run fills
            // every CTA slot, a smaller one spreads a small run over more
            // SMs; then more resident threads hide more latency
            const long resident = std::min<long>((long)occ * K, std::max<long>(1, tiles * K / h->num_sms));
            const bool full = tiles >= (long)occ * h->num_sms;
            const long score = resident * 100000 + ((full && !narrow_ties) ? K : -K) * 4096 + (long)occ * T;
            if (score > bestScore) {
                bestScore = score;
                bestK = K;
                bestT = T;
                bestOcc = occ;
            }
        }
    }
    if (!bestK) return fail(COSM_ERR_TOO_LARGE, "no replica tile fits in shared memory");
    h->K = bestK;
    h->threads = bestT;
    h->block_pairs = pairs_ok && bestK == 2;
    h->occupancy = bestOcc;
    h->smem = sweep_smem_bytes(p.storage, bestK, h->g.n, P, mode);
    // binary32 edge lists may stage each colour's records in shared memory
    // (two buffers after the tile) where that keeps the tile's occupancy.
    // Measured slower than the global loads in every case tried (the records
    // stay in L1 / L2, and the copies cost more than their latency), so it is
    // taken only when the environment variable COSM_STAGE is set.
    h->staged = false;
    if (mode == MODE_GENERAL_ && p.storage == COSM_F32 && h->C >= 1 && std::getenv("COSM_STAGE")) {
        const size_t sb = 2 * (size_t)(stage_ij_bytes(max_ec) + stage_w_bytes(max_ec));
        if (h->smem + sb <= 227 * 1024 && sweep_occupancy(p.storage, bestK, mode, bestT, h->smem + sb) >= bestOcc) {
            h->staged = true;
            h->smem += sb;
        }
    }
    const size_t esz = p.storage == COSM_F32 ? 4 : 2;
    h->tile_stride = (int64_t)(((size_t)h->g.n * bestK * esz + 15) / 16 * 16 / esz);
    return COSM_OK;
}

int cosm::ensure_run_buffers(cosm_handle *h, int replicas)
{
    const size_t esz = h->prm.storage == COSM_F32 ? 4 : 2;
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    int rc;
    if ((rc = h->d_state.ensure((size_t)tiles * (size_t)h->tile_stride * esz)) ||
        (rc = h->d_cut.ensure((size_t)replicas)) || (rc = h->d_bestp.ensure((size_t)replicas)) ||
        (rc = h->d_energy.ensure((size_t)replicas)) || (rc = h->d_bisB.ensure((size_t)replicas)) ||
        (rc = h->d_ready.ensure((size_t)tiles)))
        return rc;
    if (h->prm.track_period > 0 &&
        (rc = h->d_bits.ensure((size_t)replicas * (size_t)((h->g.n + 31) / 32))))
        return rc;
    return COSM_OK;
}

int32_t cosm::wrap_period(double alpha0_deg, double dwt_ratio, int dwt_period, int flags, int mode, int storage,
                          int64_t wbound)
{
    if (storage != COSM_F32 || (mode != MODE_LATTICE2D_ && mode != MODE_GENERAL_)) return 1;
    const double a0 = std::fabs(alpha0_deg) / 360.0;
    const bool dwt = !(flags & COSM_NO_DWT) && dwt_period > 0;
    const bool lattice = mode == MODE_LATTICE2D_;
    const double limit = lattice ? 0.999 : 1.999;
    int32_t best = lattice ? 1 : 0, best_dwt = 0;
    for (int P = 1; P <= (lattice ? 4 : 12); ++P) {
        const double twists = dwt ? std::ceil((double)P / dwt_period) : 0.0;
        if (0.5 + (double)wbound * P * a0 + twists * std::fabs(dwt_ratio) * a0 >= limit) break;
        best = P;
        if (dwt && P % dwt_period == 0) best_dwt = P;
    }
    // edge lists wrap in the twist's pass: a multiple of the twist period
    // needs no pass of its own
    return (!lattice && best_dwt) ? best_dwt : best;
}

int64_t cosm::vertex_weight_bound(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
                                  const int32_t *h)
{
    std::vector<int64_t> sum((size_t)n, 0);
    for (int64_t e = 0; e < m; ++e) {
        const int64_t a = std::abs((int64_t)w[e]);
        sum[(size_t)src[e]] += a;
        sum[(size_t)dst[e]] += a;
    }
    int64_t b = 0;
    for (int32_t v = 0; v < n; ++v) b = std::max(b, sum[(size_t)v] + (h ? std::abs((int64_t)h[v]) : 0));
    return b;
}

int64_t cosm::colour_weight_bound(const int32_t *off, int C, const int8_t *w, const int32_t *h, int32_t n)
{
    int64_t b = 0;
    for (int c = 0; c < C; ++c) {
        int32_t mx = 0;
        for (int32_t k = off[c]; k < off[c + 1]; ++k) mx = std::max(mx, (int32_t)std::abs((int32_t)w[k]));
        b += mx;
    }
    int32_t mh = 0;
    if (h)
        for (int32_t v = 0; v < n; ++v) mh = std::max(mh, std::abs(h[v]));
    return b + mh;
}

InstView cosm::inst_view(cosm_handle *h)
{
    InstView v;
    std::memset(&v, 0, sizeof(v));
    v.n = h->g.n;
    v.C = h->C;
    v.off = h->d_off.p;
    v.ij = h->d_ij.p;
    v.w = h->d_w.p;
    // test hook: COSM_SPLIT_W keeps the split records and weights
    v.ijs = std::getenv("COSM_SPLIT_W") ? nullptr : h->d_ijs.p;
    v.orig_of = h->d_orig.p;
    v.wnib = h->d_wnib.p;
    v.Q = h->Q;
    v.Wd = h->Wd;
    v.seed = h->seed;
    v.replicas = h->replicas;
    v.dwt_period = (h->prm.flags & COSM_NO_DWT) ? 0 : h->prm.dwt_period;
    v.window = (float)(h->prm.window_deg / 360.0);
    v.flags = h->prm.flags;
    v.P = h->prm.n_bisectors;
    v.mode = h->mode;
    v.K = h->K;
    v.qwin = (uint32_t)std::min(2147483648.0, std::floor(h->prm.window_deg / 360.0 * 4294967296.0 + 0.5));
    v.state = h->d_state.p;
    v.state_tile_stride = h->tile_stride;
    v.cut = h->d_cut.p;
    v.bestp = h->d_bestp.p;
    v.hv = h->fields ? h->d_h.p : nullptr;
    v.W = h->W;
    v.energy = h->d_energy.p;
    v.bisB = h->d_bisB.p;
    v.words = (h->g.n + 31) / 32;
    // the scalar lattice passes (binary32 and 16-bit storage) stay available
    // as a cross-check
    v.paired = std::getenv("COSM_SCALAR_F32") ? 0 : (h->block_pairs ? 2 : 1);
    v.wrap_p = wrap_period(h->prm.alpha0_deg, h->prm.dwt_ratio, h->prm.dwt_period, h->prm.flags, h->mode,
                           h->prm.storage, h->wbound);
    v.check = h->d_err.p;
    if (h->staged) {
        int max_ec = 0;
        for (int c = 0; c < h->C; ++c) max_ec = std::max(max_ec, h->off[c + 1] - h->off[c]);
        v.stage_ij = stage_ij_bytes(max_ec);
        v.stage_w = stage_w_bytes(max_ec);
    }
    return v;
}

static KernelArgs base_args(cosm_handle *h)
{
    KernelArgs a;
    std::memset(&a, 0, sizeof(a));
    a.v = inst_view(h);
    a.ready = h->d_ready.p;
    a.err = h->d_err.p;
    a.wait_limit_ns = h->wait_limit_ns ? h->wait_limit_ns
                                       : (uint64_t)env_int("COSM_WAIT_LIMIT_S", 20) * 1000000000ull;
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

// Work schedule for sweeps s0..s1 of an S-sweep trial (L = s1 - s0 + 1
// sweeps) of `tiles` tiles on at most G resident CTAs. With tiles <= G every
// CTA runs one tile's whole range. Otherwise the wrap-around rule of
// McNaughton (1959) gives every CTA an equal share of tiles * L sweeps: a
// tile split between CTA b and b+1 runs its head first on b and its tail
// last on b+1 (the share exceeds L, so the two never overlap), and b+1 waits
// for the head's published state before the tail. A range that starts at
// sweep 1 draws the initial phases, a later one loads the stored state; the
// range that ends at sweep S reads out; every range stores its state.
static void build_schedule(cosm_handle *h, int64_t tiles, int64_t s0, int64_t s1, int64_t S, int64_t G)
{
    if (h->sched_tiles == tiles && h->sched_S == S && h->sched_G == G && h->sched_s0 == s0 && h->sched_s1 == s1)
        return;
    h->h_segs.clear();
    h->h_segoff.assign(1, 0);
    h->segs_uploaded = false;
    const int64_t L = s1 - s0 + 1;
    const int32_t first = s0 == 1 ? SEG_INIT : SEG_LOAD;
    const int32_t last = SEG_STORE | (s1 == S ? SEG_READOUT : 0);
    if (tiles <= G) {
        for (int64_t t = 0; t < tiles; ++t) {
            h->h_segs.push_back(Segment{(int32_t)t, first | last, s0, s1});
            h->h_segoff.push_back((int32_t)h->h_segs.size());
        }
    } else {
        const __int128 TL = (__int128)tiles * L;
        for (int64_t b = 0; b < G; ++b) {
            const int64_t lo = (int64_t)(TL * b / G), hi = (int64_t)(TL * (b + 1) / G);
            std::vector<Segment> pieces;
            for (int64_t j = lo / L; j <= (hi - 1) / L && j < tiles; ++j) {
                const int64_t a0 = std::max<int64_t>(lo, j * L) - j * L;
                const int64_t z = std::min<int64_t>(hi, (j + 1) * L) - j * L;
                if (z <= a0) continue;
                Segment sg{(int32_t)j, 0, s0 + a0, s0 + z - 1};
                sg.flags = (a0 == 0) ? first : (SEG_LOAD | SEG_WAIT);
                sg.flags |= (z == L) ? last : (SEG_STORE | SEG_SIGNAL);
                pieces.push_back(sg);
            }
            // execution order: head of the tile continuing on b+1 first, the
            // tail of the tile started on b-1 last
            std::vector<Segment> ordered;
            if (!pieces.empty() && pieces.back().s_begin == s0 && pieces.back().s_end < s1) {
                ordered.push_back(pieces.back());
                pieces.pop_back();
            }
            Segment tail{};
            bool has_tail = false;
            if (!pieces.empty() && pieces.front().s_begin > s0) {
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
    h->sched_s0 = s0;
    h->sched_s1 = s1;
}

int cosm::upload_alpha(cosm_handle *h, int64_t S, cudaStream_t st)
{
    const double a0 = h->prm.alpha0_deg / 360.0, ratio = h->prm.dwt_ratio;
    if (h->alpha_S == S && h->alpha_a0 == a0 && h->alpha_ratio == ratio) return COSM_OK;
    std::vector<float2> tab((size_t)S);
    const bool q16 = h->prm.storage == COSM_Q16;
    for (int64_t s = 1; s <= S; ++s) {
        // linear ramp alpha_0 -> 0 (Table IX), FP64 rounded once to FP32, or
        // for fixed-point phases rounded to the nearest 2^-16-turn quantum
        const double a = (S <= 1) ? a0 : a0 * (double)(S - s) / (double)(S - 1);
        tab[(size_t)(s - 1)] = q16 ? make_float2((float)std::floor(a * 65536.0 + 0.5),
                                                 (float)std::floor(ratio * a * 65536.0 + 0.5))
                                   : make_float2((float)a, (float)(ratio * a));
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

// Optimal-bisector readout of every replica from the stored state, one CTA
// of 1024 threads per replica at a time, one CTA per SM.
int cosm::launch_opt_readout(cosm_handle *h, bool keep_better, cudaStream_t st)
{
    const int n = h->g.n;
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    const int grid = std::max(1, std::min(h->replicas, h->num_sms));
    int rc;
    if ((rc = h->d_qbuf.ensure((size_t)grid * n)) || (rc = h->d_delta.ensure((size_t)grid * n)) ||
        (rc = h->d_items.ensure((size_t)grid * npow2)))
        return rc;
    OptArgs o;
    std::memset(&o, 0, sizeof(o));
    o.v = inst_view(h);
    if (keep_better && h->prm.track_period > 0) o.v.bits = h->d_bits.p;
    o.qbuf = h->d_qbuf.p;
    o.delta = h->d_delta.p;
    o.items = h->d_items.p;
    o.npow2 = npow2;
    o.keep_better = keep_better ? 1 : 0;
    o.storage = h->prm.storage;
    if (opt_readout_launch(o, grid, st))
        return fail(COSM_ERR_CUDA, std::string("optimal-bisector launch: ") + cudaGetErrorString(cudaGetLastError()));
    return COSM_OK;
}

int cosm::launch_finalize(cosm_handle *h, cudaStream_t st)
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
    f.energy = h->d_energy.p;
    f.bisB = h->d_bisB.p;
    f.bits = h->bits_valid ? h->d_bits.p : nullptr;
    f.words = (h->g.n + 31) / 32;
    f.best = h->d_best.p;
    f.spins = h->d_spins.p;
    f.target = h->target;
    if (finalize_launch(f, st)) return fail(COSM_ERR_CUDA, std::string("finalize launch: ") +
                                                          cudaGetErrorString(cudaGetLastError()));
    return COSM_OK;
}

// Sweeps s0..s1 of an S-sweep trial of every replica (cosm_run: 1..S).
static int run_range(cosm_handle *h, int64_t sweeps, int64_t s0, int64_t s1, int32_t replicas, uint64_t seed,
                     int64_t target_cut, cudaStream_t st)
{
    NvtxRange range("cosm_run");
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (sweeps < 1 || sweeps >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "sweeps must be in [1, 2^31)");
    if (replicas < 1 || replicas >= (1 << 24)) return fail(COSM_ERR_INVALID_ARG, "replicas must be in [1, 2^24)");
    if (s0 < 1 || s1 < s0 || s1 > sweeps) return fail(COSM_ERR_INVALID_ARG, "need 1 <= s_from <= s_to <= sweeps");
    int rc;
    if (s0 > 1) {
        // a continued trial keeps its replicas, seed and layout
        if (!h->have_state || h->sweep_idx != s0 - 1)
            return fail(COSM_ERR_STATE, "the state is at sweep " + std::to_string(h->sweep_idx) +
                                            ", not " + std::to_string(s0 - 1));
        if (replicas != h->replicas || seed != h->seed)
            return fail(COSM_ERR_INVALID_ARG, "a continued trial keeps its replica count and seed");
        if (h->stream && h->stream != st) CK(cudaStreamSynchronize(h->stream));
    } else if (!h->K || replicas != h->replicas) {
        if ((rc = choose_layout(h, replicas))) return rc;
    }
    h->replicas = replicas;
    h->seed = seed;
    h->target = target_cut;
    if ((rc = ensure_run_buffers(h, replicas))) return rc;
    if ((rc = upload_alpha(h, sweeps, st))) return rc;
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    int64_t cap = (int64_t)h->occupancy * h->num_sms;
    const int cap_env = env_int("COSM_GRID_CAP", 0);  // test hook: fewer resident CTAs
    if (cap_env > 0) cap = std::min<int64_t>(cap, cap_env);
    build_schedule(h, tiles, s0, s1, sweeps, cap);
    if (h->fault == COSM_FAULT_DROP_SIGNAL) {
        // injected fault: the heads of split tiles do not publish their state,
        // so the tails' bounded waits give up (COSM_ERR_TIMEOUT at cosm_sync)
        for (Segment &sg : h->h_segs) sg.flags &= ~SEG_SIGNAL;
        h->segs_uploaded = false;
        rc = upload_segments(h, st);
        h->sched_tiles = -1;  // the next run rebuilds the true schedule
        h->fault = 0;
        if (rc) return rc;
    } else if ((rc = upload_segments(h, st))) {
        return rc;
    }
    const bool waits = tiles > cap;
    if (waits) CK(cudaMemsetAsync(h->d_ready.p, 0, (size_t)tiles * 4, st));
    CK(cudaMemsetAsync(h->d_err.p, 0, 4, st));
    const int track = h->prm.track_period;
    const int32_t n_trace = track > 0 ? (int32_t)((sweeps + track - 1) / track) : 0;
    if (track > 0 && (rc = h->d_trace.ensure((size_t)replicas * (size_t)n_trace))) return rc;
    KernelArgs a = base_args(h);
    a.v.alpha_tab = h->d_alpha.p;
    a.v.alpha_base = 1;
    a.v.S = sweeps;
    if (track > 0) {
        a.v.track = track;
        a.v.n_trace = n_trace;
        a.v.trace = h->d_trace.p;
        a.v.bits = h->d_bits.p;
    }
    a.segs = h->d_segs.p;
    a.seg_off = h->d_segoff.p;
    LaunchCfg cfg{h->mode, h->prm.storage, h->K, h->threads, (int)(h->h_segoff.size() - 1), h->smem, waits};
    h->grid = cfg.grid;
    if (sweep_launch(cfg, a, st))
        return fail(COSM_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString(cudaGetLastError()));
    h->launches = 1;
    h->stream = st;
    h->have_state = true;
    h->sweep_idx = s1;
    if (s1 < sweeps) {
        // mid-trial: no readout yet
        h->have_result = false;
        h->have_trace = false;
        h->bits_valid = false;
        return COSM_OK;
    }
    h->launches = 2;
    if (h->prm.flags & COSM_OPT_BISECTOR) {
        if ((rc = launch_opt_readout(h, track > 0, st))) return rc;
        h->launches = 3;
    }
    h->bits_valid = track > 0;
    h->n_trace = n_trace;
    h->have_trace = track > 0;
    if ((rc = launch_finalize(h, st))) return rc;
    h->have_result = true;
    return COSM_OK;
}

extern "C" int cosm_run(cosm_handle *h, int64_t sweeps, int32_t replicas, uint64_t seed, int64_t target_cut,
                        void *stream)
{
    return run_range(h, sweeps, 1, sweeps, replicas, seed, target_cut, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cosm_run_range(cosm_handle *h, int64_t sweeps, int64_t s_from, int64_t s_to, int32_t replicas,
                              uint64_t seed, int64_t target_cut, void *stream)
{
    return run_range(h, sweeps, s_from, s_to, replicas, seed, target_cut, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cosm_get_success(cosm_handle *h, int64_t *count)
{
    if (!h || !count) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_result) return fail(COSM_ERR_STATE, "no run or readout yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    CK(cudaMemcpy(count, h->d_best.p + 3, 8, cudaMemcpyDeviceToHost));
    return COSM_OK;
}

extern "C" int cosm_set_wait_limit(cosm_handle *h, double seconds)
{
    if (!h || !(seconds > 0.0) || seconds > 3600.0)
        return fail(COSM_ERR_INVALID_ARG, "the wait limit must be in (0, 3600] seconds");
    h->wait_limit_ns = (uint64_t)(seconds * 1e9);
    return COSM_OK;
}

extern "C" int cosm_inject_fault(cosm_handle *h, int32_t kind)
{
    if (!h || (kind != 0 && kind != COSM_FAULT_DROP_SIGNAL)) return fail(COSM_ERR_INVALID_ARG, "unknown fault");
    h->fault = kind;
    return COSM_OK;
}

extern "C" int cosm_sync(cosm_handle *h)
{
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    int err = 0;
    CK(cudaMemcpy(&err, h->d_err.p, 4, cudaMemcpyDeviceToHost));
    if (err & 2) return fail(COSM_ERR_CHECK, "a device-side index check of the checked build failed");
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

extern "C" int cosm_get_replica_energies(cosm_handle *h, int64_t *energies)
{
    if (!h || !energies) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_result) return fail(COSM_ERR_STATE, "no run or readout yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    CK(cudaMemcpy(energies, h->d_energy.p, (size_t)h->replicas * 8, cudaMemcpyDefault));
    return COSM_OK;
}

extern "C" int cosm_get_replica_bisectors(cosm_handle *h, uint32_t *B)
{
    if (!h || !B) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_result) return fail(COSM_ERR_STATE, "no run or readout yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    CK(cudaMemcpy(B, h->d_bisB.p, (size_t)h->replicas * 4, cudaMemcpyDefault));
    return COSM_OK;
}

extern "C" int cosm_get_trace(cosm_handle *h, int64_t *trace, int64_t count)
{
    if (!h || !trace) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!h->have_trace) return fail(COSM_ERR_STATE, "the last run had no tracking");
    if (count != (int64_t)h->replicas * h->n_trace)
        return fail(COSM_ERR_INVALID_ARG, "count must be replicas x ceil(sweeps / track_period) = " +
                                              std::to_string((int64_t)h->replicas * h->n_trace));
    int rc = cosm_sync(h);
    if (rc) return rc;
    CK(cudaMemcpy(trace, h->d_trace.p, (size_t)count * 8, cudaMemcpyDefault));
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
// Turn in [0, 1) of a stored representative (binary32 lattice phases may sit
// anywhere in (-1, 1) between wraps).
static inline double to_turn(double g)
{
    const double x = g - std::floor(g);
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
            } else if (h->prm.storage == COSM_BF16) {
                __nv_bfloat16 bv;
                std::memcpy(&bv, raw.data() + idx * 2, 2);
                g = (double)__bfloat162float(bv);
            } else if (h->prm.storage == COSM_F16) {
                __half hv;
                std::memcpy(&hv, raw.data() + idx * 2, 2);
                g = (double)__half2float(hv);
            } else {
                uint16_t q;
                std::memcpy(&q, raw.data() + idx * 2, 2);
                g = (double)q / 65536.0;  // fixed point: already a turn in [0, 1)
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
            double x = in[(size_t)r * h->g.n + v] + 0.0;  // -0 becomes +0
            if (!(x >= 0.0 && x < 1.0)) return fail(COSM_ERR_INVALID_ARG, "phases must be in [0, 1)");
            const double g = x >= 0.5 ? x - 1.0 : x;
            const size_t idx = base + (size_t)h->slot_of[(size_t)v] * h->K + (size_t)(r % h->K);
            if (esz == 4) {
                const float f = (float)g;
                std::memcpy(raw.data() + idx * 4, &f, 4);
            } else if (h->prm.storage == COSM_BF16) {
                const __nv_bfloat16 bv = __float2bfloat16_rn((float)g);
                std::memcpy(raw.data() + idx * 2, &bv, 2);
            } else if (h->prm.storage == COSM_F16) {
                const __half hv = __float2half_rn((float)g);
                std::memcpy(raw.data() + idx * 2, &hv, 2);
            } else {
                const uint16_t q = (uint16_t)((uint32_t)std::floor(x * 65536.0 + 0.5) & 0xFFFFu);
                std::memcpy(raw.data() + idx * 2, &q, 2);
            }
        }
    }
    CK(cudaMemcpy(h->d_state.p, raw.data(), raw.size(), cudaMemcpyHostToDevice));
    h->have_state = true;
    h->sweep_idx = 0;
    h->have_result = false;
    h->have_trace = false;
    h->bits_valid = false;
    return COSM_OK;
}

// Checkpoint of the state in its storage type: element (r, v) of the tile
// layout [tile][slot][K] <-> [replica][vertex] in original vertex order.
static size_t storage_bytes(int storage) { return storage == COSM_F32 ? 4 : 2; }

extern "C" int cosm_export_state(cosm_handle *h, void *phases, int32_t storage, int64_t *sweep_idx)
{
    if (!h || !phases) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (storage != h->prm.storage) return fail(COSM_ERR_INVALID_ARG, "storage differs from the handle's");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    int rc = cosm_sync(h);
    if (rc) return rc;
    const int64_t tiles = (h->replicas + h->K - 1) / h->K;
    const size_t esz = storage_bytes(storage);
    std::vector<unsigned char> raw((size_t)tiles * (size_t)h->tile_stride * esz);
    CK(cudaMemcpy(raw.data(), h->d_state.p, raw.size(), cudaMemcpyDeviceToHost));
    std::vector<unsigned char> out((size_t)h->replicas * h->g.n * esz);
    for (int32_t r = 0; r < h->replicas; ++r) {
        const size_t base = (size_t)(r / h->K) * (size_t)h->tile_stride;
        for (int32_t v = 0; v < h->g.n; ++v) {
            const size_t idx = base + (size_t)h->slot_of[(size_t)v] * h->K + (size_t)(r % h->K);
            std::memcpy(out.data() + ((size_t)r * h->g.n + v) * esz, raw.data() + idx * esz, esz);
        }
    }
    CK(cudaMemcpy(phases, out.data(), out.size(), cudaMemcpyDefault));
    if (sweep_idx) *sweep_idx = h->sweep_idx;
    return COSM_OK;
}

extern "C" int cosm_import_state(cosm_handle *h, const void *phases, int32_t storage, int32_t replicas,
                                 uint64_t seed, int64_t sweep_idx)
{
    if (!h || !phases) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (storage != h->prm.storage) return fail(COSM_ERR_INVALID_ARG, "storage differs from the handle's");
    if (replicas < 1 || replicas >= (1 << 24)) return fail(COSM_ERR_INVALID_ARG, "bad replica count");
    if (sweep_idx < 0 || sweep_idx >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "bad sweep index");
    int rc;
    if (h->stream) CK(cudaStreamSynchronize(h->stream));
    if (!h->K || replicas != h->replicas) {
        if ((rc = choose_layout(h, replicas))) return rc;
    }
    h->replicas = replicas;
    h->seed = seed;
    if ((rc = ensure_run_buffers(h, replicas))) return rc;
    const size_t esz = storage_bytes(storage);
    std::vector<unsigned char> in((size_t)replicas * h->g.n * esz);
    CK(cudaMemcpy(in.data(), phases, in.size(), cudaMemcpyDefault));
    const int64_t tiles = (replicas + h->K - 1) / h->K;
    std::vector<unsigned char> raw((size_t)tiles * (size_t)h->tile_stride * esz, 0);
    for (int32_t r = 0; r < replicas; ++r) {
        const size_t base = (size_t)(r / h->K) * (size_t)h->tile_stride;
        for (int32_t v = 0; v < h->g.n; ++v) {
            const size_t idx = base + (size_t)h->slot_of[(size_t)v] * h->K + (size_t)(r % h->K);
            std::memcpy(raw.data() + idx * esz, in.data() + ((size_t)r * h->g.n + v) * esz, esz);
        }
    }
    CK(cudaMemcpy(h->d_state.p, raw.data(), raw.size(), cudaMemcpyHostToDevice));
    h->have_state = true;
    h->sweep_idx = sweep_idx;
    h->have_result = false;
    h->have_trace = false;
    h->bits_valid = false;
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
    a.v.alpha_tab = tab;
    a.v.alpha_base = base;
    a.v.S = s1;
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
    NvtxRange range("cosm_step");
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    if (sweep < 1 || sweep >= ((int64_t)1 << 31)) return fail(COSM_ERR_INVALID_ARG, "bad sweep index");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc;
    DevBuf<float2> tab;  // one-entry step table for this sweep
    if ((rc = tab.ensure(1))) return rc;
    const float2 v = h->prm.storage == COSM_Q16
                         ? make_float2((float)std::floor((double)alpha * 65536.0 + 0.5),
                                       (float)std::floor(h->prm.dwt_ratio * (double)alpha * 65536.0 + 0.5))
                         : make_float2(alpha, (float)(h->prm.dwt_ratio * (double)alpha));
    if (h->stream) CK(cudaStreamSynchronize(h->stream));
    if (cudaMemcpy(tab.p, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess) {
        tab.release();
        return fail(COSM_ERR_CUDA, "alpha upload failed");
    }
    rc = launch_on_state(h, SEG_LOAD | SEG_STORE, sweep, sweep, tab.p, sweep, st);
    if (!rc) rc = cudaStreamSynchronize(st) == cudaSuccess ? COSM_OK : fail(COSM_ERR_CUDA, "step failed");
    tab.release();
    h->sweep_idx = sweep;
    h->have_result = false;
    h->have_trace = false;
    h->bits_valid = false;
    h->launches = 1;
    return rc;
}

extern "C" int cosm_readout(cosm_handle *h, void *stream)
{
    NvtxRange range("cosm_readout");
    if (!h) return fail(COSM_ERR_INVALID_ARG, "NULL handle");
    if (!h->have_state) return fail(COSM_ERR_STATE, "no state yet");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = launch_on_state(h, SEG_LOAD | SEG_READOUT, 1, 0, h->d_alpha.p, 1, st);
    if (rc) return rc;
    h->launches = 2;
    if (h->prm.flags & COSM_OPT_BISECTOR) {
        if ((rc = launch_opt_readout(h, false, st))) return rc;
        h->launches = 3;
    }
    h->bits_valid = false;
    h->have_trace = false;
    if ((rc = launch_finalize(h, st))) return rc;
    h->have_result = true;
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
    rc = cosm_run(h, sweeps, replicas, seed, INT64_MIN, nullptr);
    if (!rc) rc = cosm_get_best(h, best_cut, energy, nullptr, spins);
    if (!rc && replica_cuts) rc = cosm_get_replica_cuts(h, replica_cuts, nullptr);
    cosm_destroy(h);
    return rc;
}

// ====================================================================== batch
// Many instances of uneven size run together. Each instance is a handle as
// above; its replica tiles form units (instance, tile) = one whole trial of
// K replicas. Units of one (storage, K, kernel mode) class share a
// persistent launch whose CTAs drain a queue ordered by decreasing cost
// (longest processing time first); class launches are forked on separate
// streams so a class's tail overlaps the next class's start, and the whole
// run -- counter resets, class kernels, per-instance finalisation -- is
// captured once into a CUDA graph and replayed while the layout is unchanged.

struct BatchClass {
    int storage, K, mode;
    int threads;        // threads per CTA
    size_t smem;        // largest tile of the class
    int grid;           // CTAs (resident capacity, capped by units)
    int32_t unit0, units;
};

struct cosm_batch {
    std::vector<cosm_handle *> hs;
    std::vector<BatchClass> classes;
    std::vector<BatchUnit> h_units;
    DevBuf<BatchUnit> d_units;
    DevBuf<InstView> d_insts;
    DevBuf<BatchFinal> d_fin;
    DevBuf<int32_t> d_counters;
    std::vector<cudaStream_t> side;  // one per class (created on demand)
    std::vector<cudaEvent_t> ev;     // fork + one per class
    cudaStream_t own = nullptr;      // capture stream (the legacy stream cannot capture)
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> sig;        // layout signature of the captured graph
    int policy = 0;                  // 0: per-instance rule for a full GPU, 1: smallest tile, 2: per-instance rule,
                                     // 3: rule for a full GPU with ties to the narrower tile
    int threads = 0;                 // 0: per-class rule, else forced
    cudaStream_t last = nullptr;
    bool have_result = false;
    int64_t launches = 0;
    int64_t graph_builds = 0;
};

extern "C" void cosm_batch_destroy(cosm_batch *b)
{
    if (!b) return;
    if (b->own) cudaStreamSynchronize(b->own);
    // instances first: their handles still name the batch's stream
    for (cosm_handle *h : b->hs) {
        h->stream = nullptr;
        h->have_state = false;
        cosm_destroy(h);
    }
    b->hs.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->own) cudaStreamDestroy(b->own);
    b->d_units.release(); b->d_insts.release(); b->d_fin.release(); b->d_counters.release();
    delete b;
}

extern "C" int cosm_batch_create(int32_t count, const cosm_graph_desc *graphs, const cosm_params *params,
                                 int32_t shared_params, cosm_batch **out)
{
    NvtxRange range("cosm_batch_create");
    if (!graphs || !params || !out || count < 1 || count > (1 << 20))
        return fail(COSM_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    // host-side checks of every instance before any device work
    for (int32_t i = 0; i < count; ++i) {
        const int rc = single_only(&graphs[i], shared_params ? &params[0] : &params[i]);
        if (rc) return fail(rc, "instance " + std::to_string(i) + ": " + g_err);
    }
    cosm_batch *b = new (std::nothrow) cosm_batch();
    if (!b) return fail(COSM_ERR_NOMEM, "host allocation failed");
    // instances are created by host worker threads (validation, colouring
    // and device tables of each run in parallel), each with the caller's
    // device current; the first failing instance is reported
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete b;
        return fail(COSM_ERR_CUDA, "cudaGetDevice failed");
    }
    b->hs.assign((size_t)count, nullptr);
    std::vector<int> rcs((size_t)count, COSM_OK);
    std::vector<std::string> msgs((size_t)count);
    const int workers = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    auto work = [&](int t) {
        cudaSetDevice(dev);
        for (int32_t i = t; i < count; i += workers) {
            const cosm_params *pi = shared_params ? &params[0] : &params[i];
            const int rc = cosm_create(&graphs[i], pi, &b->hs[(size_t)i]);
            if (rc) {
                rcs[(size_t)i] = rc;
                msgs[(size_t)i] = g_err;
            }
        }
    };
    if (workers == 1 || count < 4) {
        work(0);
        for (int t = 1; t < workers; ++t) work(t);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < workers; ++t) pool.emplace_back(work, t);
        for (auto &th : pool) th.join();
    }
    for (int32_t i = 0; i < count; ++i) {
        if (rcs[(size_t)i]) {
            std::string msg = "instance " + std::to_string(i) + ": " + msgs[(size_t)i];
            const int rc = rcs[(size_t)i];
            b->hs.erase(std::remove(b->hs.begin(), b->hs.end(), nullptr), b->hs.end());
            cosm_batch_destroy(b);
            return fail(rc, msg);
        }
    }
    if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
        cosm_batch_destroy(b);
        return fail(COSM_ERR_CUDA, "stream creation failed");
    }
    *out = b;
    return COSM_OK;
}

// Tile layout of one instance inside a batch. Policy 0: the single-instance
// rule (choose_layout) scored as if the run filled every CTA slot, since the
// batch as a whole does: the tile keeping the most replicas resident per SM,
// ties to the wider tile (one edge record and one barrier serve more
// replicas). Policy 1: the narrowest tile of the storage type. Policy 2: the
// single-instance rule with the instance's own replica count. Policy 3: as
// policy 0 with ties to the narrower tile (more CTAs per SM, whose barriers
// and record loads overlap).
static int batch_instance_layout(cosm_batch *b, cosm_handle *h, int32_t replicas)
{
    int rc;
    if (b->policy == 2) return choose_layout(h, replicas);
    if ((rc = choose_layout(h, 1 << 23, b->policy == 3))) return rc;
    if (b->policy == 1 && h->K != (h->prm.storage == COSM_F32 ? 1 : 2)) {
        const int Kmin = h->prm.storage == COSM_F32 ? 1 : 2;
        const size_t esz = h->prm.storage == COSM_F32 ? 4 : 2;
        h->K = Kmin;
        h->block_pairs = false;
        h->staged = false;
        h->smem = sweep_smem_bytes(h->prm.storage, Kmin, h->g.n, h->prm.n_bisectors, h->mode);
        h->tile_stride = (int64_t)(((size_t)h->g.n * Kmin * esz + 15) / 16 * 16 / esz);
        // the narrow tile's kernel may allow fewer threads per CTA
        while (h->threads > 64 && batch_occupancy(h->prm.storage, Kmin, h->mode, h->threads, h->smem) == 0)
            h->threads /= 2;
        h->occupancy = batch_occupancy(h->prm.storage, Kmin, h->mode, h->threads, h->smem);
    }
    return COSM_OK;
}

static int batch_layout(cosm_batch *b, const int64_t *sweeps, const int32_t *replicas, const uint64_t *seeds,
                        cudaStream_t st)
{
    const int n = (int)b->hs.size();
    std::vector<InstView> views((size_t)n);
    std::vector<BatchFinal> fins((size_t)n);
    for (int i = 0; i < n; ++i) {
        cosm_handle *h = b->hs[(size_t)i];
        if (sweeps[i] < 1 || sweeps[i] >= ((int64_t)1 << 31) || replicas[i] < 1 || replicas[i] >= (1 << 24))
            return fail(COSM_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": bad sweeps or replicas");
        int rc;
        if ((rc = batch_instance_layout(b, h, replicas[i]))) return rc;
        if (b->threads) {
            h->threads = b->threads;
            while (h->threads > 64 && batch_occupancy(h->prm.storage, h->K, h->mode, h->threads, h->smem) == 0)
                h->threads /= 2;
        }
        h->replicas = replicas[i];
        h->seed = seeds[i];
        if ((rc = ensure_run_buffers(h, replicas[i]))) return rc;
        if ((rc = upload_alpha(h, sweeps[i], st))) return rc;
        InstView v = inst_view(h);
        v.alpha_tab = h->d_alpha.p;
        v.alpha_base = 1;
        v.S = sweeps[i];
        views[(size_t)i] = v;
        fins[(size_t)i] = BatchFinal{h->W, h->d_spins.p, h->d_best.p, h->prm.storage, 0};
    }
    // classes: instances of one kernel (storage, tile width, mode), thread
    // count and occupancy share a persistent launch (the class's largest
    // tile has the same occupancy as every other, occupancy falling with
    // shared memory); their units form one queue, longest trials first
    b->classes.clear();
    b->h_units.clear();
    struct Key { int storage, K, mode, threads, occ; };
    std::vector<Key> keys;
    std::vector<int> cls((size_t)n);
    for (int i = 0; i < n; ++i) {
        const cosm_handle *h = b->hs[(size_t)i];
        const Key k{h->prm.storage, h->K, h->mode, h->threads,
                    batch_occupancy(h->prm.storage, h->K, h->mode, h->threads, h->smem)};
        int c = -1;
        for (size_t q = 0; q < keys.size() && c < 0; ++q) {
            const Key &o = keys[q];
            if (o.storage == k.storage && o.K == k.K && o.mode == k.mode && o.threads == k.threads && o.occ == k.occ)
                c = (int)q;
        }
        if (c < 0) {
            keys.push_back(k);
            c = (int)keys.size() - 1;
        }
        cls[(size_t)i] = c;
    }
    int dev_sms = b->hs[0]->num_sms;
    for (size_t c = 0; c < keys.size(); ++c) {
        BatchClass bc{keys[c].storage, keys[c].K, keys[c].mode, keys[c].threads, 0, 0,
                      (int32_t)b->h_units.size(), 0};
        std::vector<std::pair<double, BatchUnit>> us;
        for (int i = 0; i < n; ++i) {
            if (cls[(size_t)i] != (int)c) continue;
            const cosm_handle *h = b->hs[(size_t)i];
            bc.smem = std::max(bc.smem, h->smem);
            const int64_t tiles = (replicas[i] + h->K - 1) / h->K;
            const double cost = (double)h->g.m * (double)h->K * (double)sweeps[i];
            for (int64_t t = 0; t < tiles; ++t)
                us.push_back({cost, BatchUnit{i, (int32_t)t, SEG_INIT | SEG_READOUT | SEG_STORE, 0, 1, sweeps[i]}});
        }
        std::stable_sort(us.begin(), us.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
        for (auto &u : us) b->h_units.push_back(u.second);
        bc.units = (int32_t)us.size();
        int T = bc.threads;
        int occ = batch_occupancy(bc.storage, bc.K, bc.mode, T, bc.smem);
        while (occ == 0 && T > 64) {
            T /= 2;
            occ = batch_occupancy(bc.storage, bc.K, bc.mode, T, bc.smem);
        }
        if (occ == 0) return fail(COSM_ERR_TOO_LARGE, "a batch tile does not fit on an SM");
        bc.threads = T;
        bc.grid = (int)std::min<int64_t>((int64_t)occ * dev_sms, bc.units);
        b->classes.push_back(bc);
    }
    int rc;
    if ((rc = b->d_insts.ensure((size_t)n)) || (rc = b->d_fin.ensure((size_t)n)) ||
        (rc = b->d_units.ensure(b->h_units.size())) || (rc = b->d_counters.ensure(b->classes.size())))
        return rc;
    CK(cudaMemcpyAsync(b->d_insts.p, views.data(), views.size() * sizeof(InstView), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->d_fin.p, fins.data(), fins.size() * sizeof(BatchFinal), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->d_units.p, b->h_units.data(), b->h_units.size() * sizeof(BatchUnit),
                       cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // host tables are released on return
    return COSM_OK;
}

// Records the class launches and the finaliser on `st` (captured or not).
static int batch_enqueue(cosm_batch *b, cudaStream_t st)
{
    const size_t nc = b->classes.size();
    while (b->side.size() < nc) {
        cudaStream_t s;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->side.push_back(s);
    }
    while (b->ev.size() < nc + 1) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->ev.push_back(e);
    }
    CK(cudaMemsetAsync(b->d_counters.p, 0, nc * 4, st));
    CK(cudaEventRecord(b->ev[0], st));
    for (size_t c = 0; c < nc; ++c) {
        const BatchClass &bc = b->classes[c];
        CK(cudaStreamWaitEvent(b->side[c], b->ev[0], 0));
        BatchArgs a{b->d_insts.p, b->d_units.p + bc.unit0, bc.units, b->d_counters.p + c};
        if (bc.units > 0 && batch_launch(bc.storage, bc.K, bc.mode, bc.grid, bc.threads, bc.smem, a, b->side[c]))
            return fail(COSM_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(cudaGetLastError()));
        CK(cudaEventRecord(b->ev[c + 1], b->side[c]));
    }
    for (size_t c = 0; c < nc; ++c) CK(cudaStreamWaitEvent(st, b->ev[c + 1], 0));
    if (batch_finalize_launch((int)b->hs.size(), b->d_insts.p, b->d_fin.p, st))
        return fail(COSM_ERR_CUDA, std::string("batch finalize: ") + cudaGetErrorString(cudaGetLastError()));
    return COSM_OK;
}

extern "C" int cosm_batch_run(cosm_batch *b, const int64_t *sweeps, const int32_t *replicas,
                              const uint64_t *seeds, void *stream)
{
    NvtxRange range("cosm_batch_run");
    if (!b || !sweeps || !replicas || !seeds) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t st = b->own;
    // order the batch after earlier work on the caller's stream
    cudaEvent_t e0;
    CK(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    CK(cudaEventRecord(e0, user));
    CK(cudaStreamWaitEvent(st, e0, 0));
    cudaEventDestroy(e0);
    int rc = batch_layout(b, sweeps, replicas, seeds, st);
    if (rc) return rc;
    std::vector<int64_t> sig;
    sig.push_back((int64_t)(uintptr_t)b->d_insts.p);
    sig.push_back((int64_t)(uintptr_t)b->d_units.p);
    sig.push_back((int64_t)(uintptr_t)b->d_counters.p);
    for (const BatchClass &bc : b->classes) {
        sig.push_back(bc.storage); sig.push_back(bc.K); sig.push_back(bc.mode); sig.push_back(bc.threads);
        sig.push_back((int64_t)bc.smem); sig.push_back(bc.grid); sig.push_back(bc.unit0); sig.push_back(bc.units);
    }
    if (!b->exec || sig != b->sig) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        rc = batch_enqueue(b, st);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(COSM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        b->sig = sig;
        b->graph_builds++;
    }
    CK(cudaGraphLaunch(b->exec, st));
    cudaEvent_t e1;
    CK(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
    CK(cudaEventRecord(e1, st));
    CK(cudaStreamWaitEvent(user, e1, 0));
    cudaEventDestroy(e1);
    for (cosm_handle *h : b->hs) {
        h->stream = st;
        h->have_state = true;
        h->have_result = true;
    }
    b->last = st;
    b->have_result = true;
    b->launches = (int64_t)b->classes.size() + 1;
    return COSM_OK;
}

extern "C" int cosm_batch_sync(cosm_batch *b)
{
    if (!b) return fail(COSM_ERR_INVALID_ARG, "NULL batch");
    CK(cudaStreamSynchronize(b->own));
    return COSM_OK;
}

extern "C" int cosm_batch_get_best(cosm_batch *b, int32_t i, int64_t *cut, int64_t *energy, int32_t *replica,
                                   int8_t *spins)
{
    if (!b || i < 0 || i >= (int32_t)b->hs.size()) return fail(COSM_ERR_INVALID_ARG, "bad instance index");
    if (!b->have_result) return fail(COSM_ERR_STATE, "no batch run yet");
    return cosm_get_best(b->hs[(size_t)i], cut, energy, replica, spins);
}

extern "C" int cosm_batch_get_replica_cuts(cosm_batch *b, int32_t i, int64_t *cuts, int32_t *best_p)
{
    if (!b || i < 0 || i >= (int32_t)b->hs.size()) return fail(COSM_ERR_INVALID_ARG, "bad instance index");
    if (!b->have_result) return fail(COSM_ERR_STATE, "no batch run yet");
    return cosm_get_replica_cuts(b->hs[(size_t)i], cuts, best_p);
}

extern "C" int cosm_batch_get_state(cosm_batch *b, int32_t i, double *phases)
{
    if (!b || i < 0 || i >= (int32_t)b->hs.size()) return fail(COSM_ERR_INVALID_ARG, "bad instance index");
    return cosm_get_state(b->hs[(size_t)i], phases);
}

// Autotuner: times short runs of the whole batch (probe_sweeps sweeps per
// instance, the caller's replica counts) for each tile policy and thread
// count and keeps the fastest. With COSM_TUNE_CACHE set, choices are read
// from / appended to that text file, keyed by the batch's shape.
extern "C" int cosm_batch_tune(cosm_batch *b, const int32_t *replicas, int64_t probe_sweeps, void *stream)
{
    NvtxRange range("cosm_batch_tune");
    if (!b || !replicas || probe_sweeps < 1) return fail(COSM_ERR_INVALID_ARG, "bad tuning arguments");
    const size_t n = b->hs.size();
    uint64_t key = 1469598103934665603ull;  // FNV-1a over the batch's shape
    auto mix = [&](uint64_t x) {
        for (int k = 0; k < 8; ++k) { key ^= (x >> (8 * k)) & 0xFF; key *= 1099511628211ull; }
    };
    for (size_t i = 0; i < n; ++i) {
        const cosm_handle *h = b->hs[i];
        mix((uint64_t)h->g.n); mix((uint64_t)h->g.m); mix((uint64_t)h->C); mix((uint64_t)h->mode);
        mix((uint64_t)h->prm.storage); mix((uint64_t)replicas[i]);
    }
    const char *cache = std::getenv("COSM_TUNE_CACHE");
    if (cache) {
        FILE *f = std::fopen(cache, "r");
        if (f) {
            unsigned long long k;
            int pol, thr;
            while (std::fscanf(f, "%llx %d %d", &k, &pol, &thr) == 3)
                if (k == key) {
                    b->policy = pol;
                    b->threads = thr;
                    std::fclose(f);
                    return COSM_OK;
                }
            std::fclose(f);
        }
    }
    std::vector<int64_t> sw(n, probe_sweeps);
    std::vector<uint64_t> seeds(n, 12345);
    float best_ms = 1e30f;
    int best_pol = 0, best_thr = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // policies with the rule's thread counts, then the default policy with
    // forced thread counts
    const int cfgs[8][2] = {{0, 0}, {1, 0}, {2, 0}, {3, 0}, {0, 128}, {0, 256}, {0, 512}, {3, 256}};
    for (const auto &cf : cfgs) {
        const int pol = cf[0], thr = cf[1];
        b->policy = pol;
        b->threads = thr;
        int rc = cosm_batch_run(b, sw.data(), replicas, seeds.data(), stream);  // warm-up + graph build
        if (rc) continue;
        CK(cudaEventRecord(e0, b->own));
        rc = cosm_batch_run(b, sw.data(), replicas, seeds.data(), stream);
        CK(cudaEventRecord(e1, b->own));
        CK(cudaEventSynchronize(e1));
        if (rc) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_pol = pol;
            best_thr = thr;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->policy = best_pol;
    b->threads = best_thr;
    if (cache) {
        FILE *f = std::fopen(cache, "a");
        if (f) {
            std::fprintf(f, "%llx %d %d\n", (unsigned long long)key, best_pol, best_thr);
            std::fclose(f);
        }
    }
    return COSM_OK;
}

extern "C" int cosm_batch_layout(cosm_batch *b, int32_t i, int32_t out[8])
{
    if (!b || i < 0 || i >= (int32_t)b->hs.size()) return fail(COSM_ERR_INVALID_ARG, "bad instance index");
    if (!b->have_result) return fail(COSM_ERR_STATE, "no batch run yet");
    return cosm_layout(b->hs[(size_t)i], out);
}

extern "C" int cosm_batch_info(cosm_batch *b, int64_t out[8])
{
    if (!b || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    out[0] = (int64_t)b->hs.size();
    out[1] = (int64_t)b->classes.size();
    out[2] = (int64_t)b->h_units.size();
    out[3] = b->launches;
    out[4] = b->graph_builds;
    out[5] = b->policy;
    out[6] = b->threads;
    int64_t ctas = 0;
    for (const BatchClass &bc : b->classes) ctas += bc.grid;
    out[7] = ctas;
    return COSM_OK;
}
