// Host graph tools: validation of the instance and of its edge partition,
// edge colourings (Alg. 1 line 1) and the lattice relabel used to lay the
// phases out in shared memory.
#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_internal.h"

namespace cosm {

int validate_graph(const Graph &g, std::string &why)
{
    if (g.n < 2 || g.n > kMaxVertices) {
        why = "n must be in [2, 65536]";
        return COSM_ERR_INVALID_ARG;
    }
    if (g.m < 1 || g.m > (int64_t)1 << 26) {
        why = "m must be in [1, 2^26]";
        return COSM_ERR_INVALID_ARG;
    }
    std::vector<int64_t> key((size_t)g.m);
    int64_t abs_sum = 0;
    for (int64_t e = 0; e < g.m; ++e) {
        int32_t a = g.src[(size_t)e], b = g.dst[(size_t)e], wt = g.w[(size_t)e];
        if (a < 0 || b >= g.n || a >= b) {
            why = "edge " + std::to_string(e) + " is not canonical (0 <= src < dst < n)";
            return COSM_ERR_INVALID_ARG;
        }
        if (wt == 0 || wt > 127 || wt < -127) {
            why = "edge " + std::to_string(e) + " weight must satisfy 1 <= |w| <= 127";
            return COSM_ERR_INVALID_ARG;
        }
        abs_sum += std::abs(wt);
        key[(size_t)e] = (int64_t)a * g.n + b;
    }
    if (abs_sum >= ((int64_t)1 << 31)) {
        why = "sum of |w| must be below 2^31";
        return COSM_ERR_INVALID_ARG;
    }
    std::sort(key.begin(), key.end());
    for (size_t e = 1; e < key.size(); ++e)
        if (key[e] == key[e - 1]) {
            why = "duplicate edge";
            return COSM_ERR_INVALID_ARG;
        }
    return COSM_OK;
}

int validate_partition(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t C,
                       const int32_t *color, std::string &why)
{
    if (C < 1 || C > kMaxColors) {
        why = "n_colors must be in [1, 64]";
        return COSM_ERR_PARTITION;
    }
    // last[v * C + c] = 1 once vertex v has an edge of colour c
    std::vector<uint8_t> seen((size_t)n * (size_t)C, 0);
    for (int64_t e = 0; e < m; ++e) {
        int32_t c = color[e];
        if (c < 0 || c >= C) {
            why = "edge " + std::to_string(e) + " has colour outside [0, n_colors)";
            return COSM_ERR_PARTITION;
        }
        size_t a = (size_t)src[e] * C + c, b = (size_t)dst[e] * C + c;
        if (seen[a] || seen[b]) {
            why = "colour " + std::to_string(c) + " is not a matching (edge " + std::to_string(e) + ")";
            return COSM_ERR_NOT_A_MATCHING;
        }
        seen[a] = seen[b] = 1;
    }
    return COSM_OK;
}

static int max_degree(int32_t n, int64_t m, const int32_t *src, const int32_t *dst)
{
    std::vector<int32_t> deg((size_t)n, 0);
    int D = 0;
    for (int64_t e = 0; e < m; ++e) {
        D = std::max(D, ++deg[(size_t)src[e]]);
        D = std::max(D, ++deg[(size_t)dst[e]]);
    }
    return D;
}

int color_greedy(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *color,
                 int32_t *C)
{
    const int K = std::max(1, 2 * max_degree(n, m, src, dst) - 1);
    // per-vertex bitmask of used colours, K <= 2*Delta - 1 words of 64 bits
    const int words = (K + 63) / 64;
    std::vector<uint64_t> used((size_t)n * words, 0);
    int32_t ncol = 0;
    for (int64_t e = 0; e < m; ++e) {
        const uint64_t *ua = &used[(size_t)src[e] * words];
        const uint64_t *ub = &used[(size_t)dst[e] * words];
        int c = -1;
        for (int wd = 0; wd < words && c < 0; ++wd) {
            uint64_t freebits = ~(ua[wd] | ub[wd]);
            if (freebits) c = wd * 64 + __builtin_ctzll(freebits);
        }
        color[e] = c;
        used[(size_t)src[e] * words + c / 64] |= 1ull << (c % 64);
        used[(size_t)dst[e] * words + c / 64] |= 1ull << (c % 64);
        ncol = std::max(ncol, c + 1);
    }
    *C = ncol;
    return COSM_OK;
}

// Misra-Gries (1992): colour edges one at a time; for an uncoloured (u, v)
// build a maximal fan at u, flip the cd-path at u, rotate a fan prefix and
// colour its last edge with d. Uses at most Delta + 1 colours.
int color_misra_gries(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *color,
                      int32_t *C)
{
    const int K = max_degree(n, m, src, dst) + 1;
    std::vector<int32_t> at((size_t)n * K, -1);  // at[v*K + c] = edge of colour c at v
    std::vector<std::vector<int32_t>> adj((size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        adj[(size_t)src[e]].push_back((int32_t)e);
        adj[(size_t)dst[e]].push_back((int32_t)e);
        color[e] = -1;
    }
    auto other = [&](int32_t e, int32_t x) { return src[e] == x ? dst[e] : src[e]; };
    auto is_free = [&](int32_t v, int c) { return at[(size_t)v * K + c] < 0; };
    auto set_col = [&](int32_t e, int c) {
        color[e] = c;
        at[(size_t)src[e] * K + c] = e;
        at[(size_t)dst[e] * K + c] = e;
    };
    auto clear_col = [&](int32_t e) {
        int c = color[e];
        if (c >= 0) {
            at[(size_t)src[e] * K + c] = -1;
            at[(size_t)dst[e] * K + c] = -1;
        }
        color[e] = -1;
    };
    std::vector<int32_t> fan, fan_e, path;
    std::vector<uint8_t> in_fan((size_t)n, 0);
    for (int64_t e0 = 0; e0 < m; ++e0) {
        const int32_t u = src[e0];
        fan.assign(1, dst[e0]);
        fan_e.assign(1, (int32_t)e0);
        in_fan[(size_t)dst[e0]] = 1;
        for (bool grown = true; grown;) {
            grown = false;
            const int32_t last = fan.back();
            for (int32_t e : adj[(size_t)u]) {
                if (color[e] < 0) continue;
                int32_t x = other(e, u);
                if (in_fan[(size_t)x] || !is_free(last, color[e])) continue;
                fan.push_back(x);
                fan_e.push_back(e);
                in_fan[(size_t)x] = 1;
                grown = true;
                break;
            }
        }
        int c = 0, d = 0;
        while (!is_free(u, c)) ++c;
        while (!is_free(fan.back(), d)) ++d;
        if (c != d) {
            // cd-path from u: starts with colour d (c is free at u)
            path.clear();
            int32_t x = u;
            int col = d;
            while (at[(size_t)x * K + col] >= 0) {
                int32_t e = at[(size_t)x * K + col];
                path.push_back(e);
                x = other(e, x);
                col = (col == d) ? c : d;
                if ((int64_t)path.size() > m) return COSM_ERR_INVALID_ARG;  // cannot happen
            }
            std::vector<int> newc(path.size());
            for (size_t k = 0; k < path.size(); ++k) newc[k] = (color[path[k]] == d) ? c : d;
            for (int32_t e : path) clear_col(e);
            for (size_t k = 0; k < path.size(); ++k) set_col(path[k], newc[k]);
        }
        // first w in the fan with d free whose prefix is still a fan
        int idx = -1;
        for (size_t k = 0; k < fan.size() && idx < 0; ++k) {
            bool prefix_ok = true;
            for (size_t t = 1; t <= k && prefix_ok; ++t)
                prefix_ok = color[fan_e[t]] >= 0 && is_free(fan[t - 1], color[fan_e[t]]);
            if (prefix_ok && is_free(fan[k], d)) idx = (int)k;
        }
        for (int32_t x : fan) in_fan[(size_t)x] = 0;
        if (idx < 0) return COSM_ERR_INVALID_ARG;  // contradicts the theorem
        std::vector<int> shifted((size_t)idx);
        for (int t = 0; t < idx; ++t) shifted[(size_t)t] = color[fan_e[(size_t)t + 1]];
        for (int t = 1; t <= idx; ++t) clear_col(fan_e[(size_t)t]);
        for (int t = 0; t < idx; ++t) set_col(fan_e[(size_t)t], shifted[(size_t)t]);
        set_col(fan_e[(size_t)idx], d);
    }
    int32_t ncol = 0;
    for (int64_t e = 0; e < m; ++e) ncol = std::max(ncol, color[e] + 1);
    *C = ncol;
    return COSM_OK;
}

int color_torus2d(int32_t L1, int32_t L2, int64_t m, const int32_t *src, const int32_t *dst,
                  int32_t *color)
{
    if (L1 < 4 || L2 < 4 || (L1 & 1) || (L2 & 1)) return COSM_ERR_INVALID_ARG;
    for (int64_t e = 0; e < m; ++e) {
        const int32_t a = src[e], b = dst[e];
        if (b >= L1 * L2) return COSM_ERR_INVALID_ARG;
        const int32_t ra = a / L2, ca = a % L2, rb = b / L2, cb = b % L2;
        // order: even-column horizontal, even-row vertical, odd-column
        // horizontal, odd-row vertical (consecutive pairs act on 2x2 blocks)
        if (ra == rb && (ca + 1) % L2 == cb) color[e] = (ca & 1) ? 2 : 0;
        else if (ra == rb && (cb + 1) % L2 == ca) color[e] = (cb & 1) ? 2 : 0;
        else if (ca == cb && (ra + 1) % L1 == rb) color[e] = (ra & 1) ? 3 : 1;
        else if (ca == cb && (rb + 1) % L1 == ra) color[e] = (rb & 1) ? 3 : 1;
        else return COSM_ERR_INVALID_ARG;
    }
    return COSM_OK;
}

int color_torus3d(int32_t L1, int32_t L2, int32_t L3, int64_t m, const int32_t *src,
                  const int32_t *dst, int32_t *color)
{
    const int32_t L[3] = {L1, L2, L3};
    for (int a = 0; a < 3; ++a)
        if (L[a] < 4 || (L[a] & 1)) return COSM_ERR_INVALID_ARG;
    for (int64_t e = 0; e < m; ++e) {
        int32_t co[2][3];
        const int32_t u[2] = {src[e], dst[e]};
        if (u[1] >= L1 * L2 * L3) return COSM_ERR_INVALID_ARG;
        for (int t = 0; t < 2; ++t) {
            co[t][2] = u[t] % L3;
            co[t][1] = (u[t] / L3) % L2;
            co[t][0] = u[t] / (L2 * L3);
        }
        int c = -1;
        for (int a = 0; a < 3 && c < 0; ++a) {
            bool same = true;
            for (int b = 0; b < 3; ++b)
                if (b != a && co[0][b] != co[1][b]) same = false;
            if (!same) continue;
            // all even classes (axes 0, 1, 2), then all odd classes
            if ((co[0][a] + 1) % L[a] == co[1][a]) c = 3 * (co[0][a] & 1) + a;
            else if ((co[1][a] + 1) % L[a] == co[0][a]) c = 3 * (co[1][a] & 1) + a;
        }
        if (c < 0) return COSM_ERR_INVALID_ARG;
        color[e] = c;
    }
    return COSM_OK;
}

// Sublattice relabel: vertices are grouped by the parity of each lattice
// coordinate, row-major inside a group. In the regular colouring every
// colour then pairs slot f of one group with slot f (or f + 1, f + row) of
// another, so consecutive threads touch consecutive shared-memory words.
bool lattice_relabel(const Graph &g, std::vector<int32_t> &slot_of, std::string &why)
{
    const int32_t *d = g.dims;
    std::vector<int32_t> col((size_t)g.m);
    slot_of.assign((size_t)g.n, 0);
    if (d[0] > 0 && d[1] > 0 && d[2] == 0) {
        const int32_t L1 = d[0], L2 = d[1];
        // any subset of the torus edges (e.g. couplings that cancelled to 0)
        if ((int64_t)L1 * L2 != g.n || g.m > 2 * (int64_t)g.n ||
            color_torus2d(L1, L2, g.m, g.src.data(), g.dst.data(), col.data()) != COSM_OK) {
            why = "dims does not describe this graph as an even-sided 2D torus";
            return false;
        }
        const int32_t q = g.n / 4, hw = L2 / 2;
        for (int32_t v = 0; v < g.n; ++v) {
            int32_t r = v / L2, c = v % L2;
            slot_of[(size_t)v] = ((r & 1) * 2 + (c & 1)) * q + (r >> 1) * hw + (c >> 1);
        }
        return true;
    }
    if (d[0] > 0 && d[1] > 0 && d[2] > 0) {
        const int32_t L1 = d[0], L2 = d[1], L3 = d[2];
        if ((int64_t)L1 * L2 * L3 != g.n || g.m > 3 * (int64_t)g.n ||
            color_torus3d(L1, L2, L3, g.m, g.src.data(), g.dst.data(), col.data()) != COSM_OK) {
            why = "dims does not describe this graph as an even-sided 3D torus";
            return false;
        }
        const int32_t q = g.n / 8, h2 = L2 / 2, h3 = L3 / 2;
        for (int32_t v = 0; v < g.n; ++v) {
            int32_t k = v % L3, j = (v / L3) % L2, i = v / (L2 * L3);
            int32_t grp = (i & 1) * 4 + (j & 1) * 2 + (k & 1);
            slot_of[(size_t)v] = grp * q + ((i >> 1) * h2 + (j >> 1)) * h3 + (k >> 1);
        }
        return true;
    }
    why = "no lattice hint";
    return false;
}

}  // namespace cosm

// QUBO -> Ising (eq. (1)) with x_i = (1 + s_i) / 2: for i < j the pair
// coefficient c_ij = Q_ij + Q_ji gives x_i x_j = (1 + s_i + s_j + s_i s_j) / 4,
// and a diagonal Q_ii gives x_i = (1 + s_i) / 2; collecting terms,
//   4 f(x) = sum_{i<j} c_ij s_i s_j + sum_i s_i (sum_j c_ij + 2 Q_ii)
//            + sum_{i<j} c_ij + 2 sum_i Q_ii,
// i.e. Max-Cut weights w_ij = c_ij, fields h_i = -(sum_j c_ij + 2 Q_ii).
extern "C" int cosm_qubo_to_ising(int32_t n, int64_t nnz, const int32_t *qi, const int32_t *qj,
                                  const int64_t *qv, int32_t *src, int32_t *dst, int32_t *w, int64_t *m,
                                  int32_t *h, int64_t *offset)
{
    using namespace cosm;
    if (n < 1 || nnz < 0 || (nnz > 0 && (!qi || !qj || !qv)) || !src || !dst || !w || !m || !h ||
        !offset) {
        set_last_error("bad arguments");
        return COSM_ERR_INVALID_ARG;
    }
    std::vector<std::pair<int64_t, int64_t>> pairs;  // (i n + j, c) with i < j
    pairs.reserve((size_t)nnz);
    std::vector<int64_t> diag((size_t)n, 0), hsum((size_t)n, 0);
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t i = qi[k], j = qj[k];
        if (i < 0 || i >= n || j < 0 || j >= n) {
            set_last_error("triplet " + std::to_string(k) + " has an index outside [0, n)");
            return COSM_ERR_INVALID_ARG;
        }
        if (i == j) diag[(size_t)i] += qv[k];
        else pairs.emplace_back((int64_t)std::min(i, j) * n + std::max(i, j), qv[k]);
    }
    std::sort(pairs.begin(), pairs.end());
    int64_t cnt = 0, off = 0;
    for (size_t a = 0; a < pairs.size();) {
        const int64_t key = pairs[a].first;
        int64_t c = 0;
        while (a < pairs.size() && pairs[a].first == key) c += pairs[a++].second;
        if (c == 0) continue;
        if (c > 127 || c < -127) {
            set_last_error("pair weight " + std::to_string(c) + " exceeds 127 in magnitude");
            return COSM_ERR_TOO_LARGE;
        }
        const int32_t i = (int32_t)(key / n), j = (int32_t)(key % n);
        src[cnt] = i;
        dst[cnt] = j;
        w[cnt] = (int32_t)c;
        ++cnt;
        hsum[(size_t)i] += c;
        hsum[(size_t)j] += c;
        off += c;
    }
    for (int32_t v = 0; v < n; ++v) {
        const int64_t hv = -(hsum[(size_t)v] + 2 * diag[(size_t)v]);
        if (hv > 32767 || hv < -32767) {
            set_last_error("field of vertex " + std::to_string(v) + " exceeds 32767 in magnitude");
            return COSM_ERR_TOO_LARGE;
        }
        h[v] = (int32_t)hv;
        off += 2 * diag[(size_t)v];
    }
    *m = cnt;
    *offset = off;
    return COSM_OK;
}
