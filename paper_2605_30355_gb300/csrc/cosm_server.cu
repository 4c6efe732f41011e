// Serving loop with continuous batching. Requests (an instance, a trial
// length, replicas, a target cut) arrive at any time; a worker thread admits
// queued requests in arrival order while a slot is free and their device
// footprint fits the memory budget, keeps every admitted request's phases on
// the device, and advances all active requests together in chunks of
// sweeps: one queue launch per (storage, tile width, kernel) class runs a
// chunk of every active request's tiles, the state staying in global memory
// between chunks. A trial that ends is read out; a request whose best cut
// reaches its target (or that has used its trials) retires, freeing its slot
// and memory for the next arrival. Trial t of a request uses the seed
// seed + t * 0x9E3779B97F4A7C15, so each trial -- and so the request's
// result -- is the same alone and in any mix, and whatever the chunk size.
#include <cuda_runtime.h>

#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cosm.h"
#include "cosm_handle.h"
#include "cosm_internal.h"

using namespace cosm;

namespace {

enum ReqStatus { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_REACHED = 2, RQ_EXHAUSTED = 3 };

struct Request {
    int64_t id = 0;
    int32_t n = 0;
    std::vector<int32_t> src, dst, w, color;
    int32_t n_colors = 0;
    int32_t dims[3] = {0, 0, 0};
    cosm_params prm;
    int64_t S = 0;
    int32_t R = 0;
    uint64_t seed = 0;
    int64_t target = 0;
    int32_t max_trials = 1;
    size_t footprint = 0;
    cosm_handle *h = nullptr;
    int32_t trial = 0;   // trial in progress (or trials done once retired)
    int64_t pos = 0;     // sweeps done in the trial in progress
    int64_t best_cut = LLONG_MIN, energy = 0;
    int32_t best_trial = -1, best_replica = -1;
    std::vector<int8_t> spins;
    int status = RQ_QUEUED;
    int error = 0;
    double t_submit = 0, t_admit = -1, t_done = -1, ttt = -1;
    int64_t updates = 0;
};

uint64_t trial_seed(uint64_t seed, int32_t t) { return seed + (uint64_t)t * 0x9E3779B97F4A7C15ull; }

}  // namespace

struct cosm_server {
    cosm_server_config cfg;
    int device = 0;
    int num_sms = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::unordered_map<int64_t, Request *> all;
    int64_t next_id = 1;
    bool stop = false;
    size_t footprint = 0, peak_footprint = 0;
    int64_t max_concurrent = 0, chunks = 0, launches = 0, retired = 0;
    cudaStream_t st = nullptr;
    DevBuf<InstView> d_insts;
    DevBuf<BatchUnit> d_units;
    DevBuf<int32_t> d_counters;
    std::thread worker;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Device bytes a request holds while admitted: edge records and weights,
// vertex table, offsets, phases of all replicas (rounded to 16-byte tiles),
// per-replica outputs, the step table, spins, block weight bits.
static size_t estimate_footprint(const Request &r)
{
    const size_t esz = r.prm.storage == COSM_F32 ? 4 : 2;
    const size_t m = r.src.size();
    const size_t state = (size_t)r.R * ((size_t)r.n * esz + 16 * 4);
    // per replica: cut, bisector index, energy, bisector position (24 bytes)
    return 5 * m + 4 * (size_t)r.n + 4 * 65 + state + 24 * (size_t)r.R + 8 * (size_t)r.S + (size_t)r.n +
           (size_t)r.n / 2 + 4096;
}

static int admit(cosm_server *s, Request *r)
{
    cosm_graph_desc d;
    std::memset(&d, 0, sizeof(d));
    d.n = r->n;
    d.m = (int64_t)r->src.size();
    d.src = r->src.data();
    d.dst = r->dst.data();
    d.w = r->w.data();
    d.n_colors = r->n_colors;
    d.color = r->color.empty() ? nullptr : r->color.data();
    for (int k = 0; k < 3; ++k) d.dims[k] = r->dims[k];
    int rc = cosm_create(&d, &r->prm, &r->h);
    if (rc) return rc;
    if ((rc = choose_layout(r->h, r->R))) return rc;
    r->h->replicas = r->R;
    if ((rc = ensure_run_buffers(r->h, r->R))) return rc;
    if ((rc = upload_alpha(r->h, r->S, s->st))) return rc;
    r->h->stream = s->st;
    return COSM_OK;
}

static void retire(cosm_server *s, Request *r, int status)
{
    r->status = status;
    r->t_done = s->now();
    if (r->h) {
        cosm_destroy(r->h);
        r->h = nullptr;
    }
    s->footprint -= r->footprint;
    s->retired++;
    s->cv_done.notify_all();
}

// One chunk for every active request: returns 0 or a CUDA error code.
static int run_chunk(cosm_server *s, const std::vector<Request *> &act)
{
    const int n = (int)act.size();
    std::vector<InstView> views((size_t)n);
    struct Key { int storage, K, mode; };
    std::vector<Key> keys;
    std::vector<std::vector<BatchUnit>> per;
    std::vector<size_t> smem;
    std::vector<int> max_ec;
    for (int i = 0; i < n; ++i) {
        Request *r = act[(size_t)i];
        cosm_handle *h = r->h;
        h->seed = trial_seed(r->seed, r->trial);
        InstView v = inst_view(h);
        v.alpha_tab = h->d_alpha.p;
        v.alpha_base = 1;
        v.S = r->S;
        views[(size_t)i] = v;
        int c = -1;
        for (size_t k = 0; k < keys.size(); ++k)
            if (keys[k].storage == h->prm.storage && keys[k].K == h->K && keys[k].mode == h->mode) c = (int)k;
        if (c < 0) {
            keys.push_back(Key{h->prm.storage, h->K, h->mode});
            per.emplace_back();
            smem.push_back(0);
            max_ec.push_back(0);
            c = (int)keys.size() - 1;
        }
        smem[(size_t)c] = std::max(smem[(size_t)c], h->smem);
        for (int cc = 0; cc < h->C; ++cc) max_ec[(size_t)c] = std::max(max_ec[(size_t)c], h->off[cc + 1] - h->off[cc]);
        const int64_t s0 = r->pos + 1, s1 = std::min<int64_t>(r->S, r->pos + s->cfg.chunk_sweeps);
        const int32_t flags = (r->pos == 0 ? SEG_INIT : SEG_LOAD) | SEG_STORE | (s1 == r->S ? SEG_READOUT : 0);
        const int64_t tiles = (r->R + h->K - 1) / h->K;
        for (int64_t t = 0; t < tiles; ++t) per[(size_t)c].push_back(BatchUnit{i, (int32_t)t, flags, 0, s0, s1});
    }
    std::vector<BatchUnit> units;
    std::vector<int32_t> unit0;
    for (auto &u : per) {
        unit0.push_back((int32_t)units.size());
        units.insert(units.end(), u.begin(), u.end());
    }
    int rc;
    if ((rc = s->d_insts.ensure(views.size())) || (rc = s->d_units.ensure(units.size())) ||
        (rc = s->d_counters.ensure(keys.size())))
        return rc;
    CK(cudaMemcpyAsync(s->d_insts.p, views.data(), views.size() * sizeof(InstView), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d_units.p, units.data(), units.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(s->d_counters.p, 0, keys.size() * 4, s->st));
    for (size_t c = 0; c < keys.size(); ++c) {
        int T = s->cfg.threads ? s->cfg.threads : std::min(512, std::max(64, ((max_ec[c] + 1) / 2 + 31) / 32 * 32));
        int occ = batch_occupancy(keys[c].storage, keys[c].K, keys[c].mode, T, smem[c]);
        while (occ == 0 && T > 64) {
            T /= 2;
            occ = batch_occupancy(keys[c].storage, keys[c].K, keys[c].mode, T, smem[c]);
        }
        if (occ == 0) return fail(COSM_ERR_TOO_LARGE, "a serving tile does not fit on an SM");
        const int32_t cnt = (int32_t)per[c].size();
        const int grid = (int)std::min<int64_t>((int64_t)occ * s->num_sms, cnt);
        BatchArgs a{s->d_insts.p, s->d_units.p + unit0[c], cnt, s->d_counters.p + c};
        if (batch_launch(keys[c].storage, keys[c].K, keys[c].mode, grid, T, smem[c], a, s->st))
            return fail(COSM_ERR_CUDA, std::string("serving launch: ") + cudaGetErrorString(cudaGetLastError()));
        s->launches++;
    }
    CK(cudaStreamSynchronize(s->st));
    return COSM_OK;
}

static void worker_main(cosm_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request *> fresh;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop) break;
            while (!s->queue.empty() && (int64_t)s->active.size() + (int64_t)fresh.size() < s->cfg.max_active) {
                Request *r = s->queue.front();
                if (s->footprint + r->footprint > (size_t)s->cfg.memory_budget) break;  // in order
                s->queue.pop_front();
                s->footprint += r->footprint;
                s->peak_footprint = std::max(s->peak_footprint, s->footprint);
                r->status = RQ_RUNNING;
                r->t_admit = s->now();
                fresh.push_back(r);
            }
            if (s->active.empty() && fresh.empty()) {
                s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
                continue;
            }
        }
        for (Request *r : fresh) {
            const int rc = admit(s, r);
            std::lock_guard<std::mutex> lock(s->mu);
            if (rc) {
                r->error = rc;
                retire(s, r, RQ_EXHAUSTED);
            } else {
                s->active.push_back(r);
            }
        }
        std::vector<Request *> act;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            act = s->active;
            s->max_concurrent = std::max<int64_t>(s->max_concurrent, (int64_t)act.size());
        }
        if (act.empty()) continue;
        int rc;
        {
            NvtxRange range("cosm_server_chunk");
            rc = run_chunk(s, act);
        }
        std::vector<Request *> keep;
        for (Request *r : act) {
            if (rc) {
                std::lock_guard<std::mutex> lock(s->mu);
                r->error = rc;
                retire(s, r, RQ_EXHAUSTED);
                continue;
            }
            const int64_t s1 = std::min<int64_t>(r->S, r->pos + s->cfg.chunk_sweeps);
            r->updates += (int64_t)r->src.size() * (int64_t)r->R * (s1 - r->pos);
            r->pos = s1;
            bool done = false;
            int status = RQ_RUNNING;
            if (r->pos == r->S) {
                // the trial ended: best replica, and its spins when it improves
                int64_t cut = 0, energy = 0;
                int32_t rep = 0;
                int frc = launch_finalize(r->h, s->st);
                r->h->have_result = true;
                std::vector<int8_t> sp((size_t)r->n);
                if (!frc) frc = cosm_get_best(r->h, &cut, &energy, &rep, sp.data());
                if (frc) {
                    r->error = frc;
                    done = true;
                    status = RQ_EXHAUSTED;
                } else {
                    if (cut > r->best_cut) {
                        r->best_cut = cut;
                        r->energy = energy;
                        r->best_trial = r->trial;
                        r->best_replica = rep;
                        r->spins.swap(sp);
                    }
                    r->trial++;
                    r->pos = 0;
                    if (r->best_cut >= r->target) {
                        r->ttt = s->now() - r->t_submit;
                        done = true;
                        status = RQ_REACHED;
                    } else if (r->trial >= r->max_trials) {
                        done = true;
                        status = RQ_EXHAUSTED;
                    }
                }
            }
            std::lock_guard<std::mutex> lock(s->mu);
            if (done) retire(s, r, status);
            else keep.push_back(r);
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->active.swap(keep);
            s->chunks++;
        }
        s->cv_done.notify_all();
    }
}

extern "C" void cosm_server_default_config(cosm_server_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->memory_budget = (int64_t)8 << 30;
    c->max_active = 64;
    c->chunk_sweeps = 500;
    c->threads = 0;
}

extern "C" int cosm_server_create(const cosm_server_config *cfg, cosm_server **out)
{
    if (!cfg || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (cfg->memory_budget < 1 || cfg->max_active < 1 || cfg->chunk_sweeps < 1 || cfg->threads < 0 ||
        cfg->threads > 512)
        return fail(COSM_ERR_INVALID_ARG, "bad server configuration");
    *out = nullptr;
    cosm_server *s = new (std::nothrow) cosm_server();
    if (!s) return fail(COSM_ERR_NOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(COSM_ERR_CUDA, "server device setup failed");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return COSM_OK;
}

extern "C" void cosm_server_destroy(cosm_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) {
        if (kv.second->h) cosm_destroy(kv.second->h);
        delete kv.second;
    }
    s->d_insts.release();
    s->d_units.release();
    s->d_counters.release();
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

extern "C" int cosm_server_submit(cosm_server *s, const cosm_graph_desc *g, const cosm_params *p, int64_t sweeps,
                                  int32_t replicas, uint64_t seed, int64_t target_cut, int32_t max_trials,
                                  int64_t *id)
{
    if (!s || !g || !p || !id) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    if (!g->src || !g->dst || !g->w || g->n < 2 || g->n > kMaxVertices || g->m < 1 || g->m > ((int64_t)1 << 26))
        return fail(COSM_ERR_INVALID_ARG, "bad graph");
    if (sweeps < 1 || sweeps >= ((int64_t)1 << 31) || replicas < 1 || replicas >= (1 << 24) || max_trials < 1)
        return fail(COSM_ERR_INVALID_ARG, "bad sweeps, replicas or max_trials");
    if (int rc = single_only(g, p)) return rc;
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(COSM_ERR_NOMEM, "host allocation failed");
    r->n = g->n;
    r->src.assign(g->src, g->src + g->m);
    r->dst.assign(g->dst, g->dst + g->m);
    r->w.assign(g->w, g->w + g->m);
    if (g->color) {
        r->color.assign(g->color, g->color + g->m);
        r->n_colors = g->n_colors;
    }
    for (int k = 0; k < 3; ++k) r->dims[k] = g->dims[k];
    r->prm = *p;
    r->S = sweeps;
    r->R = replicas;
    r->seed = seed;
    r->target = target_cut;
    r->max_trials = max_trials;
    r->footprint = estimate_footprint(*r);
    if (r->footprint > (size_t)s->cfg.memory_budget) {
        delete r;
        return fail(COSM_ERR_TOO_LARGE, "request footprint exceeds the server's memory budget");
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->id = s->next_id++;
        r->t_submit = s->now();
        s->all[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_all();
    return COSM_OK;
}

static void fill_result(const Request *r, cosm_request_result *out)
{
    std::memset(out, 0, sizeof(*out));
    out->status = r->error ? r->error : r->status;
    out->trials = r->trial;
    out->best_cut = r->best_cut == LLONG_MIN ? 0 : r->best_cut;
    out->energy = r->energy;
    out->best_trial = r->best_trial;
    out->best_replica = r->best_replica;
    out->t_submit = r->t_submit;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
    out->ttt = r->ttt;
    out->updates = r->updates;
}

extern "C" int cosm_server_poll(cosm_server *s, int64_t id, cosm_request_result *out)
{
    if (!s || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(COSM_ERR_INVALID_ARG, "unknown request");
    fill_result(it->second, out);
    return COSM_OK;
}

extern "C" int cosm_server_wait(cosm_server *s, int64_t id, double timeout_s, cosm_request_result *out)
{
    if (!s || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(COSM_ERR_INVALID_ARG, "unknown request");
    Request *r = it->second;
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->status < RQ_REACHED)
        if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout) break;
    fill_result(r, out);
    if (r->status < RQ_REACHED) return fail(COSM_ERR_TIMEOUT, "request not finished within the timeout");
    return COSM_OK;
}

extern "C" int cosm_server_get_spins(cosm_server *s, int64_t id, int8_t *spins)
{
    if (!s || !spins) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(COSM_ERR_INVALID_ARG, "unknown request");
    const Request *r = it->second;
    if (r->status < RQ_REACHED || r->spins.empty()) return fail(COSM_ERR_STATE, "request has no result yet");
    std::memcpy(spins, r->spins.data(), r->spins.size());
    return COSM_OK;
}

extern "C" int cosm_server_stats(cosm_server *s, int64_t out[8])
{
    if (!s || !out) return fail(COSM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = (int64_t)s->queue.size();
    out[1] = (int64_t)s->active.size();
    out[2] = s->retired;
    out[3] = s->chunks;
    out[4] = s->launches;
    out[5] = s->max_concurrent;
    out[6] = (int64_t)s->peak_footprint;
    out[7] = (int64_t)s->footprint;
    return COSM_OK;
}
