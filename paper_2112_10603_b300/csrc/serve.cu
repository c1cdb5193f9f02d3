// Multi-user view-interpolation server (fvv_serve_*): continuous batching of
// viewpoint requests of mixed resolution on one GPU.
//
// The paper's edge server decouples its load from the number of users by
// rendering dense views once per instant and streaming them (Sec. 3.2); it
// organises its modules around FIFO data channels with PUT/GET (supplement S.1,
// "4U" model).  This server keeps that structure — a request channel in, a
// completion channel out — around the VINet forward:
//  * per resolution, `slots` interpolator handles, each with its own CUDA stream,
//    so a batch can start while others are still on the device;
//  * a scheduler thread takes up to max_batch queued requests of one resolution
//    whenever one of its slots is free (requests that arrive meanwhile simply wait
//    for the next free slot: continuous batching), groups them by camera pair and
//    runs them as ONE batched forward (fvv_interp_run_batch: one graph launch);
//  * latest-wins per user: a new request from a user replaces that user's request
//    still waiting in the queue (the old ticket then polls FVV_ESUPERSEDED);
//  * admission by HBM budget: every admitted request holds one view-sized output
//    buffer from a pool sized from the budget left after the slots' workspaces;
//    when the pool is empty, submit returns FVV_EBUSY;
//  * a slot remembers which frame instant its pyramid/ContextNet features belong
//    to and skips recomputing them for the next batch of the same instant;
//  * completion is signalled by a host callback on the slot stream, which stamps
//    the latency (submit -> views in their output buffers);
//  * dense mode (dense_levels = n): per instant the fixed set t = k / 2^n of every
//    pair is rendered once (batches of whole pairs) into one of two stores; requests
//    snap t to that grid and are answered from the store of the newest frames, so
//    the GPU work per instant does not depend on the number of users;  with
//    dense_immediate every request is answered at once from the newest complete set,
//    whatever instant it shows, and the server records how old that content is
//    (time since its frames were set, and instants behind the newest frames).
// With cfg.fake_ms_per_view > 0 nothing touches the GPU: a batch "runs" for
// fake_ms_per_view x views milliseconds on the scheduler thread, so the queueing,
// supersession, admission and latency logic can be tested on any machine.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "interp.h"

namespace fvv {
namespace {

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_SUPERSEDED = 3, RQ_FAILED = 4 };

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int user = 0, pair = 0, res = 0, state = RQ_QUEUED, buf = -1;
    float t = 0.f;
    double t_submit = 0, t_done = 0;
    int k = 0;                   // dense mode: snapped index, t = k / 2^n
    const float *out = nullptr;  // dense mode: the view (store or camera frame)
};

struct Batch;

struct Slot {
    fvv_interp *h = nullptr;
    cudaStream_t st = nullptr;
    float *out = nullptr;       // max_batch views
    bool busy = false;
    long long frames_id = -1;   // instant whose features are in the workspace
};

struct Res {
    int H = 0, W = 0;
    std::vector<Slot> slots;
    std::vector<float *> pool; // view-sized output buffers
    std::vector<int> free_bufs;
    std::deque<uint64_t> queue;
    std::vector<const float *> cams;
    long long frames_id = -1;
    // dense mode: two stores of n_pairs x (2^n - 1) views
    float *dstore[2] = {nullptr, nullptr};
    long long d_inst[2] = {-1, -1};  // complete instant held by each store
    int d_cur = -1;                  // store of the newest complete instant
    long long d_render = -1;         // instant being rendered (-1: none)
    double frames_t = 0;             // when the newest frames were set
    double d_time[2] = {0, 0};       // when the frames of each store's instant were set
    double d_render_t = 0;           // when the frames being rendered were set
    int d_buf = 0;                   // store it renders into
    std::vector<const float *> d_cams;
    int d_next_pair = 0, d_pairs_done = 0;
    std::vector<uint64_t> d_waiting; // tickets waiting for the newest frames' views
};

} // namespace
} // namespace fvv

using namespace fvv;

struct fvv_server {
    fvv_serve_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::thread sched;
    bool stop = false;
    std::vector<Res> res;
    std::unordered_map<uint64_t, Request> reqs;
    std::unordered_map<int, uint64_t> queued_of_user; // user -> ticket still queued
    uint64_t next_ticket = 1;
    fvv_serve_stats st{};
    int nd = 0;          // dense mode: views per pair (2^n - 1), 0 = on-demand mode
    int n_pairs = 0;
    std::vector<double> lat; // completed latencies (ms)
    std::vector<double> age; // dense mode: age of the answered content (ms since its frames were set)
    std::vector<long long> stale; // dense mode: instants between the answered set and the newest frames
    size_t dev_bytes = 0;
};

namespace fvv {
namespace {

struct Batch {
    fvv_server *s;
    int res, slot;
    std::vector<uint64_t> tickets;
};

void finish_batch(Batch *b, bool ok) {
    fvv_server *s = b->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        double t = now_ms();
        for (uint64_t tk : b->tickets) {
            auto it = s->reqs.find(tk);
            if (it == s->reqs.end()) continue;
            Request &r = it->second;
            r.state = ok ? RQ_DONE : RQ_FAILED;
            r.t_done = t;
            if (ok) {
                s->st.completed++;
                s->lat.push_back(t - r.t_submit);
            } else {
                s->st.failed++;
            }
        }
        s->st.batches++;
        s->st.batched_views += b->tickets.size();
        s->res[b->res].slots[b->slot].busy = false;
    }
    s->cv.notify_all();
    delete b;
}

void CUDART_CB batch_done_cb(void *p) { finish_batch(static_cast<Batch *>(p), true); }

// ---- dense mode ------------------------------------------------------------
const float *dense_ptr(const fvv_server *s, const Res &R, int store, int pair, int k) {
    const size_t view = (size_t)R.H * R.W * 3;
    return R.dstore[store] + ((size_t)pair * s->nd + (k - 1)) * view;
}

// Answer a dense request from the newest complete store (lock held).
void dense_answer(fvv_server *s, Request &r, double t) {
    Res &R = s->res[r.res];
    r.out = dense_ptr(s, R, R.d_cur, r.pair, r.k);
    r.state = RQ_DONE;
    r.t_done = t;
    s->st.completed++;
    s->lat.push_back(t - r.t_submit);
    s->age.push_back(t - R.d_time[R.d_cur]);
    s->stale.push_back(R.frames_id - R.d_inst[R.d_cur]);
}

struct RenderBatch {
    fvv_server *s;
    int res, slot, n_pairs;
    long long instant;
    bool ok;
};

void finish_render(RenderBatch *b) {
    fvv_server *s = b->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Res &R = s->res[b->res];
        R.slots[b->slot].busy = false;
        s->st.batches++;
        s->st.batched_views += (long long)b->n_pairs * s->nd;
        if (!b->ok) {
            s->st.failed++;
            R.d_render = -1; // retried by the scheduler on the newest frames
        } else if (b->instant == R.d_render && (R.d_pairs_done += b->n_pairs) == s->n_pairs) {
            R.d_inst[R.d_buf] = R.d_render;
            R.d_time[R.d_buf] = R.d_render_t;
            R.d_cur = R.d_buf;
            R.d_render = -1;
            s->st.dense_instants++;
            // every waiting request is answered by the first set completed after it
            // arrived, even when newer frames have been set meanwhile (frames may
            // arrive faster than a whole set renders: no request starves)
            double t = now_ms();
            for (uint64_t tk : R.d_waiting) {
                auto it = s->reqs.find(tk);
                if (it != s->reqs.end() && it->second.state == RQ_QUEUED) {
                    auto q = s->queued_of_user.find(it->second.user);
                    if (q != s->queued_of_user.end() && q->second == tk) s->queued_of_user.erase(q);
                    dense_answer(s, it->second, t);
                }
            }
            R.d_waiting.clear();
        }
    }
    s->cv.notify_all();
    delete b;
}

void CUDART_CB render_done_cb(void *p) { finish_render(static_cast<RenderBatch *>(p)); }

// Render pairs [p0, p0 + np) of instant `inst` on a free slot (lock not held).
void launch_render(fvv_server *s, int r, int slot, int p0, int np, long long inst, std::vector<const float *> cams,
                   float *store) {
    Res &R = s->res[r];
    Slot &sl = R.slots[slot];
    RenderBatch *b = new RenderBatch{s, r, slot, np, inst, true};
    if (s->cfg.fake_ms_per_view > 0) {
        std::this_thread::sleep_for(
            std::chrono::microseconds((long long)(1000.0 * s->cfg.fake_ms_per_view * np * s->nd)));
        finish_render(b);
        return;
    }
    const int nd = s->nd, levels = s->cfg.dense_levels;
    std::vector<int> pair_left(np), offs(np + 1);
    std::vector<float> t((size_t)np * nd);
    for (int i = 0; i < np; ++i) {
        pair_left[i] = p0 + i;
        offs[i] = i * nd;
        for (int k = 1; k <= nd; ++k) t[(size_t)i * nd + k - 1] = (float)k / (float)(1 << levels);
    }
    offs[np] = np * nd;
    sl.h->skip_cams = sl.frames_id == inst ? 1 : 0;
    const size_t view = (size_t)R.H * R.W * 3;
    int rc = fvv_interp_run_batch(sl.h, cams.data(), (int)cams.size(), pair_left.data(), offs.data(), t.data(), np,
                                  store + (size_t)p0 * nd * view, sl.st);
    sl.h->skip_cams = 0;
    sl.frames_id = rc == FVV_OK ? inst : -1;
    if (rc == FVV_OK && cudaLaunchHostFunc(sl.st, render_done_cb, b) != cudaSuccess) rc = FVV_ECUDA;
    if (rc != FVV_OK) {
        b->ok = false;
        finish_render(b);
    }
}

// Launch one batch on a free slot (called without the lock held).
int launch_batch(fvv_server *s, Batch *b, const std::vector<Request> &rq, const std::vector<const float *> &cams,
                 long long frames_id) {
    Res &R = s->res[b->res];
    Slot &sl = R.slots[b->slot];
    const int n = (int)rq.size();
    if (s->cfg.fake_ms_per_view > 0) {
        std::this_thread::sleep_for(std::chrono::microseconds((long long)(1000.0 * s->cfg.fake_ms_per_view * n)));
        finish_batch(b, true);
        return FVV_OK;
    }
    // group by pair: rq is sorted by pair already
    std::vector<int> pair_left, offs{0};
    std::vector<float> t(n);
    for (int i = 0; i < n; ++i) {
        if (pair_left.empty() || pair_left.back() != rq[i].pair) {
            if (!pair_left.empty()) offs.push_back(i);
            pair_left.push_back(rq[i].pair);
        }
        t[i] = rq[i].t;
    }
    offs.push_back(n);
    sl.h->skip_cams = sl.frames_id == frames_id ? 1 : 0;
    int rc = fvv_interp_run_batch(sl.h, cams.data(), (int)cams.size(), pair_left.data(), offs.data(), t.data(),
                                  (int)pair_left.size(), sl.out, sl.st);
    sl.h->skip_cams = 0;
    if (rc == FVV_OK) {
        sl.frames_id = frames_id;
        const size_t view = (size_t)R.H * R.W * 3;
        for (int i = 0; i < n && rc == FVV_OK; ++i)
            if (cudaMemcpyAsync(R.pool[rq[i].buf], sl.out + i * view, view * 4, cudaMemcpyDeviceToDevice, sl.st) !=
                cudaSuccess)
                rc = FVV_ECUDA;
    }
    if (rc == FVV_OK && cudaLaunchHostFunc(sl.st, batch_done_cb, b) != cudaSuccess) rc = FVV_ECUDA;
    if (rc != FVV_OK) {
        sl.frames_id = -1;
        finish_batch(b, false);
    }
    return rc;
}

void scheduler(fvv_server *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool launched = false;
        for (int r = 0; r < (int)s->res.size() && !s->stop; ++r) {
            Res &R = s->res[r];
            if (s->nd > 0) {
                // start rendering the newest frames once the previous render is over
                if (R.d_render < 0 && R.frames_id >= 0 && !R.cams.empty() &&
                    (R.d_cur < 0 || R.d_inst[R.d_cur] != R.frames_id)) {
                    bool idle = true;
                    for (auto &sl : R.slots) idle = idle && !sl.busy;
                    if (idle) {
                        R.d_render = R.frames_id;
                        R.d_render_t = R.frames_t;
                        R.d_buf = R.d_cur == 0 ? 1 : 0;
                        R.d_inst[R.d_buf] = -1;
                        R.d_cams = R.cams;
                        R.d_next_pair = 0;
                        R.d_pairs_done = 0;
                    }
                }
                while (R.d_render >= 0 && R.d_next_pair < s->n_pairs && !s->stop) {
                    int k = -1;
                    for (int j = 0; j < (int)R.slots.size(); ++j)
                        if (!R.slots[j].busy) { k = j; break; }
                    if (k < 0) break;
                    const int per = std::max(1, s->cfg.max_batch / s->nd);
                    const int p0 = R.d_next_pair, np = std::min(per, s->n_pairs - p0);
                    R.d_next_pair += np;
                    R.slots[k].busy = true;
                    std::vector<const float *> cams = R.d_cams;
                    long long inst = R.d_render;
                    float *store = R.dstore[R.d_buf];
                    lk.unlock();
                    launch_render(s, r, k, p0, np, inst, cams, store);
                    lk.lock();
                    launched = true;
                }
                continue;
            }
            int free_slot = -1;
            for (int k = 0; k < (int)R.slots.size(); ++k)
                if (!R.slots[k].busy) { free_slot = k; break; }
            if (free_slot < 0 || R.queue.empty() || R.cams.empty()) continue;
            // take up to max_batch requests, oldest first
            Batch *b = new Batch{s, r, free_slot, {}};
            std::vector<Request> rq;
            while (!R.queue.empty() && (int)b->tickets.size() < s->cfg.max_batch) {
                uint64_t tk = R.queue.front();
                R.queue.pop_front();
                auto it = s->reqs.find(tk);
                if (it == s->reqs.end() || it->second.state != RQ_QUEUED) continue;
                it->second.state = RQ_RUNNING;
                auto q = s->queued_of_user.find(it->second.user);
                if (q != s->queued_of_user.end() && q->second == tk) s->queued_of_user.erase(q);
                b->tickets.push_back(tk);
            }
            if (b->tickets.empty()) { delete b; continue; }
            std::sort(b->tickets.begin(), b->tickets.end(),
                      [&](uint64_t a, uint64_t c) { return s->reqs[a].pair < s->reqs[c].pair; });
            for (uint64_t tk : b->tickets) rq.push_back(s->reqs[tk]);
            R.slots[free_slot].busy = true;
            std::vector<const float *> cams = R.cams;
            long long fid = R.frames_id;
            lk.unlock();
            launch_batch(s, b, rq, cams, fid);
            lk.lock();
            launched = true;
        }
        if (!launched) s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

} // namespace
} // namespace fvv

extern "C" {

void fvv_serve_default_cfg(fvv_serve_cfg *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->precision = FVV_BF16;
    c->n_res = 1;
    c->res_h[0] = 1080;
    c->res_w[0] = 1920;
    c->n_cams = 9;
    c->slots_per_res = 2;
    c->max_batch = 8;
    c->hbm_budget = 0;
    c->pool_views = 64;
    c->fake_ms_per_view = 0.0;
}

int fvv_serve_create(const float *weights, size_t n_floats, const fvv_serve_cfg *cfg, fvv_server **out) {
    clear_error();
    if (!cfg || !out || (!weights && cfg->fake_ms_per_view <= 0)) { set_error("NULL argument"); return FVV_EINVAL; }
    *out = nullptr;
    if (cfg->n_res < 1 || cfg->n_res > FVV_SERVE_MAX_RES || cfg->slots_per_res < 1 || cfg->max_batch < 1 ||
        cfg->n_cams < 2 || cfg->pool_views < 1) {
        set_error("bad server configuration"); return FVV_EINVAL;
    }
    if (cfg->precision != FVV_FP32 && cfg->precision != FVV_BF16 && cfg->precision != FVV_FP8) {
        set_error("server precision must be FVV_FP32, FVV_BF16 or FVV_FP8"); return FVV_EINVAL;
    }
    if (cfg->dense_levels < 0 || cfg->dense_levels > 8 ||
        (cfg->dense_levels > 0 && (1 << cfg->dense_levels) - 1 > cfg->max_batch)) {
        set_error("dense_levels must give 2^n - 1 <= max_batch views per pair"); return FVV_EINVAL;
    }
    fvv_server *s = new fvv_server();
    s->cfg = *cfg;
    s->nd = cfg->dense_levels > 0 ? (1 << cfg->dense_levels) - 1 : 0;
    s->n_pairs = cfg->n_cams - 1;
    s->res.resize(cfg->n_res);
    int rc = FVV_OK;
    for (int r = 0; r < cfg->n_res && rc == FVV_OK; ++r) {
        Res &R = s->res[r];
        R.H = cfg->res_h[r];
        R.W = cfg->res_w[r];
        R.slots.resize(cfg->slots_per_res);
        if (cfg->fake_ms_per_view > 0) {
            R.pool.assign(cfg->pool_views, nullptr);
        } else {
            fvv_opts o;
            fvv_default_opts(&o);
            o.precision = cfg->precision;
            o.max_views = cfg->max_batch;
            o.max_cams = cfg->n_cams;
            for (auto &sl : R.slots) {
                if ((rc = fvv_interp_create(weights, n_floats, R.H, R.W, &o, &sl.h)) != FVV_OK) break;
                if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaMalloc(&sl.out, (size_t)cfg->max_batch * R.H * R.W * 3 * 4) != cudaSuccess) {
                    set_error("server: slot allocation failed"); rc = FVV_ENOMEM; break;
                }
                s->dev_bytes += fvv_interp_device_bytes(sl.h) + (size_t)cfg->max_batch * R.H * R.W * 12;
            }
        }
    }
    // output pool: pool_views per resolution, cut to what the HBM budget leaves
    for (int r = 0; r < cfg->n_res && rc == FVV_OK && cfg->fake_ms_per_view <= 0 && s->nd == 0; ++r) {
        Res &R = s->res[r];
        size_t view = (size_t)R.H * R.W * 12;
        int n = cfg->pool_views;
        if (cfg->hbm_budget > 0) {
            size_t left = cfg->hbm_budget > s->dev_bytes ? cfg->hbm_budget - s->dev_bytes : 0;
            size_t per_res = left / (size_t)(cfg->n_res - r);
            n = (int)std::min<size_t>((size_t)n, per_res / view);
        }
        if (n < 1) { set_error("HBM budget leaves no output buffer at %dx%d", R.H, R.W); rc = FVV_EBUSY; break; }
        R.pool.assign(n, nullptr);
        for (auto &p : R.pool)
            if (cudaMalloc(&p, view) != cudaSuccess) { set_error("server: pool allocation failed"); rc = FVV_ENOMEM; break; }
        s->dev_bytes += (size_t)n * view;
    }
    // dense stores: two per resolution (fake mode: distinct never-dereferenced bases)
    for (int r = 0; r < cfg->n_res && rc == FVV_OK && s->nd > 0; ++r) {
        Res &R = s->res[r];
        const size_t bytes = (size_t)s->n_pairs * s->nd * R.H * R.W * 12;
        for (int b = 0; b < 2 && rc == FVV_OK; ++b) {
            if (cfg->fake_ms_per_view > 0) {
                R.dstore[b] = reinterpret_cast<float *>((uintptr_t)(r * 2 + b + 1) << 40);
            } else if (cudaMalloc(&R.dstore[b], bytes) != cudaSuccess) {
                R.dstore[b] = nullptr;
                set_error("server: dense store allocation failed"); rc = FVV_ENOMEM;
            } else {
                s->dev_bytes += bytes;
            }
        }
    }
    if (rc != FVV_OK) { fvv_serve_destroy(s); return rc; }
    for (auto &R : s->res)
        for (int i = (int)R.pool.size() - 1; i >= 0; --i) R.free_bufs.push_back(i);
    s->sched = std::thread(scheduler, s);
    *out = s;
    return FVV_OK;
}

int fvv_serve_calibrate_fp8(fvv_server *s, int res_id, const float *frames, int n_pairs) {
    clear_error();
    if (!s || !frames || res_id < 0 || res_id >= (int)s->res.size() || n_pairs < 1) {
        set_error("bad arguments"); return FVV_EINVAL;
    }
    if (s->cfg.precision != FVV_FP8) { set_error("the server does not run FP8"); return FVV_EINVAL; }
    if (s->cfg.fake_ms_per_view > 0) return FVV_OK;
    Res &R = s->res[res_id];
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &sl : R.slots)
            if (sl.busy) { set_error("calibrate before the first frames of this resolution"); return FVV_EBUSY; }
        for (auto &sl : R.slots) sl.busy = true; // the scheduler keeps off these slots meanwhile
    }
    int rc = FVV_OK;
    for (auto &sl : R.slots)
        if ((rc = fvv_calibrate_fp8(sl.h, frames, n_pairs, sl.st)) != FVV_OK) break;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &sl : R.slots) sl.busy = false;
    }
    s->cv.notify_all();
    return rc;
}

int fvv_serve_set_frames(fvv_server *s, int64_t instant, int res_id, const float *const *cams_dev) {
    clear_error();
    if (!s || !cams_dev || res_id < 0 || res_id >= (int)s->res.size()) { set_error("bad arguments"); return FVV_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    Res &R = s->res[res_id];
    R.cams.assign(cams_dev, cams_dev + s->cfg.n_cams);
    R.frames_id = instant;
    R.frames_t = now_ms();
    s->cv.notify_all();
    return FVV_OK;
}

int fvv_serve_submit(fvv_server *s, int user, int pair, float t, int res_id, uint64_t *ticket) {
    clear_error();
    if (!s || !ticket || res_id < 0 || res_id >= (int)s->res.size() || pair < 0 || pair + 1 >= s->cfg.n_cams ||
        !(t >= 0.f && t <= 1.f)) {
        set_error("bad request"); return FVV_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Res &R = s->res[res_id];
    s->st.submitted++;
    if (s->nd > 0) {
        if (R.cams.empty()) { set_error("no frames set for this resolution"); return FVV_EINVAL; }
        // latest wins: the user's request still waiting is replaced
        auto q = s->queued_of_user.find(user);
        if (q != s->queued_of_user.end()) {
            Request &old = s->reqs[q->second];
            if (old.state == RQ_QUEUED) {
                old.state = RQ_SUPERSEDED;
                old.t_done = now_ms();
                s->st.superseded++;
            }
            s->queued_of_user.erase(q);
        }
        const int full = 1 << s->cfg.dense_levels;
        Request r;
        r.user = user; r.pair = pair; r.res = res_id; r.t = t; r.t_submit = now_ms();
        r.k = std::min(full, std::max(0, (int)std::lround(t * full)));
        const uint64_t tk = s->next_ticket++;
        if (r.k == 0 || r.k == full) {
            // a camera: its own frame
            r.out = R.cams[r.k == 0 ? pair : pair + 1];
            r.state = RQ_DONE;
            r.t_done = r.t_submit;
            s->st.completed++;
            s->lat.push_back(0.0);
            s->age.push_back(r.t_submit - R.frames_t);
            s->stale.push_back(0);
            s->reqs[tk] = r;
        } else if (R.d_cur >= 0 && (R.d_inst[R.d_cur] == R.frames_id || s->cfg.dense_immediate)) {
            s->reqs[tk] = r;
            dense_answer(s, s->reqs[tk], now_ms());
        } else {
            s->reqs[tk] = r;
            R.d_waiting.push_back(tk);
            s->queued_of_user[user] = tk;
        }
        *ticket = tk;
        s->cv.notify_all();
        return FVV_OK;
    }
    // latest wins: the user's request still waiting is replaced (its buffer reused)
    int buf = -1;
    auto q = s->queued_of_user.find(user);
    if (q != s->queued_of_user.end()) {
        Request &old = s->reqs[q->second];
        if (old.state == RQ_QUEUED) {
            old.state = RQ_SUPERSEDED;
            old.t_done = now_ms();
            s->st.superseded++;
            if (old.res == res_id) buf = old.buf;
            else s->res[old.res].free_bufs.push_back(old.buf);
            old.buf = -1;
        }
        s->queued_of_user.erase(q);
    }
    if (buf < 0) {
        if (R.free_bufs.empty()) { s->st.rejected++; set_error("admission refused: output pool (HBM budget) full"); return FVV_EBUSY; }
        buf = R.free_bufs.back();
        R.free_bufs.pop_back();
    }
    uint64_t tk = s->next_ticket++;
    Request r;
    r.user = user; r.pair = pair; r.res = res_id; r.t = t; r.buf = buf; r.t_submit = now_ms();
    s->reqs[tk] = r;
    R.queue.push_back(tk);
    s->queued_of_user[user] = tk;
    *ticket = tk;
    s->cv.notify_all();
    return FVV_OK;
}

int fvv_serve_poll(fvv_server *s, uint64_t ticket, const float **out_dev, double *latency_ms) {
    clear_error();
    if (!s) { set_error("NULL server"); return FVV_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket"); return FVV_ENOTFOUND; }
    Request &r = it->second;
    switch (r.state) {
    case RQ_DONE:
        if (out_dev) *out_dev = s->nd > 0 ? r.out : (r.buf >= 0 ? s->res[r.res].pool[r.buf] : nullptr);
        if (latency_ms) *latency_ms = r.t_done - r.t_submit;
        return 0;
    case RQ_SUPERSEDED: set_error("superseded by a newer request of the same user"); return FVV_ESUPERSEDED;
    case RQ_FAILED: set_error("the batch holding this request failed"); return FVV_ECUDA;
    default: return 1;
    }
}

int fvv_serve_release(fvv_server *s, uint64_t ticket) {
    clear_error();
    if (!s) { set_error("NULL server"); return FVV_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket"); return FVV_ENOTFOUND; }
    Request &r = it->second;
    if (r.state == RQ_QUEUED || r.state == RQ_RUNNING) { set_error("request still pending"); return 1; }
    if (r.buf >= 0) s->res[r.res].free_bufs.push_back(r.buf);
    s->reqs.erase(it);
    return FVV_OK;
}

int fvv_serve_stats_get(fvv_server *s, fvv_serve_stats *out) {
    clear_error();
    if (!s || !out) { set_error("NULL argument"); return FVV_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    std::vector<double> l = s->lat;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.empty() ? 0.0 : l.back();
    l = s->age;
    std::sort(l.begin(), l.end());
    out->age_p50_ms = pct(0.50);
    out->age_p99_ms = pct(0.99);
    double st_sum = 0;
    long long st_max = 0;
    for (long long v : s->stale) { st_sum += (double)v; st_max = std::max(st_max, v); }
    out->stale_mean = s->stale.empty() ? 0.0 : st_sum / (double)s->stale.size();
    out->stale_max = st_max;
    out->device_bytes = s->dev_bytes;
    out->queued = 0;
    for (auto &R : s->res) out->queued += (long long)R.queue.size() + (long long)R.d_waiting.size();
    return FVV_OK;
}

void fvv_serve_destroy(fvv_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();
    if (s->cfg.fake_ms_per_view <= 0) {
        for (auto &R : s->res) {
            for (auto &sl : R.slots) {
                if (sl.st) cudaStreamSynchronize(sl.st); // host callbacks of in-flight batches run first
                if (sl.st) cudaStreamDestroy(sl.st);
                if (sl.out) cudaFree(sl.out);
                fvv_interp_destroy(sl.h);
            }
            for (float *p : R.pool) if (p) cudaFree(p);
            for (float *p : R.dstore) if (p) cudaFree(p);
        }
    }
    delete s;
}

} // extern "C"
