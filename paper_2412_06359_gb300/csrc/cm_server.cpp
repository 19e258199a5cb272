// cm_server.cpp -- serving: continuous batching of loss + gradient requests
// from many event streams on one GPU.
//
// The server reserves its whole HBM budget once (one cudaMalloc at creation)
// and carves it with a first-fit pool: per client stream a resident state (the
// window's scratch -- images of warped events, flow, reduction buffers -- plus
// inverse depth, gradients and an event buffer that grows with the largest
// request seen), and per lane a batch plan.  A scheduler thread forms batches
// continuously: queued requests whose stream is not already on the GPU are
// admitted while a lane is free and their state fits the budget (idle streams'
// state is evicted least-recently-used first when it does not); each batch is
// copied in, evaluated by its lane's plan (one CUDA graph), and copied out on
// the lane's own CUDA stream, so batches on different lanes overlap on the
// device.  Requests arriving while others run are taken into the next batch as
// soon as a lane and memory free up.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <unordered_set>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cm.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// first-fit allocator over [0, size) with coalescing of free neighbours
class Pool {
public:
    void init(size_t size)
    {
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
        size_ = size;
    }
    static constexpr size_t kNone = ~(size_t)0;
    size_t alloc(size_t n)
    {
        n = up256(n ? n : 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            used_ += n;
            if (used_ > peak_) peak_ = used_;
            return off;
        }
        return kNone;
    }
    void release(size_t off, size_t n)
    {
        n = up256(n ? n : 256);
        used_ -= n;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0, size_ = 0;
};

struct StreamState {
    int32_t id = 0;
    int32_t W = 0, H = 0;
    size_t fixed_off = Pool::kNone, fixed_bytes = 0;  // scratch, inverse depth, its gradient, small values
    size_t ev_off = Pool::kNone, ev_cap = 0, ev_bytes = 0;
    size_t o_scratch = 0, o_rho = 0, o_drho = 0, o_small = 0;
    bool busy = false;
    uint64_t last_use = 0;
};

struct Request {
    cm_request r;
    double t_submit = 0, t_start = 0, t_done = 0;
    int32_t status = CM_OK;
    int32_t batch_size = 0;
    bool done = false;
};

struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    cm_batch* plan = nullptr;
    size_t plan_off = Pool::kNone, plan_bytes = 0;
    std::vector<uint64_t> tickets;
    bool busy = false;
};

bool request_ok(const cm_request* q)
{
    if (!q) return false;
    const cm_camera& c = q->cam;
    if (c.width < 2 || c.height < 2 || c.width > 32767 || c.height > 32767) return false;
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f)) return false;
    if (q->n < 0 || (q->n > 0 && (!q->x || !q->y || !q->t || !q->p))) return false;
    if (!(q->t1 - q->t0 > 0.0f)) return false;
    if (!q->inv_depth || !q->ego6 || !q->loss_out) return false;
    return true;
}

}  // namespace

struct cm_server {
    cm_server_cfg cfg{};
    cm_loss_cfg lcfg{};
    char* dev = nullptr;
    Pool pool;
    std::mutex mu;
    std::condition_variable cv;       // wakes the scheduler
    std::condition_variable done_cv;  // wakes waiters
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::unordered_map<int32_t, StreamState> streams;
    std::vector<Lane> lanes;
    uint64_t clock = 0;
    cm_server_stats st{};

    char* at(size_t off) const { return dev + off; }

    size_t fixed_bytes_for(int W, int H, size_t* o_scratch, size_t* o_rho, size_t* o_drho, size_t* o_small)
    {
        cm_camera c{W, H, 1.0f, 1.0f, 0.0f, 0.0f};
        size_t sb = 0;
        cm_window_scratch_query(&c, &lcfg, &sb);
        const size_t HW = (size_t)W * H;
        size_t o = 0;
        *o_scratch = o;
        o = up256(o + sb);
        *o_rho = o;
        o = up256(o + HW * 4);
        *o_drho = o;
        o = up256(o + HW * 4);
        *o_small = o;  // ego[6], dego[6], loss, dloss
        o = up256(o + 16 * 4);
        return o;
    }

    static size_t events_bytes(size_t cap) { return up256(2 * cap) * 2 + up256(4 * cap) + up256(cap); }

    // free an idle stream's memory (least recently used first) until `need`
    // bytes could fit; returns false when nothing more can be evicted
    bool evict_one(int32_t keep)
    {
        StreamState* victim = nullptr;
        for (auto& kv : streams) {
            StreamState& s = kv.second;
            if (s.busy || s.id == keep || (s.fixed_off == Pool::kNone && s.ev_off == Pool::kNone)) continue;
            if (!victim || s.last_use < victim->last_use) victim = &s;
        }
        if (!victim) return false;
        if (victim->fixed_off != Pool::kNone) pool.release(victim->fixed_off, victim->fixed_bytes);
        if (victim->ev_off != Pool::kNone) pool.release(victim->ev_off, victim->ev_bytes);
        victim->fixed_off = victim->ev_off = Pool::kNone;
        victim->ev_cap = 0;
        st.evictions += 1;
        return true;
    }

    size_t alloc_evicting(size_t n, int32_t keep)
    {
        for (;;) {
            const size_t off = pool.alloc(n);
            if (off != Pool::kNone) return off;
            if (!evict_one(keep)) return Pool::kNone;
        }
    }

    // Run every lane's plan once on an empty 2x2 window, so that each lane
    // captures its graph now instead of inside the first requests' latency
    // (the lanes' schedule takes every window slot in one group: the graph
    // stays valid for any later mix of windows).
    int warm_lanes()
    {
        const cm_camera cam{2, 2, 1.0f, 1.0f, 0.5f, 0.5f};
        size_t sb = 0;
        if (cm_window_scratch_query(&cam, &lcfg, &sb) != CM_OK) return CM_ECUDA;
        const size_t bytes = up256(sb) + 256;
        const size_t off = pool.alloc(bytes);
        if (off == Pool::kNone) return CM_ENOMEM;
        char* m = at(off);
        float* small = reinterpret_cast<float*>(m + up256(sb));  // rho[4], ego[6], dego[6], loss, dloss
        int rc = cudaMemsetAsync(m, 0, bytes, lanes[0].s) == cudaSuccess &&
                         cudaStreamSynchronize(lanes[0].s) == cudaSuccess
                     ? CM_OK
                     : CM_ECUDA;
        cm_window w;
        std::memset(&w, 0, sizeof(w));
        w.cam = cam;
        w.ev = cm_events{nullptr, nullptr, nullptr, nullptr, 0, 0.0f, 1.0f};
        w.inv_depth = small;
        w.ego6 = small + 4;
        w.dego6 = small + 10;
        w.loss_out = small + 16;
        w.dloss = small + 17;
        w.dt_window = 1.0f;
        w.scratch = m;
        for (Lane& L : lanes) {
            if (rc) break;
            if ((rc = cm_batch_set_windows(L.plan, &w, 1))) break;
            if ((rc = cm_batch_run(L.plan, L.s))) break;
            if (cudaStreamSynchronize(L.s) != cudaSuccess) rc = CM_ECUDA;
        }
        pool.release(off, bytes);
        return rc;
    }

    // make the stream's resident state fit request q; false when memory is short now
    bool ensure_state(StreamState& s, const cm_request& q)
    {
        if (s.fixed_off != Pool::kNone && (s.W != q.cam.width || s.H != q.cam.height)) {
            pool.release(s.fixed_off, s.fixed_bytes);
            s.fixed_off = Pool::kNone;
        }
        if (s.fixed_off == Pool::kNone) {
            const size_t b = fixed_bytes_for(q.cam.width, q.cam.height, &s.o_scratch, &s.o_rho, &s.o_drho, &s.o_small);
            const size_t off = alloc_evicting(b, s.id);
            if (off == Pool::kNone) return false;
            s.fixed_off = off;
            s.fixed_bytes = b;
            s.W = q.cam.width;
            s.H = q.cam.height;
        }
        if (s.ev_off == Pool::kNone || s.ev_cap < (size_t)q.n) {
            if (s.ev_off != Pool::kNone) pool.release(s.ev_off, s.ev_bytes);
            s.ev_off = Pool::kNone;
            size_t cap = 1024;
            while (cap < (size_t)q.n) cap += cap / 2;
            const size_t b = events_bytes(cap);
            const size_t off = alloc_evicting(b, s.id);
            if (off == Pool::kNone) {
                s.ev_cap = 0;
                return false;
            }
            s.ev_off = off;
            s.ev_bytes = b;
            s.ev_cap = cap;
        }
        return true;
    }

    // what the launch of one request needs, copied out under the lock
    struct Item {
        cm_request r;
        char* fixed;
        char* ev;
        size_t cap, o_scratch, o_rho, o_drho, o_small;
    };

    // enqueue copies in, the plan, copies out for one batch on a lane reserved
    // for it; runs without the lock (the streams involved are marked busy, so
    // nothing else touches their memory)
    int launch(Lane& L, const std::vector<Item>& items)
    {
        std::vector<cm_window> wins(items.size());
        for (size_t i = 0; i < items.size(); ++i) {
            const Item& it = items[i];
            const cm_request& q = it.r;
            const size_t cap = it.cap;
            int16_t* dx = reinterpret_cast<int16_t*>(it.ev);
            int16_t* dy = reinterpret_cast<int16_t*>(it.ev + up256(2 * cap));
            float* dt = reinterpret_cast<float*>(it.ev + 2 * up256(2 * cap));
            int8_t* dp = reinterpret_cast<int8_t*>(it.ev + 2 * up256(2 * cap) + up256(4 * cap));
            float* rho = reinterpret_cast<float*>(it.fixed + it.o_rho);
            float* drho = reinterpret_cast<float*>(it.fixed + it.o_drho);
            float* small = reinterpret_cast<float*>(it.fixed + it.o_small);  // ego[6], dego[6], loss, dloss
            const size_t HW = (size_t)q.cam.width * q.cam.height;
            bool ok = true;
            // the upstream gradient dL/dloss = 1, written on every launch: the fixed
            // block may have been (re)allocated from pool memory that held anything
            static const float one = 1.0f;
            ok = ok && cudaMemcpyAsync(small + 13, &one, 4, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
            if (q.n > 0) {
                ok = ok && cudaMemcpyAsync(dx, q.x, 2 * q.n, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
                ok = ok && cudaMemcpyAsync(dy, q.y, 2 * q.n, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
                ok = ok && cudaMemcpyAsync(dt, q.t, 4 * q.n, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
                ok = ok && cudaMemcpyAsync(dp, q.p, q.n, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
            }
            ok = ok && cudaMemcpyAsync(rho, q.inv_depth, 4 * HW, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(small, q.ego6, 24, cudaMemcpyHostToDevice, L.s) == cudaSuccess;
            if (!ok) return CM_ECUDA;
            cm_window& w = wins[i];
            std::memset(&w, 0, sizeof(w));
            w.cam = q.cam;
            w.ev = cm_events{dx, dy, dt, dp, q.n, q.t0, q.t1};
            w.inv_depth = rho;
            w.ego6 = small;
            w.dt_window = q.dt_window;
            w.dego6 = small + 6;
            w.loss_out = small + 12;
            w.dloss = small + 13;
            w.dinv_depth = q.dinv_depth_out ? drho : nullptr;
            w.scratch = it.fixed + it.o_scratch;
        }
        int rc = cm_batch_set_windows(L.plan, wins.data(), (int32_t)wins.size());
        if (rc) return rc;
        if ((rc = cm_batch_run(L.plan, L.s))) return rc;
        for (const Item& it : items) {
            const cm_request& q = it.r;
            float* small = reinterpret_cast<float*>(it.fixed + it.o_small);
            const size_t HW = (size_t)q.cam.width * q.cam.height;
            bool ok = cudaMemcpyAsync(q.loss_out, small + 12, 4, cudaMemcpyDeviceToHost, L.s) == cudaSuccess;
            if (q.dego6_out)
                ok = ok && cudaMemcpyAsync(q.dego6_out, small + 6, 24, cudaMemcpyDeviceToHost, L.s) == cudaSuccess;
            if (q.dinv_depth_out)
                ok = ok && cudaMemcpyAsync(q.dinv_depth_out, it.fixed + it.o_drho, 4 * HW, cudaMemcpyDeviceToHost,
                                           L.s) == cudaSuccess;
            if (!ok) return CM_ECUDA;
        }
        return cudaEventRecord(L.done, L.s) == cudaSuccess ? CM_OK : CM_ECUDA;
    }

    // one pass of the scheduler: called and returning with the lock held, which
    // it releases while a batch's copies and graph are enqueued
    bool step(std::unique_lock<std::mutex>& lk)
    {
        bool worked = false;
        // completions
        for (Lane& L : lanes) {
            if (!L.busy || L.tickets.empty()) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            const double t = now_s();
            for (uint64_t tk : L.tickets) {
                Request& R = reqs[tk];
                R.done = true;
                R.t_done = t;
                R.status = q == cudaSuccess ? CM_OK : CM_ECUDA;
                StreamState& s = streams[R.r.stream_id];
                s.busy = false;
                s.last_use = ++clock;
                st.completed += 1;
            }
            L.tickets.clear();
            L.busy = false;
            worked = true;
            done_cv.notify_all();
        }
        // admission into free lanes
        for (Lane& L : lanes) {
            if (L.busy || queue.empty()) continue;
            std::vector<uint64_t> batch;
            std::vector<Item> items;
            std::unordered_set<int32_t> seen;  // streams with an earlier request still queued keep their order
            std::vector<uint64_t> rest;         // requests passed over, in queue order
            // scan from the front until the batch is full: a pass costs what it admits
            // and passes over, not the length of the queue
            while (!queue.empty() && (int)batch.size() < cfg.max_batch) {
                const uint64_t tk = queue.front();
                queue.pop_front();
                Request& R = reqs[tk];
                StreamState& s = streams[R.r.stream_id];
                s.id = R.r.stream_id;
                bool blocked = s.busy || seen.count(s.id) != 0;
                if (!blocked && !ensure_state(s, R.r)) {
                    blocked = true;
                    st.memory_waits += 1;
                }
                if (blocked) {
                    seen.insert(s.id);
                    rest.push_back(tk);
                    continue;
                }
                s.busy = true;
                batch.push_back(tk);
                items.push_back(Item{R.r, at(s.fixed_off), at(s.ev_off), s.ev_cap, s.o_scratch, s.o_rho, s.o_drho,
                                     s.o_small});
            }
            // the requests passed over go back to the front, in their order
            for (auto it = rest.rbegin(); it != rest.rend(); ++it) queue.push_front(*it);
            if (batch.empty()) break;
            const double t = now_s();
            for (uint64_t tk : batch) {
                reqs[tk].t_start = t;
                reqs[tk].batch_size = (int32_t)batch.size();
            }
            L.busy = true;  // reserved: the completion check skips it until its tickets are set
            lk.unlock();
            const int rc = launch(L, items);
            lk.lock();
            if (rc != CM_OK) {
                for (uint64_t tk : batch) {
                    Request& R = reqs[tk];
                    R.done = true;
                    R.status = rc;
                    R.t_done = now_s();
                    streams[R.r.stream_id].busy = false;
                }
                L.busy = false;
                done_cv.notify_all();
            } else {
                L.tickets = batch;
                st.batches += 1;
                st.batched_requests += (int64_t)batch.size();
            }
            worked = true;
        }
        st.pool_used = pool.used();
        st.pool_peak = pool.peak();
        st.queued = (int64_t)queue.size();
        return worked;
    }

    void loop()
    {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            const bool worked = step(lk);
            bool busy = false;
            for (const Lane& L : lanes) busy = busy || L.busy;
            if (!worked) cv.wait_for(lk, std::chrono::microseconds(busy ? 20 : 500));
        }
    }
};

extern "C" {

int cm_server_create(const cm_server_cfg* cfg, cm_server** out)
{
    if (!cfg || !out || cfg->hbm_budget < (1u << 20) || cfg->max_batch < 1 || cfg->lanes < 1 || cfg->lanes > 16 ||
        cfg->max_queue < 1 || cfg->nbins < 1 || cfg->nbins > CM_MAX_BINS || cfg->group_events < 0 ||
        cfg->group_events > ((int64_t)1 << 36) ||
        (cfg->ref_mode != CM_REF_END && cfg->ref_mode != CM_REF_ALL_EDGES))
        return CM_EINVAL;
    cm_server* S = new (std::nothrow) cm_server;
    if (!S) return CM_ENOMEM;
    S->cfg = *cfg;
    S->lcfg = cm_loss_cfg{cfg->nbins, cfg->ref_mode, CM_SPLAT_ATOMIC, 0, cfg->eps};
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete S;
        return CM_ECUDA;
    }
    if (cudaMalloc(reinterpret_cast<void**>(&S->dev), cfg->hbm_budget) != cudaSuccess) {
        delete S;
        return CM_ENOMEM;
    }
    S->pool.init(cfg->hbm_budget);
    // one plan per lane, sized for max_batch windows that bring their own scratch
    // and, with group_events, for the band grouping of that many events (the
    // prototype windows share them out; they are never run, their event
    // pointers only need to be non-null)
    std::vector<cm_window> proto(cfg->max_batch);
    const int64_t per = (cfg->group_events + cfg->max_batch - 1) / cfg->max_batch;
    for (cm_window& w : proto) {
        std::memset(&w, 0, sizeof(w));
        w.cam = cm_camera{per > 0 ? 1280 : 2, per > 0 ? 720 : 2, 1.0f, 1.0f, 0.5f, 0.5f};
        w.ev = cm_events{nullptr, nullptr, nullptr, nullptr, per, 0.0f, 1.0f};
        if (per > 0) {
            w.ev.x = reinterpret_cast<const int16_t*>(S->dev);
            w.ev.y = reinterpret_cast<const int16_t*>(S->dev);
            w.ev.t = reinterpret_cast<const float*>(S->dev);
            w.ev.p = reinterpret_cast<const int8_t*>(S->dev);
        }
        w.flow = reinterpret_cast<const float*>(S->dev);
        w.dloss = reinterpret_cast<const float*>(S->dev);
        w.loss_out = reinterpret_cast<float*>(S->dev);
        w.scratch = S->dev;
    }
    int rc = CM_OK;
    S->lanes.resize(cfg->lanes);
    for (Lane& L : S->lanes) {
        if (rc) break;
        size_t b = 0;
        if ((rc = cm_batch_query(proto.data(), cfg->max_batch, &S->lcfg, &b))) break;
        L.plan_bytes = b;
        L.plan_off = S->pool.alloc(b);
        if (L.plan_off == Pool::kNone) {
            rc = CM_ENOMEM;
            break;
        }
        if ((rc = cm_batch_create(S->dev + L.plan_off, b, proto.data(), cfg->max_batch, &S->lcfg, &L.plan))) break;
        // one graph for every mix of windows, events grouped by band while the lane's memory lasts
        const cm_batch_schedule wide{1, 0, cfg->group_events > 0 ? 2 : 0, 0};
        if ((rc = cm_batch_set_schedule(L.plan, &wide))) break;
        if (cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)
            rc = CM_ECUDA;
    }
    if (!rc) rc = S->warm_lanes();
    if (rc) {
        cm_server_destroy(S);
        return rc;
    }
    S->th = std::thread([S] { S->loop(); });
    *out = S;
    return CM_OK;
}

int cm_batch_submit(cm_server* S, const cm_request* req, uint64_t* ticket)
{
    if (!S || !ticket || !request_ok(req)) return CM_EINVAL;
    size_t a, b, c, d;
    const size_t need = S->fixed_bytes_for(req->cam.width, req->cam.height, &a, &b, &c, &d) +
                        cm_server::events_bytes((size_t)req->n) + 4096;
    size_t plans = 0;
    for (const Lane& L : S->lanes) plans += up256(L.plan_bytes);
    if (need + plans > S->pool.size()) return CM_ENOMEM;  // can never fit the budget
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->cfg.max_queue) return CM_EBUSY;
    const uint64_t t = S->next_ticket++;
    Request R;
    R.r = *req;
    R.t_submit = now_s();
    S->reqs[t] = R;
    S->queue.push_back(t);
    S->st.submitted += 1;
    *ticket = t;
    S->cv.notify_one();
    return CM_OK;
}

static void fill_result(const Request& R, cm_result* res)
{
    if (!res) return;
    res->status = R.status;
    res->batch_size = R.batch_size;
    res->t_submit = R.t_submit;
    res->t_start = R.t_start;
    res->t_done = R.t_done;
}

int cm_batch_poll(cm_server* S, uint64_t ticket, cm_result* res, int32_t* done)
{
    if (!S || !done) return CM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CM_ENOTFOUND;
    *done = it->second.done ? 1 : 0;
    if (it->second.done) {
        fill_result(it->second, res);
        S->reqs.erase(it);
    }
    return CM_OK;
}

int cm_batch_wait(cm_server* S, uint64_t ticket, double timeout_s, cm_result* res)
{
    if (!S) return CM_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return CM_ENOTFOUND;
        if (it->second.done) {
            fill_result(it->second, res);
            S->reqs.erase(it);
            return CM_OK;
        }
        if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = S->reqs.find(ticket);
            if (it != S->reqs.end() && it->second.done) continue;
            return CM_ETIMEOUT;
        }
    }
}

int cm_server_get_stats(cm_server* S, cm_server_stats* out)
{
    if (!S || !out) return CM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->pool_bytes = S->pool.size();
    return CM_OK;
}

int cm_server_destroy(cm_server* S)
{
    if (!S) return CM_OK;
    if (S->th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv.notify_all();
        S->th.join();
    }
    for (Lane& L : S->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        if (L.plan) cm_batch_destroy(L.plan);
        if (L.done) cudaEventDestroy(L.done);
        if (L.s) cudaStreamDestroy(L.s);
    }
    if (S->dev) cudaFree(S->dev);
    delete S;
    return CM_OK;
}

}  // extern "C"
