// Continuous-batching server (gf_server_* in gaussbox.h).
//
// A host thread owns the schedule.  Requests wait FIFO until their release
// time has passed and their output fits the HBM arena (the admission budget);
// admitted requests are packed into steps (batch_plan / batch_enqueue, one
// persistent launch per fused class, two launches per two-pass request, whose
// FP32 intermediate is held in the arena while its step is in flight) issued
// round-robin on a pool of streams,
// so consecutive steps overlap on the device while new requests keep arriving.
// A step retires when its CUDA event has completed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "plan.h"
#include "serve.h"

namespace gb {

double clock_now() {
    using namespace std::chrono;
    static const steady_clock::time_point t0 = steady_clock::now();
    return duration<double>(steady_clock::now() - t0).count();
}

namespace {

constexpr size_t kArenaAlign = 256;

// First-fit allocator over [0, size) with coalescing free list.
struct Arena {
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    void reset(size_t n) {
        size = n;
        used = peak = 0;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first;
                free_.erase(it);
                if (rest) free_[o + bytes] = rest;
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    gf_image_desc d{};
    Image im;
    BoxKernel bk;
    double t_release = 0, t_admit = 0, t_done = 0;
    size_t out_off = 0, out_bytes = 0;
    size_t inter_off = 0, inter_bytes = 0;   // two-pass intermediate (0 bytes: fused)
    int status = GF_OK;
    int state = 0;   // 0 queued, 1 in a step, 2 done
    bool auto_release = false;
};

struct Step {
    int slot = -1;
    std::vector<long long> tickets;
};

}  // namespace

struct Server {
    gf_handle_s* h = nullptr;
    gf_server_config cfg{};
    unsigned char* arena_dev = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<Scratch> scratch;       // per stream slot: batch staging (device + pinned)
    std::vector<Step> slots;            // in-flight step per slot (slot < 0: free)
    // plain-mode bookkeeping
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<long long> queue;
    std::unordered_map<long long, Req> reqs;
    long long next_ticket = 1;
    long long outstanding = 0;
    bool stopping = false;
    std::thread th;
    gf_server_stats stats{};
    int next_slot = 0;
    // reusable planning storage
    std::vector<Image> ims;
    std::vector<BoxKernel> bks;
    std::vector<Prepared> pr;
    std::vector<int> order;
    std::vector<BatchClass> cls;
    std::vector<TwoPass> tps;
    std::vector<size_t> tp_off;
    std::vector<int> tp_img;
    std::vector<int> wk_img;
};

namespace {

size_t out_bytes_of(const gf_image_desc& d, size_t* pitch) {
    const size_t row = (size_t)d.W * d.C * dtype_size(d.out_dtype);
    *pitch = (row + 15) / 16 * 16;
    return *pitch * (size_t)d.H;
}

// Launches one step of admitted requests on slot `sl`.  Called with mu held.
void launch_step(Server& s, int sl, std::vector<long long>& batch) {
    const int n = (int)batch.size();
    cudaStream_t q = s.streams[sl];
    gf_status st = GF_OK;
    if (s.cfg.plain) {
        for (long long t : batch) {
            Req& r = s.reqs[t];
            gf_status e = launch_filter_into(r.im, r.bk, s.arena_dev + r.inter_off, q);
            if (e != GF_OK) r.status = e;
            else s.stats.launches += planned_path(r.im, r.bk) == GF_PATH_TWO_PASS ? 2 : 1;
        }
    } else {
        if ((int)s.ims.size() < n) {
            s.ims.resize(n);
            s.bks.resize(n);
            s.pr.resize(n);
            s.order.resize(n);
            s.cls.resize(n);
            s.tps.resize(n);
            s.tp_off.resize(n);
            s.tp_img.resize(n);
            s.wk_img.resize(n);
        }
        for (int i = 0; i < n; ++i) {
            s.ims[i] = s.reqs[batch[i]].im;
            s.bks[i] = s.reqs[batch[i]].bk;
        }
        BatchWork w;
        w.pr = s.pr.data();
        w.order = s.order.data();
        w.cls = s.cls.data();
        w.tp = s.tps.data();
        w.tp_off = s.tp_off.data();
        w.tp_img = s.tp_img.data();
        w.wk_img = s.wk_img.data();
        st = batch_plan(s.ims.data(), s.bks.data(), n, w);
        // two-pass intermediates were reserved in the arena at admission
        for (int t = 0; st == GF_OK && t < w.ntp; ++t)
            st = bind_twopass(w.tp[t], s.arena_dev + s.reqs[batch[w.tp_img[t]]].inter_off);
        if (st == GF_OK) {
            // the slot's previous step has retired, so its staging is free to reuse
            st = scratch_reserve(s.scratch[sl], w.total, w.total);
        }
        if (st == GF_OK) {
            unsigned char* hp = static_cast<unsigned char*>(s.scratch[sl].pinned);
            unsigned char* dp = static_cast<unsigned char*>(s.scratch[sl].dev);
            batch_stage(w, n, hp, dp);
            st = batch_enqueue(w, dp, hp, q);
            if (st == GF_OK) s.stats.launches += batch_launches(w);
        }
        if (st != GF_OK)
            for (long long t : batch) s.reqs[t].status = st;
    }
    cudaEventRecord(s.events[sl], q);
    s.slots[sl].slot = sl;
    s.slots[sl].tickets = batch;
    s.stats.steps += 1;
    s.stats.sum_batch += n;
}

void server_loop(Server* sp) {
    Server& s = *sp;
    cudaSetDevice(s.h->device);
    // the server's kernels report into its handle's status word
    HandleScope scope(s.h->status_word, s.h->wait_cycles);
    std::vector<long long> batch;
    std::unique_lock<std::mutex> lk(s.mu);
    for (;;) {
        bool progress = false;
        const double now = clock_now();
        // retire completed steps
        for (size_t sl = 0; sl < s.slots.size(); ++sl) {
            Step& st = s.slots[sl];
            if (st.slot < 0) continue;
            const cudaError_t q = cudaEventQuery(s.events[sl]);
            if (q == cudaErrorNotReady) continue;
            const double t = clock_now();
            for (long long tk : st.tickets) {
                Req& r = s.reqs[tk];
                if (r.inter_bytes) {
                    s.arena.release(r.inter_off, r.inter_bytes);
                    r.inter_bytes = 0;
                }
                if (q != cudaSuccess && r.status == GF_OK) r.status = GF_ECUDA;
                r.t_done = t;
                r.state = 2;
                s.stats.completed += 1;
                s.outstanding -= 1;
                s.stats.busy_last_done = std::max(s.stats.busy_last_done, t);
                if (r.auto_release) {
                    s.arena.release(r.out_off, r.out_bytes);
                    s.reqs.erase(tk);
                }
            }
            st.slot = -1;
            st.tickets.clear();
            progress = true;
        }
        if (progress) s.cv_done.notify_all();
        // admit released requests FIFO while their outputs fit, one step per free slot
        for (size_t k = 0; k < s.slots.size() && !s.queue.empty(); ++k) {
            const int sl = s.next_slot;
            if (s.slots[sl].slot >= 0) break;   // slots retire in order: wait for this one
            batch.clear();
            const int maxb = s.cfg.plain ? 1 : s.cfg.max_batch;
            while (!s.queue.empty() && (int)batch.size() < maxb) {
                Req& r = s.reqs[s.queue.front()];
                if (r.t_release > now) break;
                size_t off, ioff = 0;
                if (!s.arena.alloc(r.out_bytes, &off)) break;   // head waits for memory
                if (r.inter_bytes && !s.arena.alloc(r.inter_bytes, &ioff)) {
                    s.arena.release(off, r.out_bytes);
                    break;
                }
                r.inter_off = ioff;
                r.out_off = off;
                r.d.d_out = s.arena_dev + off;
                r.im.out = r.d.d_out;
                r.t_admit = now;
                r.state = 1;
                batch.push_back(s.queue.front());
                s.queue.pop_front();
            }
            if (batch.empty()) break;
            s.stats.arena_peak = std::max(s.stats.arena_peak, s.arena.peak);
            launch_step(s, sl, batch);
            s.next_slot = (sl + 1) % (int)s.slots.size();
            progress = true;
        }
        if (s.stopping && s.queue.empty() && s.outstanding == 0) break;
        if (!progress) {
            // nothing to do right now: release the lock briefly
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace

void server_destroy(gf_handle_s* h) {
    if (!h || !h->server) return;
    Server* s = h->server;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    if (s->th.joinable()) s->th.join();
    for (size_t i = 0; i < s->streams.size(); ++i) {
        cudaStreamSynchronize(s->streams[i]);
        cudaStreamDestroy(s->streams[i]);
        cudaEventDestroy(s->events[i]);
        scratch_free(s->scratch[i]);
    }
    if (s->arena_dev) cudaFree(s->arena_dev);
    delete s;
    h->server = nullptr;
}

}  // namespace gb

using namespace gb;

extern "C" {

double gf_clock_now(void) { return clock_now(); }

gf_status gf_server_start(gf_handle h, const gf_server_config* cfg) {
    if (!h) return GF_EINVAL;
    if (h->server) return GF_EBUSY;
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    Server* s = new Server();
    s->h = h;
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_batch <= 0) s->cfg.max_batch = 64;
    if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 4;
    size_t budget = s->cfg.hbm_budget_bytes ? s->cfg.hbm_budget_bytes : h->hbm_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = fr / 2;
    }
    budget = budget / kArenaAlign * kArenaAlign;
    if (cudaMalloc(reinterpret_cast<void**>(&s->arena_dev), budget) != cudaSuccess) {
        delete s;
        return GF_ENOMEM;
    }
    s->arena.reset(budget);
    s->stats.arena_bytes = budget;
    const int ns = s->cfg.plain ? 1 : s->cfg.max_inflight;
    s->streams.resize(ns);
    s->events.resize(ns);
    s->scratch.resize(ns);
    s->slots.resize(ns);
    for (int i = 0; i < ns; ++i) {
        cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
    }
    s->stats.busy_first_release = -1.0;
    h->server = s;
    s->th = std::thread(server_loop, s);
    return GF_OK;
}

gf_status gf_server_submit(gf_handle h, const gf_image_desc* req, double release_time, int auto_release,
                           long long* ticket) {
    if (!h || !h->server || !req || !ticket) return GF_EINVAL;
    Server& s = *h->server;
    gf_image_desc d = *req;
    size_t pitch;
    const size_t ob = out_bytes_of(d, &pitch);
    d.d_out = reinterpret_cast<void*>((uintptr_t)16);   // placeholder for validation; set at admission
    d.out_pitch = pitch;
    Image im;
    BoxKernel bk;
    BatchSpan spans[2];
    gf_status st = collect_batch(&d, 1, &im, &bk, spans);
    if (st != GF_OK) return st;
    apply_tuned(h, im, bk);
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.stopping) return GF_EBUSY;
    // a two-pass request also holds its FP32 intermediate while in a step;
    // radii beyond the shared-memory paths are for single-image calls
    const int path = planned_path(im, bk);
    if (path == GF_PATH_HBM) return GF_EUNSUPPORTED;
    if (path == GF_PATH_WALK && im.plan.path == GF_PATH_WALK) return GF_EUNSUPPORTED;   // single images only
    const size_t ib = path == GF_PATH_TWO_PASS ? twopass_inter_bytes(im) : 0;
    const auto arena_bytes = [](size_t b) { return (b + kArenaAlign - 1) / kArenaAlign * kArenaAlign; };
    if (arena_bytes(ob) + arena_bytes(ib) > s.arena.size) {
        s.stats.rejected += 1;
        return GF_EADMIT;
    }
    const double tr = release_time > 0 ? release_time : clock_now();
    const long long t = s.next_ticket++;
    Req& r = s.reqs[t];
    r.d = d;
    r.im = im;
    r.bk = bk;
    r.t_release = tr;
    r.out_bytes = ob;
    r.inter_bytes = ib;
    r.auto_release = auto_release != 0;
    s.queue.push_back(t);
    s.outstanding += 1;
    s.stats.submitted += 1;
    if (s.stats.busy_first_release < 0 || tr < s.stats.busy_first_release) s.stats.busy_first_release = tr;
    *ticket = t;
    return GF_OK;
}

gf_status gf_server_poll(gf_handle h, long long ticket, gf_completion* out) {
    if (!h || !h->server) return GF_EINVAL;
    Server& s = *h->server;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return GF_EINVAL;
    const Req& r = it->second;
    if (r.state != 2) return GF_EBUSY;
    if (out) {
        out->d_out = r.d.d_out;
        out->out_pitch = r.d.out_pitch;
        out->t_release = r.t_release;
        out->t_admit = r.t_admit;
        out->t_done = r.t_done;
        out->status = r.status;
    }
    return GF_OK;
}

gf_status gf_server_wait(gf_handle h, long long ticket, double timeout_s, gf_completion* out) {
    if (!h || !h->server) return GF_EINVAL;
    const double t_end = clock_now() + timeout_s;
    for (;;) {
        gf_status st = gf_server_poll(h, ticket, out);
        if (st != GF_EBUSY) return st;
        if (clock_now() > t_end) return GF_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

gf_status gf_server_release(gf_handle h, long long ticket) {
    if (!h || !h->server) return GF_EINVAL;
    Server& s = *h->server;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return GF_EINVAL;
    if (it->second.state != 2) return GF_EBUSY;
    s.arena.release(it->second.out_off, it->second.out_bytes);
    s.reqs.erase(it);
    return GF_OK;
}

gf_status gf_server_drain(gf_handle h, double timeout_s) {
    if (!h || !h->server) return GF_EINVAL;
    Server& s = *h->server;
    const double t_end = clock_now() + timeout_s;
    std::unique_lock<std::mutex> lk(s.mu);
    while (s.outstanding > 0) {
        if (clock_now() > t_end) return GF_ETIMEOUT;
        s.cv_done.wait_for(lk, std::chrono::milliseconds(5));
    }
    return GF_OK;
}

gf_status gf_server_stats_get(gf_handle h, gf_server_stats* out) {
    if (!h || !h->server || !out) return GF_EINVAL;
    Server& s = *h->server;
    std::lock_guard<std::mutex> lk(s.mu);
    *out = s.stats;
    out->arena_peak = s.arena.peak;
    return GF_OK;
}

gf_status gf_server_stop(gf_handle h) {
    if (!h) return GF_EINVAL;
    server_destroy(h);
    return GF_OK;
}

}  // extern "C"
