// ds_serve.cu -- continuous-batching render server (host code over the C ABI).
//
// Soups stay resident on the device.  Requests (one view each) are queued
// without blocking; a scheduler thread hands them to k workers, each a
// library context on its own stream.  When a worker is free it takes the
// oldest queued request together with the other queued requests that share
// its mode, background and texture shape (grid_n, C), whatever their soup
// (up to max_batch views, one multi-soup forward launch), so requests that
// arrive while others are on the GPU join the next batch, and batches on
// different streams overlap on the device.  Admission is by device memory: a batch is
// launched only if the scratch estimate of all in-flight batches stays within
// the budget (a lone request is always admitted).  Completion is signalled by
// a host function enqueued behind each batch (no polling).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ds_internal.h"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct Request {
    uint64_t ticket = 0;
    int soup = 0;
    ds_camera cam{};
    uint64_t seed = 0;
    uint32_t mode = 0;
    float bg[DS_MAX_CHANNELS] = {0};
    ds_view_out out{};
    size_t bytes = 0;
    int state = kQueued;
    ds_status status = DS_OK;
    int64_t t_submit = 0, t_launch = 0, t_done = 0;
    int batch = 0;
};

struct Worker;

struct Batch {
    ds_server* srv = nullptr;
    Worker* w = nullptr;
    std::vector<Request*> reqs;
    std::vector<int32_t> soup_ids;   // each request's soup, as ids in the worker's context
    size_t bytes = 0;
};

struct Worker {
    ds_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;
    Batch batch;
    std::mutex call_mu;   // serialises calls into ctx (launches, soup registration)
};

struct ServerSoup {
    float* mem = nullptr;   // server-owned copy: vertices then texture logits
    int T = 0, N = 0, C = 0;
    std::vector<int32_t> ids;   // soup id in each worker context
};

}  // namespace

struct ds_server {
    int device = 0;
    size_t budget = 0, in_flight = 0;
    int max_batch = 16;
    size_t max_queue = 1 << 20;
    std::vector<Worker> workers;
    std::vector<ServerSoup> soups;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    bool stop = false, paused = false;
    std::vector<Batch*> finished;
    std::thread thread;
};

namespace {

// Scratch estimate of one request: per-(view, triangle) set-up arrays, about
// four bin pairs per triangle (double-buffered keys and values) and the tile
// ranges.
size_t request_bytes(const ServerSoup& s, const ds_camera& c) {
    const size_t tiles = (size_t)((c.width + 15) / 16) * ((c.height + 15) / 16);
    return (size_t)s.T * (64 + 4 + 4 + 16 + 4) + (size_t)s.T * 4 * 16 + tiles * 8;
}

void CUDART_CB batch_done(void* p) {
    Batch* b = static_cast<Batch*>(p);
    ds_server* srv = b->srv;
    const int64_t t = now_ns();
    std::lock_guard<std::mutex> lk(srv->mu);
    for (Request* r : b->reqs) r->t_done = t;
    srv->finished.push_back(b);
    srv->cv_sched.notify_one();
}

bool any_free(ds_server* s) {
    for (auto& w : s->workers)
        if (!w.busy) return true;
    return false;
}

bool any_busy(ds_server* s) {
    for (auto& w : s->workers)
        if (w.busy) return true;
    return false;
}

// A queued request can be launched now: not paused, a worker is free and the
// oldest request fits the memory budget (or nothing is in flight).  The
// scheduler sleeps unless this (or a completion, or stop) holds; it must be
// false while admission is blocked, else the scheduler would spin on the lock.
bool can_launch(ds_server* s) {
    return !s->paused && !s->queue.empty() && any_free(s) &&
           (s->in_flight == 0 || s->in_flight + s->queue.front()->bytes <= s->budget);
}

// Launch a batch (called without the server lock held).
ds_status launch(ds_server* s, Worker& w, Batch& b) {
    const int n = (int)b.reqs.size();
    std::vector<ds_camera> cams(n);
    std::vector<uint64_t> seeds(n);
    std::vector<ds_view_out> outs(n);
    for (int i = 0; i < n; ++i) {
        cams[i] = b.reqs[i]->cam;
        seeds[i] = b.reqs[i]->seed;
        outs[i] = b.reqs[i]->out;
    }
    const Request* r0 = b.reqs[0];
    std::lock_guard<std::mutex> cl(w.call_mu);
    ds_status st = ds_raster_forward_multi(w.ctx, b.soup_ids.data(), cams.data(), seeds.data(), n, 1,
                                           r0->mode | DS_NO_SYNC, r0->bg, outs.data(), w.stream);
    if (st != DS_OK) return st;
    if (cudaLaunchHostFunc(w.stream, batch_done, &b) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_CUDA;
    }
    return DS_OK;
}

void scheduler(ds_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_sched.wait(lk, [&] {
            return !s->finished.empty() || (s->stop ? !any_busy(s) : can_launch(s));
        });
        // ---- retire finished batches
        while (!s->finished.empty()) {
            Batch* b = s->finished.back();
            s->finished.pop_back();
            Worker& w = *b->w;
            lk.unlock();
            // a bin overflow in the no-sync launch: render the batch again with
            // synchronised sizing (rare; the contexts reserve ample capacity)
            std::unique_lock<std::mutex> cl(w.call_mu);
            ds_status st = ds_ctx_status(w.ctx);
            if (st == DS_ERR_CAPACITY) {
                const int n = (int)b->reqs.size();
                std::vector<ds_camera> cams(n);
                std::vector<uint64_t> seeds(n);
                std::vector<ds_view_out> outs(n);
                for (int i = 0; i < n; ++i) {
                    cams[i] = b->reqs[i]->cam;
                    seeds[i] = b->reqs[i]->seed;
                    outs[i] = b->reqs[i]->out;
                }
                const Request* r0 = b->reqs[0];
                st = ds_raster_forward_multi(w.ctx, b->soup_ids.data(), cams.data(), seeds.data(), n, 1, r0->mode,
                                             r0->bg, outs.data(), w.stream);
                if (st == DS_OK && cudaStreamSynchronize(w.stream) != cudaSuccess) st = DS_ERR_CUDA;
                const int64_t t = now_ns();
                for (Request* r : b->reqs) r->t_done = t;
            }
            cl.unlock();
            lk.lock();
            for (Request* r : b->reqs) {
                r->status = st;
                r->state = st == DS_OK ? kDone : kFailed;
            }
            s->in_flight -= b->bytes;
            w.busy = false;
            b->reqs.clear();
            s->cv_done.notify_all();
        }
        if (s->stop) {
            if (!any_busy(s)) break;
            continue;   // wait for the batches in flight
        }
        // ---- form and launch batches on free workers
        while (can_launch(s)) {
            Worker* w = nullptr;
            for (auto& x : s->workers)
                if (!x.busy) {
                    w = &x;
                    break;
                }
            Request* first = s->queue.front();
            const ServerSoup& fs = s->soups[first->soup];
            Batch& b = w->batch;
            b.srv = s;
            b.w = w;
            b.reqs.clear();
            b.soup_ids.clear();
            b.bytes = 0;
            const size_t wi = (size_t)(w - s->workers.data());
            for (auto it = s->queue.begin(); it != s->queue.end() && (int)b.reqs.size() < s->max_batch;) {
                Request* r = *it;
                const ServerSoup& rs = s->soups[r->soup];
                const bool same = r->mode == first->mode && rs.N == fs.N && rs.C == fs.C &&
                                  std::memcmp(r->bg, first->bg, sizeof(r->bg)) == 0;
                if (same && (b.reqs.empty() || s->in_flight + b.bytes + r->bytes <= s->budget)) {
                    b.reqs.push_back(r);
                    b.soup_ids.push_back(rs.ids[wi]);
                    b.bytes += r->bytes;
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            const int64_t t = now_ns();
            for (Request* r : b.reqs) {
                r->state = kRunning;
                r->t_launch = t;
                r->batch = (int)b.reqs.size();
            }
            w->busy = true;
            s->in_flight += b.bytes;
            lk.unlock();
            const ds_status st = launch(s, *w, b);
            lk.lock();
            if (st != DS_OK) {
                for (Request* r : b.reqs) {
                    r->status = st;
                    r->state = kFailed;
                }
                s->in_flight -= b.bytes;
                w->busy = false;
                b.reqs.clear();
                s->cv_done.notify_all();
            }
        }
    }
}

bool finite_cam(const ds_camera& c) {
    const float* f = &c.fx;
    for (int i = 0; i < 17; ++i)
        if (!(f[i] == f[i]) || f[i] > 3.0e38f || f[i] < -3.0e38f) return false;
    return c.fx != 0.f && c.fy != 0.f && c.near_z > 0.f && c.width >= 1 && c.height >= 1 &&
           c.width <= DS_MAX_RESOLUTION && c.height <= DS_MAX_RESOLUTION;
}

ds_status sfail(ds_status code, const std::string& msg) {
    ds::report_error(msg);
    return code;
}

}  // namespace

extern "C" {

ds_status ds_server_create(int32_t device, int32_t n_streams, size_t mem_budget, int32_t max_batch,
                           int64_t reserve_pairs, ds_server** out) {
    if (!out || n_streams < 1 || n_streams > 32 || max_batch < 1 || max_batch > DS_MAX_VIEWS || reserve_pairs < 0)
        return sfail(DS_ERR_INVALID_ARG, "bad server arguments");
    *out = nullptr;
    ds_server* s = new (std::nothrow) ds_server();
    if (!s) return sfail(DS_ERR_OOM, "host allocation failed");
    s->device = device;
    s->budget = mem_budget;
    s->max_batch = max_batch;
    s->workers = std::vector<Worker>(n_streams);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return sfail(DS_ERR_INVALID_ARG, "bad device index");
    }
    for (auto& w : s->workers) {
        ds_status st = ds_create(&w.ctx, device);
        if (st == DS_OK && reserve_pairs > 0) st = ds_reserve(w.ctx, reserve_pairs);
        if (st == DS_OK && cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = DS_ERR_CUDA;
        }
        if (st != DS_OK) {
            for (auto& x : s->workers) {
                if (x.ctx) ds_destroy(x.ctx);
                if (x.stream) cudaStreamDestroy(x.stream);
            }
            delete s;
            return st;
        }
    }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return DS_OK;
}

ds_status ds_server_add_soup(ds_server* s, const float* verts, const float* tex, int32_t T, int32_t grid_n, int32_t C,
                             int32_t* soup_id) {
    if (!s || !verts || !tex || !soup_id) return sfail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES || grid_n < 1 || grid_n > DS_MAX_GRID_N || C < 2 || C > DS_MAX_CHANNELS)
        return sfail(DS_ERR_INVALID_ARG, "T, grid_n or C out of range");
    const size_t V = (size_t)(grid_n + 1) * (grid_n + 2) / 2;
    const size_t nv = 9 * (size_t)T, nt = (size_t)T * V * C, nv4 = (nv + 3) & ~size_t(3);
    ServerSoup ss;
    ss.T = T;
    ss.N = grid_n;
    ss.C = C;
    cudaSetDevice(s->device);
    if (cudaMalloc(reinterpret_cast<void**>(&ss.mem), sizeof(float) * (nv4 + nt)) != cudaSuccess) {
        cudaGetLastError();
        return sfail(DS_ERR_OOM, "cudaMalloc failed for a served soup");
    }
    if (cudaMemcpy(ss.mem, verts, sizeof(float) * nv, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(ss.mem + nv4, tex, sizeof(float) * nt, cudaMemcpyDeviceToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ss.mem);
        return sfail(DS_ERR_CUDA, "copy of a served soup failed");
    }
    std::lock_guard<std::mutex> lk(s->mu);   // the scheduler reads soups[] under this lock
    for (auto& w : s->workers) {
        std::lock_guard<std::mutex> cl(w.call_mu);
        int32_t id = -1;
        const ds_status st = ds_soup_upload(w.ctx, ss.mem, ss.mem + nv4, T, grid_n, C, DS_BORROW | DS_STATIC, &id,
                                            nullptr);
        if (st != DS_OK) {
            for (size_t k = 0; k < ss.ids.size(); ++k) {
                std::lock_guard<std::mutex> ck(s->workers[k].call_mu);
                ds_soup_free(s->workers[k].ctx, ss.ids[k]);
            }
            cudaFree(ss.mem);
            return st;
        }
        ss.ids.push_back(id);
    }
    *soup_id = (int32_t)s->soups.size();
    s->soups.push_back(ss);
    return DS_OK;
}

ds_status ds_render_request(ds_server* s, int32_t soup_id, const ds_camera* cam, uint64_t seed, uint32_t mode,
                            const float* bg, const ds_view_out* out, uint64_t* ticket) {
    if (!s || !cam || !out || !ticket) return sfail(DS_ERR_INVALID_ARG, "NULL argument");
    if (mode != DS_MODE_STOCHASTIC && mode != DS_MODE_THRESHOLD_HALF) return sfail(DS_ERR_INVALID_ARG, "bad mode");
    if (!finite_cam(*cam)) return sfail(DS_ERR_INVALID_ARG, "invalid camera");
    if (!out->gbuf || !out->color || ((uintptr_t)out->gbuf & 15)) return sfail(DS_ERR_INVALID_ARG, "bad output");
    std::lock_guard<std::mutex> lk(s->mu);
    if (soup_id < 0 || soup_id >= (int)s->soups.size()) return sfail(DS_ERR_NOT_FOUND, "unknown soup");
    if (s->stop) return sfail(DS_ERR_BUSY, "server is shutting down");
    if (s->queue.size() >= s->max_queue) return sfail(DS_ERR_BUSY, "request queue is full");
    Request* r = new (std::nothrow) Request();
    if (!r) return sfail(DS_ERR_OOM, "host allocation failed");
    r->ticket = s->next_ticket++;
    r->soup = soup_id;
    r->cam = *cam;
    r->seed = seed;
    r->mode = mode;
    const int Co = s->soups[soup_id].C - 1;
    for (int c = 0; c < Co; ++c) r->bg[c] = bg ? bg[c] : 0.f;
    r->out = *out;
    r->bytes = request_bytes(s->soups[soup_id], *cam);
    r->t_submit = now_ns();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv_sched.notify_one();
    return DS_OK;
}

ds_status ds_request_wait(ds_server* s, uint64_t ticket, int32_t timeout_ms, ds_request_stats* stats) {
    if (!s) return sfail(DS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(DS_ERR_NOT_FOUND, "unknown ticket");
    Request* r = it->second;
    auto finished = [&] { return r->state >= kDone; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, finished);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
        return sfail(DS_ERR_TIMEOUT, "request not finished within the time limit");
    if (stats) {
        stats->submit_ns = r->t_submit;
        stats->launch_ns = r->t_launch;
        stats->done_ns = r->t_done;
        stats->batch = r->batch;
    }
    const ds_status st = r->state == kCancelled ? DS_ERR_BUSY : r->status;
    s->reqs.erase(it);
    delete r;
    if (st != DS_OK) return sfail(st, "request failed or was cancelled");
    return DS_OK;
}

ds_status ds_server_pause(ds_server* s, int32_t paused) {
    if (!s) return sfail(DS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->cv_sched.notify_one();
    return DS_OK;
}

ds_status ds_server_destroy(ds_server* s) {
    if (!s) return sfail(DS_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request* r : s->queue) {
            r->state = kCancelled;
            r->status = DS_ERR_BUSY;
        }
        s->queue.clear();
        s->cv_sched.notify_one();
        s->cv_done.notify_all();
    }
    if (s->thread.joinable()) s->thread.join();   // in-flight batches complete first
    cudaSetDevice(s->device);
    for (auto& w : s->workers) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.ctx) ds_destroy(w.ctx);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    for (auto& ss : s->soups) cudaFree(ss.mem);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return DS_OK;
}

}  // extern "C"
