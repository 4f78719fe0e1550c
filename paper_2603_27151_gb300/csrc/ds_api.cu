// ds_api.cu -- the C ABI declared in include/diffsoup.h: contexts, soups,
// scratch management and the launch sequence of the forward and backward
// passes.  Host code only.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ds_internal.h"

namespace {

thread_local std::string g_err;

ds_status fail(ds_status code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define DS_TRY_CUDA(call)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(DS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define DS_TRY(call)                          \
    do {                                      \
        ds_status s_ = (call);                \
        if (s_ != DS_OK) return s_;           \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    ds_status ensure(size_t bytes, const char* what) {
        if (bytes <= cap && p) return DS_OK;
        size_t want = bytes + bytes / 4 + 256;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(DS_ERR_OOM, std::string("cudaMalloc failed for ") + what);
        }
        cap = want;
        return DS_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

struct Soup {
    bool live = false;
    bool owned = false;
    bool fixed = false;       // DS_STATIC: contents never change, activate once
    bool act_valid = false;   // activations of a fixed soup are current
    const float* verts = nullptr;
    const float* tex = nullptr;
    float* own = nullptr;   // owned copy of verts and tex
    float* act = nullptr;   // [T][V][C] and [T][V] (one allocation)
    int T = 0, N = 0, C = 0, V = 0;
    // multi-resolution soups: tex holds levels r_min..r_max (N = 2^r_max)
    int r_min = -1, r_max = -1;
    bool levels() const { return r_min >= 0 && r_min < r_max; }
    size_t tex_floats() const {
        return r_min >= 0 ? ds::level_floats(T, r_min, r_max, C) : (size_t)T * V * C;
    }
};

struct Plan {
    bool valid = false;
    bool devcam = false;   // built from device-resident cameras
    int n_views = 0;
    int soup = -1;
    std::vector<ds_camera> cams;
    int DB = 0;
    int res = 0;
    uint32_t kcap = 0;
    int n_tiles = 0;
};

}  // namespace

namespace ds {
void report_error(const std::string& msg) { g_err = msg; }

bool finite_cam(const ds_camera& c) {
    const float* f = &c.fx;
    for (int i = 0; i < 17; ++i)
        if (!std::isfinite(f[i])) return false;
    return c.fx != 0.f && c.fy != 0.f && c.near_z > 0.f && c.width >= 1 && c.height >= 1 &&
           c.width <= DS_MAX_RESOLUTION && c.height <= DS_MAX_RESOLUTION;
}
}  // namespace ds

using ds::finite_cam;

struct ds_ctx {
    int device = 0;
    std::mutex mu;
    std::vector<Soup> soups;
    DevBuf recs, counts, offs, tbox, zkeys, keys[2], vals[2], hist, hist_scan, ranges, scanbuf, misc, geom;
    DevBuf acc_tex, acc_verts;   // FP64 gradient accumulators of the backward
    DevBuf shade_part;           // per-CTA partials of the shading parameter gradients
    DevBuf plan_dev;             // device copy of an adaptive-control plan
    ds::ScanScratch scan;
    int64_t scan_cap = 0;
    uint32_t* h_word = nullptr;   // pinned host words
    Plan plan;
    ds_tuning tune{16, -1, 0, 256};   // tile shape, depth bits, grid, staging chunk
    int32_t shade_path = DS_SHADE_TENSOR_CORES;   // kernel of ds_shade_forward
    cudaStream_t last_stream = nullptr;
    ds::ViewTable* vt = nullptr;   // host staging of the kernel parameter tables (~9 KB each): [0] the
                                   // call's views, [1] the same views in the edge kernel's tiles

    // optional stage profiler: CUDA events around each pipeline stage
    struct ProfRec {
        int stage;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[ds::kNumStages] = {0};
    long long prof_n[ds::kNumStages] = {0};

    // misc layout
    int* d_status() const { return misc.as<int>(); }
    int* d_counter() const { return misc.as<int>() + 4; }
    uint32_t* d_K() const { return reinterpret_cast<uint32_t*>(misc.as<int>() + 12); }
    unsigned long long* d_total() const { return reinterpret_cast<unsigned long long*>(misc.as<char>() + 64); }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

cudaEvent_t take_event(ds_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one pipeline stage with events on `st` while profiling is on.
struct StageScope {
    ds_ctx* c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageScope(ds_ctx* c_, int stage_, cudaStream_t st_) : c(c_), stage(stage_), st(st_) {
        if (c->prof_on) {
            a = take_event(c);
            if (a) cudaEventRecord(a, st);
        }
    }
    ~StageScope() {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) {
            c->prof_pool.push_back(a);
            return;
        }
        cudaEventRecord(b, st);
        c->prof_pending.push_back({stage, a, b});
    }
};

ds_status prof_flush(ds_ctx* c) {
    for (auto& r : c->prof_pending) {
        DS_TRY_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        DS_TRY_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_ms[r.stage] += ms;
        c->prof_n[r.stage] += 1;
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    c->prof_pending.clear();
    return DS_OK;
}

ds_status ensure_scan(ds_ctx* c, int64_t n) {
    if (n <= c->scan_cap && c->scanbuf.p) return DS_OK;
    int64_t sizes[6] = {0};
    const int lv = ds::scan_levels(n, sizes);
    int64_t total = 0;
    for (int i = 0; i < lv; ++i) total += 2 * sizes[i];
    DS_TRY(c->scanbuf.ensure(sizeof(uint32_t) * (size_t)(total + 1), "scan scratch"));
    uint32_t* p = c->scanbuf.as<uint32_t>();
    c->scan.levels = lv;
    for (int i = 0; i < lv; ++i) {
        c->scan.level_n[i] = sizes[i];
        c->scan.level[i] = p;
        p += sizes[i];
        c->scan.level_out[i] = p;
        p += sizes[i];
    }
    c->scan_cap = n;
    return DS_OK;
}

int bits_for(uint32_t n_values) {   // bits needed for indices 0 .. n_values-1
    int b = 0;
    while (b < 32 && (1ull << b) < n_values) ++b;
    return b;
}

ds::SoupDev soup_dev(const Soup& s) {
    ds::SoupDev d;
    d.verts = s.verts;
    d.tex = s.tex;
    d.act = s.act;
    d.act_a = s.act + (size_t)s.T * s.V * s.C;
    d.T = s.T;
    d.N = s.N;
    d.C = s.C;
    d.V = s.V;
    return d;
}

ds_status get_soup(ds_ctx* c, int32_t id, Soup** out) {
    if (id < 0 || id >= (int)c->soups.size() || !c->soups[id].live)
        return fail(DS_ERR_NOT_FOUND, "unknown soup id " + std::to_string(id));
    *out = &c->soups[id];
    return DS_OK;
}

ds_status check_views(const ds_camera* cams, int32_t n_views, int32_t S) {
    if (!cams) return fail(DS_ERR_INVALID_ARG, "cams is NULL");
    if (n_views < 1 || n_views > DS_MAX_VIEWS)
        return fail(DS_ERR_INVALID_ARG, "n_views must be in [1, " + std::to_string(DS_MAX_VIEWS) + "]");
    if (S < 1 || S > DS_MAX_SAMPLES) return fail(DS_ERR_INVALID_ARG, "S must be in [1, 64]");
    for (int v = 0; v < n_views; ++v)
        if (!finite_cam(cams[v])) return fail(DS_ERR_INVALID_ARG, "camera " + std::to_string(v) + " is invalid");
    return DS_OK;
}

}  // namespace

namespace ds {
// Fill the view table (tiles, work items, per-view pointers).
void build_table(ViewTable& vt, const ds_tuning& tu, const ds_camera* cams, const uint64_t* seeds, int32_t n_views,
                 int32_t S,
                 const ds_view_out* out, const ds_view_gin* gin) {
    std::memset(&vt, 0, sizeof(vt));
    vt.n = n_views;
    vt.S = S;
    vt.n_groups = (S + ds::kSampleGroup - 1) / ds::kSampleGroup;
    vt.tile_w = tu.tile_w;
    vt.tile_h = ds::kTilePix / tu.tile_w;
    vt.chunk = tu.chunk;
    int tile_base = 0, item_base = 0;
    for (int v = 0; v < n_views; ++v) {
        ds::ViewDesc& d = vt.v[v];
        const ds_camera& c = cams[v];
        d.cam.fx = c.fx;
        d.cam.fy = c.fy;
        d.cam.cx = c.cx;
        d.cam.cy = c.cy;
        for (int i = 0; i < 9; ++i) d.cam.R[i] = c.R[i];
        for (int i = 0; i < 3; ++i) d.cam.t[i] = c.t[i];
        d.cam.near_z = c.near_z;
        d.W = c.width;
        d.H = c.height;
        d.tiles_x = (c.width + vt.tile_w - 1) / vt.tile_w;
        d.tiles_y = (c.height + vt.tile_h - 1) / vt.tile_h;
        d.tile_base = tile_base;
        d.item_base = item_base;
        tile_base += d.tiles_x * d.tiles_y;
        item_base += d.tiles_x * d.tiles_y * vt.n_groups;
        const uint64_t sd = seeds ? seeds[v] : 0ull;
        d.seed_lo = (uint32_t)sd;
        d.seed_hi = (uint32_t)(sd >> 32);
        if (out) {
            d.gbuf = out[v].gbuf;
            d.color = out[v].color;
            d.n_front = out[v].n_front;
        }
        if (gin) {
            d.grad_color = gin[v].grad_color;
            d.score_w = gin[v].score_w;
        }
    }
    vt.n_items = item_base;
}

}  // namespace ds

using ds::build_table;

namespace {

int total_tiles(const ds::ViewTable& vt) {
    const ds::ViewDesc& d = vt.v[vt.n - 1];
    return d.tile_base + d.tiles_x * d.tiles_y;
}

// The edge kernel reads G-buffers, colours and set-up records but no bins, so
// its pixel partition need not be the binning tiles: it runs on 32 x 8
// tiles, in which a warp covers one row of 32 pixels and every per-pixel load
// of a warp is one contiguous 128-byte line (the binning tiles of 8 x 32 cut
// a warp's pixels into four 32-byte segments of four lines).
constexpr int kEdgeTileW = 32;

void retile(const ds::ViewTable& vt, int tw, ds::ViewTable& out) {
    out = vt;
    out.tile_w = tw;
    out.tile_h = ds::kTilePix / tw;
    int tile_base = 0, item_base = 0;
    for (int v = 0; v < vt.n; ++v) {
        ds::ViewDesc& d = out.v[v];
        d.tiles_x = (d.W + out.tile_w - 1) / out.tile_w;
        d.tiles_y = (d.H + out.tile_h - 1) / out.tile_h;
        d.tile_base = tile_base;
        d.item_base = item_base;
        tile_base += d.tiles_x * d.tiles_y;
        item_base += d.tiles_x * d.tiles_y * out.n_groups;
    }
    out.n_items = item_base;
}

// Activation, set-up and binning of `vt`'s views into the context's plan;
// view v is of soup *soups[v] (the same soup for every view but in a
// multi-soup forward, whose plan is keyed by plan_soup = -1).
ds_status prepare(ds_ctx* c, int32_t plan_soup, Soup* const* soups, const ds_camera* cams, ds::ViewTable& vt,
                  bool sync, cudaStream_t st) {
    ds::SoupDev sds[DS_MAX_VIEWS];
    const ds::SoupDev* sdp[DS_MAX_VIEWS];
    for (int v = 0; v < vt.n; ++v) {
        sds[v] = soup_dev(*soups[v]);
        sdp[v] = &sds[v];
    }
    ds::set_view_soups(vt, sdp);
    const size_t nvt = (size_t)ds::view_records(vt);
    const int n_tiles = total_tiles(vt);
    c->plan.valid = false;
    DS_TRY(c->recs.ensure(sizeof(ds::SetupRec) * nvt, "set-up records"));
    DS_TRY(c->counts.ensure(4 * nvt, "tile counts"));
    DS_TRY(c->offs.ensure(4 * nvt, "tile offsets"));
    DS_TRY(c->tbox.ensure(16 * nvt, "tile boxes"));
    DS_TRY(c->zkeys.ensure(4 * nvt, "depth keys"));
    DS_TRY(c->ranges.ensure(8 * (size_t)n_tiles, "tile ranges"));
    DS_TRY(ensure_scan(c, (int64_t)nvt));

    for (int v = 0; v < vt.n; ++v) {
        Soup& s = *soups[v];
        bool seen = false;   // activate each soup once
        for (int u = 0; u < v && !seen; ++u) seen = soups[u] == soups[v];
        if (seen || (s.fixed && s.act_valid)) continue;
        StageScope p(c, ds::kStActivate, st);
        if (s.levels())
            DS_TRY_CUDA(ds::launch_compose(s.tex, s.T, s.r_min, s.r_max, s.C, sds[v].act, true, sds[v].act_a, st));
        else
            DS_TRY_CUDA(ds::launch_activate(sds[v], st));
        s.act_valid = s.fixed;
    }
    {
        StageScope p(c, ds::kStSetup, st);
        DS_TRY_CUDA(ds::launch_setup(vt, c->recs.as<ds::SetupRec>(), c->counts.as<uint32_t>(), c->tbox.as<int4>(),
                                     c->zkeys.as<uint32_t>(), st));
    }
    {
        StageScope p(c, ds::kStScan, st);
        DS_TRY_CUDA(ds::scan_exclusive(c->counts.as<uint32_t>(), c->offs.as<uint32_t>(), (int64_t)nvt, c->d_K(), c->scan, st));
    }

    uint32_t kcap = (uint32_t)(c->keys[0].cap / 4);
    if (sync || kcap == 0) {
        DS_TRY_CUDA(cudaMemcpyAsync(c->h_word, c->d_K(), 4, cudaMemcpyDeviceToHost, st));
        DS_TRY_CUDA(cudaStreamSynchronize(st));
        const uint32_t K = *c->h_word;
        if ((size_t)K * 4 > c->keys[0].cap || !c->keys[0].p) {
            for (int b = 0; b < 2; ++b) {
                DS_TRY(c->keys[b].ensure(4 * (size_t)(K > 0 ? K : 1), "bin keys"));
                DS_TRY(c->vals[b].ensure(4 * (size_t)(K > 0 ? K : 1), "bin values"));
            }
        }
        kcap = K;
    }
    const uint32_t nblk = (kcap + ds::kSortBlock - 1) / ds::kSortBlock;
    DS_TRY(c->hist.ensure(4 * 256 * (size_t)(nblk > 0 ? nblk : 1), "radix histogram"));
    DS_TRY(c->hist_scan.ensure(4 * 256 * (size_t)(nblk > 0 ? nblk : 1), "radix offsets"));
    DS_TRY(ensure_scan(c, (int64_t)256 * (nblk > 0 ? nblk : 1)));

    const int tile_bits = bits_for((uint32_t)n_tiles);
    const int DB = std::min(c->tune.depth_bits >= 0 ? c->tune.depth_bits : 16, 32 - tile_bits);
    {
        StageScope p(c, ds::kStEmit, st);
        DS_TRY_CUDA(ds::launch_emit(vt, c->recs.as<ds::SetupRec>(), c->counts.as<uint32_t>(), c->offs.as<uint32_t>(),
                                    c->tbox.as<int4>(), c->zkeys.as<uint32_t>(), DB, c->keys[0].as<uint32_t>(),
                                    c->vals[0].as<uint32_t>(), kcap, c->d_status(), st));
    }
    cudaError_t se = cudaSuccess;
    StageScope* sort_scope = new StageScope(c, ds::kStSort, st);
    const int res = ds::radix_sort_pairs(c->keys[0].as<uint32_t>(), c->vals[0].as<uint32_t>(), c->keys[1].as<uint32_t>(),
                                         c->vals[1].as<uint32_t>(), c->d_K(), kcap, tile_bits + DB,
                                         c->hist.as<uint32_t>(), c->hist_scan.as<uint32_t>(), c->scan, st, &se);
    delete sort_scope;
    DS_TRY_CUDA(se);
    {
        StageScope p(c, ds::kStRanges, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->ranges.p, 0, 8 * (size_t)n_tiles, st));
        DS_TRY_CUDA(ds::launch_tile_ranges(c->keys[res].as<uint32_t>(), c->d_K(), kcap, DB, c->ranges.as<uint2>(), st));
    }

    c->plan.valid = true;
    c->plan.soup = plan_soup;
    c->plan.devcam = cams == nullptr;
    c->plan.n_views = vt.n;
    if (cams)
        c->plan.cams.assign(cams, cams + vt.n);
    else
        c->plan.cams.clear();
    c->plan.DB = DB;
    c->plan.res = res;
    c->plan.kcap = kcap;
    c->plan.n_tiles = n_tiles;
    return DS_OK;
}

// Every view of one soup.
ds_status prepare(ds_ctx* c, int32_t soup_id, Soup& s, const ds_camera* cams, ds::ViewTable& vt, bool sync,
                  cudaStream_t st) {
    Soup* soups[DS_MAX_VIEWS];
    for (int v = 0; v < vt.n; ++v) soups[v] = &s;
    return prepare(c, soup_id, soups, cams, vt, sync, st);
}

bool plan_matches(const ds_ctx* c, int32_t soup_id, const ds_camera* cams, int32_t n_views) {
    if (!c->plan.valid || c->plan.devcam || c->plan.soup != soup_id || (int)c->plan.cams.size() != n_views) return false;
    return std::memcmp(c->plan.cams.data(), cams, sizeof(ds_camera) * n_views) == 0;
}

}  // namespace

extern "C" {

int32_t ds_version(void) { return 100; }

const char* ds_last_error(void) { return g_err.c_str(); }

ds_status ds_create(ds_ctx** out, int32_t device) {
    if (!out) return fail(DS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return fail(DS_ERR_CUDA, "no CUDA device available");
    }
    if (device < 0 || device >= n) return fail(DS_ERR_INVALID_ARG, "bad device index");
    ds_ctx* c = new (std::nothrow) ds_ctx();
    if (!c) return fail(DS_ERR_OOM, "host allocation failed");
    c->vt = new (std::nothrow) ds::ViewTable[2]();
    if (!c->vt) {
        delete c;
        return fail(DS_ERR_OOM, "host allocation failed");
    }
    c->device = device;
    DeviceGuard g(device);
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_word), 64, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        delete[] c->vt;
        delete c;
        return fail(DS_ERR_CUDA, "cudaHostAlloc failed");
    }
    if (c->misc.ensure(256, "context words") != DS_OK) {
        cudaFreeHost(c->h_word);
        delete[] c->vt;
        delete c;
        return DS_ERR_OOM;
    }
    cudaMemset(c->misc.p, 0, c->misc.cap);
    *out = c;
    return DS_OK;
}

void ds_destroy(ds_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (Soup& s : c->soups) {
        if (s.own) cudaFree(s.own);
        if (s.act) cudaFree(s.act);
    }
    DevBuf* bufs[] = {&c->recs,  &c->counts,  &c->offs,      &c->tbox,   &c->zkeys,   &c->keys[0], &c->keys[1],
                      &c->vals[0], &c->vals[1], &c->hist, &c->hist_scan, &c->ranges, &c->scanbuf, &c->misc,
                      &c->geom, &c->acc_tex, &c->acc_verts, &c->shade_part, &c->plan_dev};
    for (DevBuf* b : bufs) b->release();
    if (c->h_word) cudaFreeHost(c->h_word);
    for (auto& r : c->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    delete[] c->vt;
    delete c;
}

}  // extern "C"

namespace {
// Registration of a soup: plain (r_min = r_max = -1, tex [T][V][C]) or
// multi-resolution (tex = levels r_min..r_max, grid_n = 2^r_max).
ds_status upload_impl(ds_ctx* c, const float* verts, const float* tex, int32_t T, int32_t grid_n, int32_t C,
                      int32_t r_min, int32_t r_max, uint32_t flags, int32_t* soup_id, void* stream) {
    if (!c || !verts || !tex || !soup_id) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    if (C < 2 || C > DS_MAX_CHANNELS) return fail(DS_ERR_INVALID_ARG, "C out of range");
    if ((flags & ~(DS_BORROW | DS_STATIC)) != 0) return fail(DS_ERR_INVALID_ARG, "bad flags");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Soup s;
    s.T = T;
    s.N = grid_n;
    s.C = C;
    s.V = (grid_n + 1) * (grid_n + 2) / 2;
    s.r_min = r_min;
    s.r_max = r_max;
    const size_t nv = 9 * (size_t)T, nt = s.tex_floats(), nact = (size_t)T * s.V * C;
    if (cudaMalloc(reinterpret_cast<void**>(&s.act), sizeof(float) * (nact + (size_t)T * s.V)) != cudaSuccess) {
        cudaGetLastError();
        return fail(DS_ERR_OOM, "cudaMalloc failed for activations");
    }
    s.fixed = (flags & DS_STATIC) != 0;
    if ((flags & DS_BORROW) == 0) {
        if (cudaMalloc(reinterpret_cast<void**>(&s.own), sizeof(float) * (nv + nt + 4)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(s.act);
            return fail(DS_ERR_OOM, "cudaMalloc failed for the soup copy");
        }
        float* tex_dst = s.own + ((nv + 3) & ~size_t(3));   // 16-byte aligned texture copy
        DS_TRY_CUDA(cudaMemcpyAsync(s.own, verts, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
        DS_TRY_CUDA(cudaMemcpyAsync(tex_dst, tex, sizeof(float) * nt, cudaMemcpyDeviceToDevice, st));
        s.verts = s.own;
        s.tex = tex_dst;
        s.owned = true;
    } else {
        s.verts = verts;
        s.tex = tex;
    }
    s.live = true;
    int id = -1;
    for (int i = 0; i < (int)c->soups.size(); ++i)
        if (!c->soups[i].live) {
            id = i;
            break;
        }
    if (id < 0) {
        id = (int)c->soups.size();
        c->soups.push_back(s);
    } else {
        c->soups[id] = s;
    }
    if (c->plan.soup == id) c->plan.valid = false;
    *soup_id = id;
    return DS_OK;
}
}  // namespace

extern "C" {

ds_status ds_soup_upload(ds_ctx* c, const float* verts, const float* tex, int32_t T, int32_t grid_n, int32_t C,
                         uint32_t flags, int32_t* soup_id, void* stream) {
    if (grid_n < 1 || grid_n > DS_MAX_GRID_N) return fail(DS_ERR_INVALID_ARG, "grid_n out of range");
    return upload_impl(c, verts, tex, T, grid_n, C, -1, -1, flags, soup_id, stream);
}

ds_status ds_soup_upload_levels(ds_ctx* c, const float* verts, const float* tex_levels, int32_t T, int32_t r_min,
                                int32_t r_max, int32_t C, uint32_t flags, int32_t* soup_id, void* stream) {
    if (r_min < 0 || r_min > r_max || (1 << r_max) > DS_MAX_GRID_N)
        return fail(DS_ERR_INVALID_ARG, "levels must satisfy 0 <= r_min <= r_max, 2^r_max <= DS_MAX_GRID_N");
    return upload_impl(c, verts, tex_levels, T, 1 << r_max, C, r_min, r_max, flags, soup_id, stream);
}

ds_status ds_levels_compose(const float* levels, int32_t T, int32_t r_min, int32_t r_max, int32_t C, int32_t activate,
                            float* out, void* stream) {
    if (!levels || !out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    if (C < 1 || C > DS_MAX_CHANNELS) return fail(DS_ERR_INVALID_ARG, "C out of range");
    if (r_min < 0 || r_min > r_max || (1 << r_max) > DS_MAX_GRID_N) return fail(DS_ERR_INVALID_ARG, "bad levels");
    DS_TRY_CUDA(ds::launch_compose(levels, T, r_min, r_max, C, out, activate != 0, nullptr,
                                   static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

ds_status ds_levels_resample(const float* src, int32_t T, int32_t r_src, int32_t C, float* dst, int32_t r_dst,
                             void* stream) {
    if (!src || !dst) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    if (C < 1 || C > DS_MAX_CHANNELS) return fail(DS_ERR_INVALID_ARG, "C out of range");
    if (r_src < 0 || r_dst < 0 || (1 << r_src) > DS_MAX_GRID_N || (1 << r_dst) > DS_MAX_GRID_N)
        return fail(DS_ERR_INVALID_ARG, "bad levels");
    DS_TRY_CUDA(ds::launch_resample(src, T, r_src, C, dst, r_dst, static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

ds_status ds_soup_free(ds_ctx* c, int32_t soup_id) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    cudaDeviceSynchronize();
    if (s->own) cudaFree(s->own);
    if (s->act) cudaFree(s->act);
    *s = Soup();
    if (c->plan.soup == soup_id) c->plan.valid = false;
    return DS_OK;
}

}  // extern "C"

namespace {

}  // namespace

namespace ds {
ds_status check_outputs(const ds_view_out* out, int32_t n_views) {
    if (n_views < 1 || n_views > DS_MAX_VIEWS) return fail(DS_ERR_INVALID_ARG, "n_views out of range");
    if (!out) return fail(DS_ERR_INVALID_ARG, "out is NULL");
    for (int v = 0; v < n_views; ++v) {
        if (!out[v].gbuf || !out[v].color) return fail(DS_ERR_INVALID_ARG, "view output buffer is NULL");
        if (((uintptr_t)out[v].gbuf & 15) != 0) return fail(DS_ERR_INVALID_ARG, "gbuf must be 16-byte aligned");
    }
    return DS_OK;
}

}  // namespace ds

using ds::check_outputs;

namespace {

ds_status check_mode(uint32_t mode, bool have_seeds) {
    const uint32_t base_mode = mode & 0xffu;
    if (base_mode != DS_MODE_STOCHASTIC && base_mode != DS_MODE_THRESHOLD_HALF)
        return fail(DS_ERR_INVALID_ARG, "bad mode");
    if ((mode & ~(0xffu | DS_NO_SYNC)) != 0) return fail(DS_ERR_INVALID_ARG, "unknown mode bits");
    if (!have_seeds && base_mode == DS_MODE_STOCHASTIC) return fail(DS_ERR_INVALID_ARG, "seeds is NULL");
    return DS_OK;
}

ds_status check_gin(const ds_view_out* fwd, const ds_view_gin* gin, int32_t n_views, uint32_t grad_flags) {
    if ((grad_flags & ~(DS_G_ALL | DS_REUSE_FORWARD | DS_OVERWRITE)) != 0)
        return fail(DS_ERR_INVALID_ARG, "unknown gradient flags");
    if (!fwd || !gin) return fail(DS_ERR_INVALID_ARG, "fwd or gin is NULL");
    if (n_views < 1 || n_views > DS_MAX_VIEWS) return fail(DS_ERR_INVALID_ARG, "n_views out of range");
    const bool need_color = (grad_flags & (DS_G_TEX | DS_G_INTERIOR | DS_G_EDGE)) != 0;
    for (int v = 0; v < n_views; ++v) {
        if (!fwd[v].gbuf) return fail(DS_ERR_INVALID_ARG, "fwd gbuf is NULL");
        if (((uintptr_t)fwd[v].gbuf & 15) != 0) return fail(DS_ERR_INVALID_ARG, "gbuf must be 16-byte aligned");
        if (need_color && !gin[v].grad_color) return fail(DS_ERR_INVALID_ARG, "grad_color is NULL");
        if ((grad_flags & DS_G_EDGE) && !fwd[v].color) return fail(DS_ERR_INVALID_ARG, "fwd color is NULL");
    }
    return DS_OK;
}

// Persistent grid of the tile kernels: the tuning's CTAs per SM, or 0 (the
// occupancy limit of each kernel).
int tile_grid(const ds_ctx* c, const ds::ViewTable& vt) {
    return c->tune.blocks_per_sm > 0 ? ds::persistent_grid(vt.n_items, c->tune.blocks_per_sm) : 0;
}

// Forward after validation; vt is filled.  host_cams is NULL for device cameras.
ds_status forward_impl(ds_ctx* c, int32_t soup_id, Soup& s, const ds_camera* host_cams, uint32_t mode, const float* bg,
                       const ds_view_out* out, cudaStream_t st) {
    ds::ViewTable& vt = *c->vt;
    DS_TRY(prepare(c, soup_id, s, host_cams, vt, (mode & DS_NO_SYNC) == 0, st));
    ds::Bg b{};
    for (int i = 0; i < s.C - 1; ++i) b.c[i] = bg[i];
    const ds::SoupDev sd = soup_dev(s);
    const int grid = tile_grid(c, vt);
    {
        StageScope p(c, ds::kStRasterFwd, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter(), 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_fwd(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                          c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB,
                                          mode & 0xffu, b, c->d_counter(), grid, st));
    }
    bool want_front = false;
    for (int v = 0; v < vt.n; ++v) want_front = want_front || out[v].n_front;
    if (want_front) {
        StageScope p(c, ds::kStCount, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 1, 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_count(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                            c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB, 0,
                                            nullptr, c->d_counter() + 1, grid, st));
    }
    return DS_OK;
}

// Arguments of the fused training pass (forward + L2 loss in the same kernel
// as the texture, score and interior gradients).
struct FusedL2 {
    uint32_t mode;
    ds::Bg bg;
    float scale;
    float* loss;
    // Schedule.  Full fusion (one kernel for forward, loss and the texture,
    // score and interior terms) for groups of one sample; for larger sample
    // groups the forward with the loss epilogue and the backward kernel run
    // as two launches, because holding a group's forward and backward state
    // in one kernel spills registers (measured slower on the 1080p batch).
    bool split;
};

// Backward after validation; vt is filled and the plan is current.  With
// `fused` the forward has not run: the fused kernel renders, evaluates the
// loss and takes the texture, score and interior terms in one pass.
ds_status backward_impl(ds_ctx* c, Soup& s, uint32_t grad_flags, float* grad_verts, float* grad_tex, cudaStream_t st,
                        const FusedL2* fused = nullptr, const ds::AdamTex* tex_adam = nullptr) {
    ds::ViewTable& vt = *c->vt;
    const int n_views = vt.n;
    const ds::SoupDev sd = soup_dev(s);
    const int grid = tile_grid(c, vt);
    const uint32_t gflags = grad_flags & DS_G_ALL;
    const size_t n_tex = (size_t)s.T * s.V * s.C, n_verts = 9 * (size_t)s.T;
    const bool want_tex = (grad_tex || tex_adam) && (gflags & (DS_G_TEX | DS_G_SCORE));
    const bool want_verts = grad_verts && (gflags & (DS_G_INTERIOR | DS_G_EDGE));
    const bool overwrite = (grad_flags & DS_OVERWRITE) != 0;
    double* acc_tex = nullptr;
    double* acc_verts = nullptr;
    if (want_tex) {
        DS_TRY(c->acc_tex.ensure(sizeof(double) * n_tex, "texture gradient accumulator"));
        acc_tex = c->acc_tex.as<double>();
        DS_TRY_CUDA(cudaMemsetAsync(acc_tex, 0, sizeof(double) * n_tex, st));
    }
    if (want_verts) {
        DS_TRY(c->acc_verts.ensure(sizeof(double) * n_verts, "vertex gradient accumulator"));
        acc_verts = c->acc_verts.as<double>();
        DS_TRY_CUDA(cudaMemsetAsync(acc_verts, 0, sizeof(double) * n_verts, st));
        DS_TRY(c->geom.ensure(sizeof(ds::GeomRec) * (size_t)n_views * s.T, "vertex-gradient geometry"));
        StageScope p(c, ds::kStGeom, st);
        DS_TRY_CUDA(ds::launch_geom(vt, sd, c->geom.as<ds::GeomRec>(), st));
    }
    if (fused && fused->split) {
        // split schedule: forward with the loss epilogue, then the backward
        {
            StageScope p(c, ds::kStRasterFwd, st);
            DS_TRY_CUDA(cudaMemsetAsync(c->d_counter(), 0, 4, st));
            DS_TRY_CUDA(ds::launch_raster_fwd(vt, sd, c->recs.as<ds::SetupRec>(),
                                              c->keys[c->plan.res].as<uint32_t>(), c->vals[c->plan.res].as<uint32_t>(),
                                              c->ranges.as<uint2>(), c->plan.DB, fused->mode & 0xffu, fused->bg,
                                              c->d_counter(), grid, st, true, fused->scale, fused->loss));
        }
        if (want_tex || (want_verts && (gflags & DS_G_INTERIOR))) {
            StageScope p(c, ds::kStRasterBwd, st);
            DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 2, 0, 4, st));
            DS_TRY_CUDA(ds::launch_raster_bwd(vt, sd, c->recs.as<ds::SetupRec>(),
                                              c->keys[c->plan.res].as<uint32_t>(), c->vals[c->plan.res].as<uint32_t>(),
                                              c->ranges.as<uint2>(), c->plan.DB, gflags, c->geom.as<ds::GeomRec>(),
                                              acc_tex, acc_verts, c->d_counter() + 2, grid, st));
        }
    } else if (fused) {
        StageScope p(c, ds::kStTrain, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 2, 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_train(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                            c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB,
                                            fused->mode & 0xffu, fused->bg, fused->scale, fused->loss, gflags,
                                            c->geom.as<ds::GeomRec>(), acc_tex, acc_verts, c->d_counter() + 2, grid,
                                            st));
    } else if (want_tex || (want_verts && (gflags & DS_G_INTERIOR))) {
        StageScope p(c, ds::kStRasterBwd, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 2, 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_bwd(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                          c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB,
                                          gflags, c->geom.as<ds::GeomRec>(), acc_tex, acc_verts, c->d_counter() + 2,
                                          grid, st));
    }
    if (want_verts && (gflags & DS_G_EDGE)) {
        StageScope p(c, ds::kStEdgeBwd, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 3, 0, 4, st));
        ds::ViewTable& ve = c->vt[1];
        retile(vt, kEdgeTileW, ve);
        DS_TRY_CUDA(ds::launch_edge_bwd(ve, sd, c->recs.as<ds::SetupRec>(), c->geom.as<ds::GeomRec>(), acc_verts,
                                        c->d_counter() + 3, tile_grid(c, ve), st));
    }
    {
        StageScope p(c, ds::kStFinish, st);
        if (want_tex && tex_adam && s.levels())
            DS_TRY_CUDA(ds::launch_restrict_adam(acc_tex, s.T, s.r_min, s.r_max, s.C, *tex_adam, st));
        else if (want_tex && tex_adam)
            DS_TRY_CUDA(ds::launch_grad_finish_adam(acc_tex, *tex_adam, (long long)n_tex, st));
        else if (want_tex && s.levels())
            DS_TRY_CUDA(ds::launch_restrict(acc_tex, s.T, s.r_min, s.r_max, s.C, grad_tex, overwrite, st));
        else if (want_tex)
            DS_TRY_CUDA(ds::launch_grad_finish(acc_tex, grad_tex, (long long)n_tex, overwrite, st));
        else if (grad_tex && overwrite)
            DS_TRY_CUDA(cudaMemsetAsync(grad_tex, 0, sizeof(float) * s.tex_floats(), st));
        if (want_verts) DS_TRY_CUDA(ds::launch_grad_finish(acc_verts, grad_verts, (long long)n_verts, overwrite, st));
        else if (grad_verts && overwrite) DS_TRY_CUDA(cudaMemsetAsync(grad_verts, 0, sizeof(float) * n_verts, st));
    }
    return DS_OK;
}

// Loss views of the fused training pass: targets present, gradients
// written; the table's gradient pointers are the pass's outputs.
ds_status set_loss_views(ds::ViewTable& vt, const ds_view_loss* lv) {
    if (!lv) return fail(DS_ERR_INVALID_ARG, "loss views are NULL");
    for (int v = 0; v < vt.n; ++v) {
        if (!lv[v].target || !lv[v].grad_color) return fail(DS_ERR_INVALID_ARG, "target or grad_color is NULL");
        vt.v[v].target = lv[v].target;
        vt.v[v].grad_color = lv[v].grad_color;
        vt.v[v].score_w = lv[v].score_w;
    }
    return DS_OK;
}

ds_status train_impl(ds_ctx* c, int32_t soup_id, Soup& s, const ds_camera* host_cams, uint32_t mode, const float* bg,
                     const ds_view_out* out, float scale, float* loss, uint32_t grad_flags, float* grad_verts,
                     float* grad_tex, cudaStream_t st) {
    for (int v = 0; v < c->vt->n; ++v)
        if (out[v].n_front) return fail(DS_ERR_INVALID_ARG, "the fused training pass does not write n_front");
    DS_TRY(prepare(c, soup_id, s, host_cams, *c->vt, (mode & DS_NO_SYNC) == 0, st));
    FusedL2 f{};
    f.mode = mode;
    for (int i = 0; i < s.C - 1; ++i) f.bg.c[i] = bg[i];
    f.scale = scale;
    f.loss = loss;
    f.split = c->vt->S > 1;
    return backward_impl(c, s, grad_flags, grad_verts, grad_tex, st, &f);
}

// View table for device-resident cameras: sizes from the host, cameras and
// seeds read by the kernels from device memory.
ds_status build_table_devcam(ds::ViewTable& vt, const ds_tuning& tu, const int32_t* wh, const ds_camera* dcams,
                             const uint64_t* dseeds,
                             int32_t n_views, int32_t S, const ds_view_out* out, const ds_view_gin* gin) {
    if (!wh || !dcams) return fail(DS_ERR_INVALID_ARG, "wh or cams is NULL");
    if (n_views < 1 || n_views > DS_MAX_VIEWS) return fail(DS_ERR_INVALID_ARG, "n_views out of range");
    if (S < 1 || S > DS_MAX_SAMPLES) return fail(DS_ERR_INVALID_ARG, "S must be in [1, 64]");
    static thread_local std::vector<ds_camera> tmp;
    tmp.assign(n_views, ds_camera{});
    for (int v = 0; v < n_views; ++v) {
        if (wh[2 * v] < 1 || wh[2 * v + 1] < 1 || wh[2 * v] > DS_MAX_RESOLUTION || wh[2 * v + 1] > DS_MAX_RESOLUTION)
            return fail(DS_ERR_INVALID_ARG, "view size out of range");
        tmp[v].width = wh[2 * v];
        tmp[v].height = wh[2 * v + 1];
    }
    build_table(vt, tu, tmp.data(), nullptr, n_views, S, out, gin);
    vt.dcam = dcams;
    vt.dseed = reinterpret_cast<const unsigned long long*>(dseeds);
    return DS_OK;
}

}  // namespace

extern "C" {

ds_status ds_raster_forward(ds_ctx* c, int32_t soup_id, const ds_camera* cams, const uint64_t* seeds, int32_t n_views,
                            int32_t S, uint32_t mode, const float* bg, const ds_view_out* out, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_views(cams, n_views, S));
    DS_TRY(check_mode(mode, seeds != nullptr));
    if (!bg) return fail(DS_ERR_INVALID_ARG, "bg is NULL");
    DS_TRY(check_outputs(out, n_views));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    build_table(*c->vt, c->tune, cams, seeds, n_views, S, out, nullptr);   // calls on one context are serialised
    return forward_impl(c, soup_id, *s, cams, mode, bg, out, st);
}

ds_status ds_raster_forward_multi(ds_ctx* c, const int32_t* soup_ids, const ds_camera* cams, const uint64_t* seeds,
                                  int32_t n_views, int32_t S, uint32_t mode, const float* bg, const ds_view_out* out,
                                  void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    if (!soup_ids) return fail(DS_ERR_INVALID_ARG, "soup_ids is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    DS_TRY(check_views(cams, n_views, S));
    DS_TRY(check_mode(mode, seeds != nullptr));
    if (!bg) return fail(DS_ERR_INVALID_ARG, "bg is NULL");
    DS_TRY(check_outputs(out, n_views));
    Soup* soups[DS_MAX_VIEWS];
    for (int v = 0; v < n_views; ++v) {
        DS_TRY(get_soup(c, soup_ids[v], &soups[v]));
        if (soups[v]->N != soups[0]->N || soups[v]->C != soups[0]->C)
            return fail(DS_ERR_INVALID_ARG, "the soups of one multi-soup forward must share grid_n and C");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    ds::ViewTable& vt = *c->vt;
    build_table(vt, c->tune, cams, seeds, n_views, S, out, nullptr);
    DS_TRY(prepare(c, -1, soups, cams, vt, (mode & DS_NO_SYNC) == 0, st));
    const Soup& s0 = *soups[0];
    ds::Bg b{};
    for (int i = 0; i < s0.C - 1; ++i) b.c[i] = bg[i];
    const ds::SoupDev sd = soup_dev(s0);   // N, C, V; the views read their own soups
    const int grid = tile_grid(c, vt);
    {
        StageScope p(c, ds::kStRasterFwd, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter(), 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_fwd(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                          c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB,
                                          mode & 0xffu, b, c->d_counter(), grid, st, false, 0.f, nullptr, true));
    }
    bool want_front = false;
    for (int v = 0; v < vt.n; ++v) want_front = want_front || out[v].n_front;
    if (want_front) {
        StageScope p(c, ds::kStCount, st);
        DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 1, 0, 4, st));
        DS_TRY_CUDA(ds::launch_raster_count(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                            c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB, 0,
                                            nullptr, c->d_counter() + 1, grid, st));
    }
    return DS_OK;
}

ds_status ds_raster_forward_devcam(ds_ctx* c, int32_t soup_id, const int32_t* wh, const ds_camera* cams,
                                   const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode, const float* bg,
                                   const ds_view_out* out, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_mode(mode, seeds != nullptr));
    if (!bg) return fail(DS_ERR_INVALID_ARG, "bg is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    DS_TRY(build_table_devcam(*c->vt, c->tune, wh, cams, seeds, n_views, S, out, nullptr));   // validates n_views
    DS_TRY(check_outputs(out, n_views));
    return forward_impl(c, soup_id, *s, nullptr, mode, bg, out, st);
}

ds_status ds_raster_backward(ds_ctx* c, int32_t soup_id, const ds_camera* cams, int32_t n_views, int32_t S,
                             const ds_view_out* fwd, const ds_view_gin* gin, uint32_t grad_flags, float* grad_verts,
                             float* grad_tex, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_views(cams, n_views, S));
    DS_TRY(check_gin(fwd, gin, n_views, grad_flags));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    build_table(*c->vt, c->tune, cams, nullptr, n_views, S, fwd, gin);
    if (!((grad_flags & DS_REUSE_FORWARD) && plan_matches(c, soup_id, cams, n_views)))
        DS_TRY(prepare(c, soup_id, *s, cams, *c->vt, true, st));
    return backward_impl(c, *s, grad_flags, grad_verts, grad_tex, st);
}

ds_status ds_raster_backward_adam(ds_ctx* c, int32_t soup_id, const ds_camera* cams, int32_t n_views, int32_t S,
                                  const ds_view_out* fwd, const ds_view_gin* gin, uint32_t grad_flags,
                                  float* grad_verts, const ds_adam_args* tex_adam, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    if (!tex_adam || !tex_adam->m || !tex_adam->v) return fail(DS_ERR_INVALID_ARG, "NULL Adam state");
    if (tex_adam->step < 1) return fail(DS_ERR_INVALID_ARG, "step must be >= 1");
    if (!(tex_adam->beta1 >= 0.f && tex_adam->beta1 < 1.f && tex_adam->beta2 >= 0.f && tex_adam->beta2 < 1.f &&
          tex_adam->eps >= 0.f) || !std::isfinite(tex_adam->lr))
        return fail(DS_ERR_INVALID_ARG, "bad hyperparameters");
    if (!(grad_flags & (DS_G_TEX | DS_G_SCORE))) return fail(DS_ERR_INVALID_ARG, "no texture gradient term selected");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    if (s->fixed) return fail(DS_ERR_INVALID_ARG, "the soup is static (DS_STATIC): its texture cannot be updated");
    if (tex_adam->n != (int64_t)s->tex_floats())
        return fail(DS_ERR_INVALID_ARG, "m and v must hold " + std::to_string(s->tex_floats()) + " values");
    if (s->levels() && (s->C % 4 != 0 || (((uintptr_t)s->tex | (uintptr_t)tex_adam->m | (uintptr_t)tex_adam->v) & 15)))
        return fail(DS_ERR_INVALID_ARG, "a level soup's fused Adam needs C a multiple of 4 and 16-byte-aligned "
                                        "texture, m and v");
    DS_TRY(check_views(cams, n_views, S));
    DS_TRY(check_gin(fwd, gin, n_views, grad_flags));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    build_table(*c->vt, c->tune, cams, nullptr, n_views, S, fwd, gin);
    if (!((grad_flags & DS_REUSE_FORWARD) && plan_matches(c, soup_id, cams, n_views)))
        DS_TRY(prepare(c, soup_id, *s, cams, *c->vt, true, st));
    const ds::AdamTex at{const_cast<float*>(s->tex), tex_adam->m, tex_adam->v,
                         ds::make_adam(tex_adam->lr, tex_adam->beta1, tex_adam->beta2, tex_adam->eps,
                                       (long long)tex_adam->step)};
    return backward_impl(c, *s, grad_flags, grad_verts, nullptr, st, nullptr, &at);
}

ds_status ds_raster_backward_devcam(ds_ctx* c, int32_t soup_id, const int32_t* wh, const ds_camera* cams,
                                    int32_t n_views, int32_t S, const ds_view_out* fwd, const ds_view_gin* gin,
                                    uint32_t grad_flags, float* grad_verts, float* grad_tex, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_gin(fwd, gin, n_views, grad_flags));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    DS_TRY(build_table_devcam(*c->vt, c->tune, wh, cams, nullptr, n_views, S, fwd, gin));
    const bool reuse = (grad_flags & DS_REUSE_FORWARD) && c->plan.valid && c->plan.devcam && c->plan.soup == soup_id &&
                       c->plan.n_tiles == total_tiles(*c->vt) && c->plan.n_views == n_views;
    if (!reuse) DS_TRY(prepare(c, soup_id, *s, nullptr, *c->vt, true, st));
    return backward_impl(c, *s, grad_flags, grad_verts, grad_tex, st);
}

ds_status ds_reserve(ds_ctx* c, int64_t pairs) {
    if (!c || pairs < 0 || pairs > 0x7fffffffLL) return fail(DS_ERR_INVALID_ARG, "bad context or pair count");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    const size_t K = (size_t)(pairs > 0 ? pairs : 1);
    for (int b = 0; b < 2; ++b) {
        DS_TRY(c->keys[b].ensure(4 * K, "bin keys"));
        DS_TRY(c->vals[b].ensure(4 * K, "bin values"));
    }
    const size_t nblk = (K + ds::kSortBlock - 1) / ds::kSortBlock;
    DS_TRY(c->hist.ensure(4 * 256 * nblk, "radix histogram"));
    DS_TRY(c->hist_scan.ensure(4 * 256 * nblk, "radix offsets"));
    DS_TRY(ensure_scan(c, (int64_t)(256 * nblk)));
    return DS_OK;
}

ds_status ds_fragment_count(ds_ctx* c, int32_t soup_id, const ds_camera* cams, int32_t n_views,
                            int64_t* n_cover_total, void* stream) {
    if (!c || !n_cover_total) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_views(cams, n_views, 1));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    ds::ViewTable& vt = *c->vt;
    build_table(vt, c->tune, cams, nullptr, n_views, 1, nullptr, nullptr);
    DS_TRY(prepare(c, soup_id, *s, cams, vt, true, st));
    const ds::SoupDev sd = soup_dev(*s);
    const int grid = tile_grid(c, vt);
    DS_TRY_CUDA(cudaMemsetAsync(c->d_total(), 0, 8, st));
    DS_TRY_CUDA(cudaMemsetAsync(c->d_counter() + 4, 0, 4, st));
    DS_TRY_CUDA(ds::launch_raster_count(vt, sd, c->recs.as<ds::SetupRec>(), c->keys[c->plan.res].as<uint32_t>(),
                                        c->vals[c->plan.res].as<uint32_t>(), c->ranges.as<uint2>(), c->plan.DB, 1,
                                        c->d_total(), c->d_counter() + 4, grid, st));
    DS_TRY_CUDA(cudaMemcpyAsync(c->h_word, c->d_total(), 8, cudaMemcpyDeviceToHost, st));
    DS_TRY_CUDA(cudaStreamSynchronize(st));
    uint64_t v = 0;
    std::memcpy(&v, c->h_word, 8);
    *n_cover_total = (int64_t)v;
    return DS_OK;
}

ds_status ds_profile_enable(ds_ctx* c, int32_t on) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    c->prof_on = on != 0;
    return DS_OK;
}

int32_t ds_profile_stages(void) { return ds::kNumStages; }

ds_status ds_profile_read(ds_ctx* c, int32_t stage, const char** name, int64_t* launches, double* ms) {
    if (!c || stage < 0 || stage >= ds::kNumStages) return fail(DS_ERR_INVALID_ARG, "bad context or stage");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    DS_TRY(prof_flush(c));
    if (name) *name = ds::kStageNames[stage];
    if (launches) *launches = c->prof_n[stage];
    if (ms) *ms = c->prof_ms[stage];
    return DS_OK;
}

ds_status ds_profile_reset(ds_ctx* c) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    DS_TRY(prof_flush(c));
    for (int i = 0; i < ds::kNumStages; ++i) {
        c->prof_ms[i] = 0.0;
        c->prof_n[i] = 0;
    }
    return DS_OK;
}

int64_t ds_kernel_launches(void) { return ds::launches_total(); }

ds_status ds_plan_stats(ds_ctx* c, int64_t* pairs, int64_t* tiles) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    if (pairs) *pairs = c->plan.valid ? (int64_t)c->plan.kcap : 0;
    if (tiles) *tiles = c->plan.valid ? (int64_t)c->plan.n_tiles : 0;
    return DS_OK;
}

ds_status ds_ctx_status(ds_ctx* c) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    DS_TRY_CUDA(cudaStreamSynchronize(c->last_stream));
    int st = 0;
    DS_TRY_CUDA(cudaMemcpy(&st, c->d_status(), 4, cudaMemcpyDeviceToHost));
    DS_TRY_CUDA(cudaMemset(c->d_status(), 0, 4));
    if (st & 1) return fail(DS_ERR_CAPACITY, "bin capacity exceeded in a DS_NO_SYNC forward");
    if (st & 2) return fail(DS_ERR_TIMEOUT, "a tensor-core shading launch timed out waiting for its MMAs");
    return DS_OK;
}

ds_status ds_set_tuning(ds_ctx* c, const ds_tuning* t) {
    if (!c || !t) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (t->tile_w != 8 && t->tile_w != 16 && t->tile_w != 32) return fail(DS_ERR_INVALID_ARG, "tile_w must be 8, 16 or 32");
    if (t->depth_bits < -1 || t->depth_bits > 16) return fail(DS_ERR_INVALID_ARG, "depth_bits must be in [-1, 16]");
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 8) return fail(DS_ERR_INVALID_ARG, "blocks_per_sm must be in [0, 8]");
    if (t->chunk < 32 || t->chunk > ds::kChunk || t->chunk % 32 != 0)
        return fail(DS_ERR_INVALID_ARG, "chunk must be a multiple of 32 in [32, 256]");
    std::lock_guard<std::mutex> lk(c->mu);
    c->tune = *t;
    c->plan.valid = false;   // the next pass bins again with the new tile shape
    return DS_OK;
}

ds_status ds_get_tuning(ds_ctx* c, ds_tuning* t) {
    if (!c || !t) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    *t = c->tune;
    return DS_OK;
}

ds_status ds_raster_train_l2(ds_ctx* c, int32_t soup_id, const ds_camera* cams, const uint64_t* seeds,
                             int32_t n_views, int32_t S, uint32_t mode, const float* bg, const ds_view_out* out,
                             const ds_view_loss* lv, float scale, float* loss, uint32_t grad_flags, float* grad_verts,
                             float* grad_tex, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_views(cams, n_views, S));
    DS_TRY(check_mode(mode, seeds != nullptr));
    if (!bg) return fail(DS_ERR_INVALID_ARG, "bg is NULL");
    DS_TRY(check_outputs(out, n_views));
    if (!std::isfinite(scale)) return fail(DS_ERR_INVALID_ARG, "scale is not finite");
    if ((grad_flags & ~(DS_G_ALL | DS_OVERWRITE)) != 0) return fail(DS_ERR_INVALID_ARG, "unknown gradient flags");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    build_table(*c->vt, c->tune, cams, seeds, n_views, S, out, nullptr);
    DS_TRY(set_loss_views(*c->vt, lv));
    return train_impl(c, soup_id, *s, cams, mode, bg, out, scale, loss, grad_flags, grad_verts, grad_tex, st);
}

ds_status ds_raster_train_l2_devcam(ds_ctx* c, int32_t soup_id, const int32_t* wh, const ds_camera* cams,
                                    const uint64_t* seeds, int32_t n_views, int32_t S, uint32_t mode, const float* bg,
                                    const ds_view_out* out, const ds_view_loss* lv, float scale, float* loss,
                                    uint32_t grad_flags, float* grad_verts, float* grad_tex, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    Soup* s = nullptr;
    DS_TRY(get_soup(c, soup_id, &s));
    DS_TRY(check_mode(mode, seeds != nullptr));
    if (!bg) return fail(DS_ERR_INVALID_ARG, "bg is NULL");
    if (!std::isfinite(scale)) return fail(DS_ERR_INVALID_ARG, "scale is not finite");
    if ((grad_flags & ~(DS_G_ALL | DS_OVERWRITE)) != 0) return fail(DS_ERR_INVALID_ARG, "unknown gradient flags");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    DS_TRY(build_table_devcam(*c->vt, c->tune, wh, cams, seeds, n_views, S, out, nullptr));   // validates n_views
    DS_TRY(check_outputs(out, n_views));
    DS_TRY(set_loss_views(*c->vt, lv));
    return train_impl(c, soup_id, *s, nullptr, mode, bg, out, scale, loss, grad_flags, grad_verts, grad_tex, st);
}

}  // extern "C"

// Deferred shading (Sec. 3.3): view table of the shading kernels.
namespace {
ds_status shade_views(const ds_camera* cams, int32_t n_views, int32_t S, const float* params,
                      const float* const* feats, std::vector<ds::ShadeView>& v) {
    if (n_views == 0 && S >= 1 && S <= DS_MAX_SAMPLES && params) return DS_OK;
    DS_TRY(check_views(cams, n_views, S));
    if (!params) return fail(DS_ERR_INVALID_ARG, "params is NULL");
    if (!feats) return fail(DS_ERR_INVALID_ARG, "feats is NULL");
    v.resize(n_views);
    for (int i = 0; i < n_views; ++i) {
        if (!feats[i]) return fail(DS_ERR_INVALID_ARG, "feats[" + std::to_string(i) + "] is NULL");
        if (cams[i].fx == 0.f || cams[i].fy == 0.f)
            return fail(DS_ERR_INVALID_ARG, "camera " + std::to_string(i) + " has a zero focal length");
        ds::ShadeView& d = v[i];
        std::memset(&d, 0, sizeof(d));
        d.feat = feats[i];
        d.W = cams[i].width;
        d.H = cams[i].height;
        d.fx = cams[i].fx;
        d.fy = cams[i].fy;
        d.cx = cams[i].cx;
        d.cy = cams[i].cy;
        for (int k = 0; k < 9; ++k) d.R[k] = cams[i].R[k];
    }
    return DS_OK;
}
}  // namespace

extern "C" {

ds_status ds_shade_forward(ds_ctx* c, int32_t n_views, int32_t S, const ds_camera* cams, const float* params,
                           const float* const* feats, float* const* rgbs, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    std::vector<ds::ShadeView> v;
    DS_TRY(shade_views(cams, n_views, S, params, feats, v));
    if (n_views == 0) return DS_OK;
    if (!rgbs) return fail(DS_ERR_INVALID_ARG, "rgbs is NULL");
    for (int i = 0; i < n_views; ++i) {
        if (!rgbs[i]) return fail(DS_ERR_INVALID_ARG, "rgbs[" + std::to_string(i) + "] is NULL");
        v[i].rgb = rgbs[i];
    }
    if (c->shade_path == DS_SHADE_TENSOR_CORES || c->shade_path == DS_SHADE_TENSOR_CORES_WAIT_TEST)
        DS_TRY_CUDA(ds::launch_shade_fwd_tc(v.data(), n_views, S, params, c->d_status(),
                                            static_cast<cudaStream_t>(stream),
                                            c->shade_path == DS_SHADE_TENSOR_CORES_WAIT_TEST));
    else
        DS_TRY_CUDA(ds::launch_shade_fwd(v.data(), n_views, S, params, static_cast<cudaStream_t>(stream)));
    c->last_stream = static_cast<cudaStream_t>(stream);
    return DS_OK;
}

ds_status ds_set_shade_path(ds_ctx* c, int32_t path) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    if (path != DS_SHADE_CUDA_CORES && path != DS_SHADE_TENSOR_CORES && path != DS_SHADE_TENSOR_CORES_WAIT_TEST)
        return fail(DS_ERR_INVALID_ARG, "bad shade path");
    std::lock_guard<std::mutex> lk(c->mu);
    c->shade_path = path;
    return DS_OK;
}

ds_status ds_get_shade_path(ds_ctx* c, int32_t* path) {
    if (!c || !path) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    *path = c->shade_path;
    return DS_OK;
}

ds_status ds_shade_backward(ds_ctx* c, int32_t n_views, int32_t S, const ds_camera* cams, const float* params,
                            const float* const* feats, const float* const* grad_rgbs, float* const* grad_feats,
                            float* grad_params, uint32_t flags, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    if ((flags & ~DS_OVERWRITE) != 0) return fail(DS_ERR_INVALID_ARG, "unknown flags");
    std::vector<ds::ShadeView> v;
    DS_TRY(shade_views(cams, n_views, S, params, feats, v));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool overwrite = (flags & DS_OVERWRITE) != 0;
    if (n_views > 0) {
        if (!grad_rgbs) return fail(DS_ERR_INVALID_ARG, "grad_rgbs is NULL");
        for (int i = 0; i < n_views; ++i) {
            if (!grad_rgbs[i]) return fail(DS_ERR_INVALID_ARG, "grad_rgbs[" + std::to_string(i) + "] is NULL");
            v[i].grad_rgb = grad_rgbs[i];
            v[i].grad_feat = grad_feats ? grad_feats[i] : nullptr;
        }
    }
    const int grid = ds::shade_bwd_grid();
    DS_TRY(c->shade_part.ensure(sizeof(float) * ds::shade_partial_floats(grid), "shading gradient partials"));
    DS_TRY_CUDA(ds::launch_shade_bwd(v.data(), n_views, S, params, overwrite, c->shade_part.as<float>(), grid,
                                     grad_params, st));
    return DS_OK;
}

}  // extern "C"

extern "C" {

// Adaptive control of primitives (Sec. 3.4).
ds_status ds_coverage_count(const ds_gbuf* const* gbufs, const int32_t* hw, int32_t n_views, int32_t S, int32_t T,
                            int32_t* counts, void* stream) {
    if (!gbufs || !hw || !counts) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (n_views < 1 || n_views > DS_MAX_VIEWS) return fail(DS_ERR_INVALID_ARG, "n_views out of range");
    if (S < 1 || S > DS_MAX_SAMPLES) return fail(DS_ERR_INVALID_ARG, "S out of range");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    const int4* g[DS_MAX_VIEWS];
    long long n[DS_MAX_VIEWS];
    for (int v = 0; v < n_views; ++v) {
        if (!gbufs[v]) return fail(DS_ERR_INVALID_ARG, "gbufs[" + std::to_string(v) + "] is NULL");
        if (hw[2 * v] < 1 || hw[2 * v + 1] < 1 || hw[2 * v] > DS_MAX_RESOLUTION || hw[2 * v + 1] > DS_MAX_RESOLUTION)
            return fail(DS_ERR_INVALID_ARG, "bad view size");
        g[v] = reinterpret_cast<const int4*>(gbufs[v]);
        n[v] = (long long)S * hw[2 * v] * hw[2 * v + 1];
    }
    DS_TRY_CUDA(ds::launch_coverage(g, n, n_views, T, counts, static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

ds_status ds_edge_ratios(const float* verts, int32_t T, const ds_camera* cams, int32_t n_views, float* ratios,
                         void* stream) {
    if (!verts || !ratios) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    DS_TRY(check_views(cams, n_views, 1));
    DS_TRY_CUDA(ds::launch_edge_ratios(verts, T, cams, n_views, ratios, static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

ds_status ds_adapt_plan(const int32_t* counts, const float* ratios, int32_t T, float threshold, int64_t budget,
                        int32_t* plan, int32_t* n_out) {
    if (!counts || !ratios || !plan || !n_out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES / 2) return fail(DS_ERR_INVALID_ARG, "T out of range");
    if (!std::isfinite(threshold)) return fail(DS_ERR_INVALID_ARG, "threshold is not finite");
    *n_out = ds::adapt_plan(counts, ratios, T, threshold, (long long)budget, plan);
    return DS_OK;
}

ds_status ds_adapt_plan_fill(const int32_t* counts, const float* ratios, int32_t T, int64_t target, int32_t* plan,
                             int32_t* n_out) {
    if (!counts || !ratios || !plan || !n_out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES / 2) return fail(DS_ERR_INVALID_ARG, "T out of range");
    *n_out = ds::adapt_plan_fill(counts, ratios, T, (long long)target, plan);
    return DS_OK;
}

ds_status ds_soup_rebuild(ds_ctx* c, const float* verts, const float* tex, int32_t T, const int32_t* grid_ns,
                          int32_t n_levels, int32_t C, const int32_t* plan, int32_t n_out, float* verts_out,
                          float* tex_out, void* stream) {
    if (!c) return fail(DS_ERR_INVALID_ARG, "NULL context");
    if (!verts || !tex || !grid_ns || !verts_out || !tex_out || (n_out > 0 && !plan))
        return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || T >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "T out of range");
    if (n_out < 0 || n_out >= DS_MAX_TRIANGLES) return fail(DS_ERR_INVALID_ARG, "n_out out of range");
    if (n_levels < 1 || n_levels > 6) return fail(DS_ERR_INVALID_ARG, "n_levels must be in [1, 6]");
    if (C < 1 || C > DS_MAX_CHANNELS) return fail(DS_ERR_INVALID_ARG, "C out of range");
    for (int l = 0; l < n_levels; ++l)
        if (grid_ns[l] < 1 || grid_ns[l] > DS_MAX_GRID_N) return fail(DS_ERR_INVALID_ARG, "grid_n out of range");
    for (int k = 0; k < n_out; ++k)
        if ((plan[k] >> 3) < 0 || (plan[k] >> 3) >= T || (plan[k] & 7) > 6)
            return fail(DS_ERR_INVALID_ARG, "plan entry " + std::to_string(k) + " is invalid");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_out == 0) return DS_OK;
    DS_TRY(c->plan_dev.ensure(sizeof(int32_t) * (size_t)n_out, "rebuild plan"));
    DS_TRY_CUDA(cudaMemcpyAsync(c->plan_dev.p, plan, sizeof(int32_t) * (size_t)n_out, cudaMemcpyHostToDevice, st));
    DS_TRY_CUDA(ds::launch_rebuild(verts, tex, T, grid_ns, n_levels, C, c->plan_dev.as<int32_t>(), n_out, verts_out,
                                   tex_out, st));
    // the call returns with the rebuild complete (a once-per-round operation)
    DS_TRY_CUDA(cudaStreamSynchronize(st));
    return DS_OK;
}

}  // extern "C"

extern "C" {

// Adam / VectorAdam (Sec. 3.4, supplementary hyperparameters).
ds_status ds_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, int32_t dim, float lr,
                       float beta1, float beta2, float eps, int64_t step, void* stream) {
    if (n < 0) return fail(DS_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!params || !grads || !m || !v)) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (dim < 1 || dim > 4 || n % dim != 0) return fail(DS_ERR_INVALID_ARG, "dim must be in [1, 4] and divide n");
    if (step < 1) return fail(DS_ERR_INVALID_ARG, "step must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f) || !std::isfinite(lr))
        return fail(DS_ERR_INVALID_ARG, "bad hyperparameters");
    DS_TRY_CUDA(ds::launch_adam(params, grads, m, v, (long long)n, dim, lr, beta1, beta2, eps, (long long)step,
                                static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

}  // extern "C"

extern "C" {

ds_status ds_loss_l1_ssim(int32_t n_views, int32_t S, int32_t C, const int32_t* hw, const float* const* colors,
                          const float* const* targets, float* const* grad_colors, float* const* score_ws,
                          float lambda, float scale, float* loss, void* stream) {
    if (n_views < 1 || n_views > DS_MAX_VIEWS) return fail(DS_ERR_INVALID_ARG, "n_views out of range");
    if (S < 1 || S > DS_MAX_SAMPLES) return fail(DS_ERR_INVALID_ARG, "S out of range");
    if (C < 2 || C > DS_MAX_CHANNELS) return fail(DS_ERR_INVALID_ARG, "C out of range");
    if (!hw || !colors || !targets) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (!(lambda >= 0.f && lambda <= 1.f) || !std::isfinite(scale)) return fail(DS_ERR_INVALID_ARG, "bad lambda or scale");
    for (int v = 0; v < n_views; ++v) {
        if (hw[2 * v] < 1 || hw[2 * v + 1] < 1 || hw[2 * v] > DS_MAX_RESOLUTION || hw[2 * v + 1] > DS_MAX_RESOLUTION)
            return fail(DS_ERR_INVALID_ARG, "bad view size");
        if (!colors[v] || !targets[v]) return fail(DS_ERR_INVALID_ARG, "NULL colour or target");
    }
    DS_TRY_CUDA(ds::launch_loss_l1_ssim(n_views, S, C - 1, hw, colors, targets, grad_colors, score_ws, lambda, scale,
                                        loss, static_cast<cudaStream_t>(stream)));
    return DS_OK;
}

}  // extern "C"

