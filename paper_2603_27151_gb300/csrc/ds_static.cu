// ds_static.cu -- ds_raster_forward_noalloc: the forward pass for callers
// that cannot allocate device memory.  All of its scratch (activations,
// set-up records, bin keys and values, sort and scan buffers, tile ranges,
// counters) lives in one file-scope device array of fixed size; the caller
// passes inputs and outputs as usual.  No cudaMalloc, cudaFree or other
// allocating call is made.
#include <cstring>
#include <mutex>
#include <string>

#include "ds_internal.h"

namespace {

// Size limits of one call (validated before any launch).
constexpr long long kMaxTexFloats = 1LL << 20;   // T * V * C
constexpr long long kMaxViewTris = 1LL << 16;    // n_views * T
constexpr long long kMaxPairs = 1LL << 19;       // (tile, triangle) pairs after binning
constexpr int kTileEdge = 16;                    // tiles of 16x16 pixels
constexpr long long kMaxTiles = 1LL << 16;       // 16x16 tiles over all views
constexpr long long kMaxSortBlocks = kMaxPairs / ds::kSortBlock;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve-out of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffAct = 0;
constexpr size_t kOffActA = align256(kOffAct + 4 * kMaxTexFloats);
constexpr size_t kOffRecs = align256(kOffActA + 4 * (kMaxTexFloats / 2));
constexpr size_t kOffCounts = align256(kOffRecs + sizeof(ds::SetupRec) * kMaxViewTris);
constexpr size_t kOffOffs = align256(kOffCounts + 4 * kMaxViewTris);
constexpr size_t kOffBox = align256(kOffOffs + 4 * kMaxViewTris);
constexpr size_t kOffZkeys = align256(kOffBox + 16 * kMaxViewTris);
constexpr size_t kOffKeys0 = align256(kOffZkeys + 4 * kMaxViewTris);
constexpr size_t kOffVals0 = align256(kOffKeys0 + 4 * kMaxPairs);
constexpr size_t kOffKeys1 = align256(kOffVals0 + 4 * kMaxPairs);
constexpr size_t kOffVals1 = align256(kOffKeys1 + 4 * kMaxPairs);
constexpr size_t kOffHist = align256(kOffVals1 + 4 * kMaxPairs);
constexpr size_t kOffHistScan = align256(kOffHist + 4 * 256 * kMaxSortBlocks);
constexpr size_t kOffScan = align256(kOffHistScan + 4 * 256 * kMaxSortBlocks);
constexpr size_t kScanWords = 2 * 64;            // level buffers: inputs up to 2^18 items
constexpr size_t kOffRanges = align256(kOffScan + 4 * kScanWords);
constexpr size_t kOffMisc = align256(kOffRanges + 8 * kMaxTiles);
constexpr size_t kStaticBytes = align256(kOffMisc + 256);   // about 21 MiB

// The scratch.  Every GPU that loads the library holds it until the process
// exits; every call of ds_raster_forward_noalloc on that GPU shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};   // device address of the array, per device ordinal

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

thread_local ds::ViewTable t_vt;   // host staging of the kernel parameter table

// Every caller pointer must be device memory of the current device (or
// managed memory): a host or foreign-device pointer would be dereferenced by
// the kernels.  cudaPointerGetAttributes allocates nothing.
bool on_current_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

ds_status reject(ds_status code, const std::string& msg) {
    ds::report_error(msg);
    return code;
}

}  // namespace

extern "C" DS_API ds_status ds_raster_forward_noalloc(const float* verts, const float* tex, int32_t T, int32_t grid_n,
                                                      int32_t C, const ds_camera* cams, const uint64_t* seeds,
                                                      int32_t n_views, int32_t S, uint32_t mode, const float* bg,
                                                      const ds_view_out* out, void* stream) {
    // ---- validation: everything is checked before the first launch
    if (!verts || !tex || !cams || !bg || !out) return reject(DS_ERR_INVALID_ARG, "NULL argument");
    if (T < 1 || grid_n < 1 || grid_n > DS_MAX_GRID_N || C < 2 || C > DS_MAX_CHANNELS)
        return reject(DS_ERR_INVALID_ARG, "T, grid_n or C out of range");
    if (n_views < 1 || n_views > DS_MAX_VIEWS || S < 1 || S > DS_MAX_SAMPLES)
        return reject(DS_ERR_INVALID_ARG, "n_views or S out of range");
    if (mode != DS_MODE_STOCHASTIC && mode != DS_MODE_THRESHOLD_HALF)
        return reject(DS_ERR_INVALID_ARG, "bad mode (flag bits such as DS_NO_SYNC are not accepted here)");
    if (mode == DS_MODE_STOCHASTIC && !seeds) return reject(DS_ERR_INVALID_ARG, "seeds is NULL");
    const int V = (grid_n + 1) * (grid_n + 2) / 2;
    if ((long long)T * V * C > kMaxTexFloats)
        return reject(DS_ERR_INVALID_ARG, "T*V*C exceeds the no-alloc limit of 2^20 texture values");
    if ((long long)n_views * T > kMaxViewTris)
        return reject(DS_ERR_INVALID_ARG, "n_views*T exceeds the no-alloc limit of 65536");
    if (ds::check_outputs(out, n_views) != DS_OK) return DS_ERR_INVALID_ARG;   // message set
    long long tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        if (!ds::finite_cam(cams[v])) return reject(DS_ERR_INVALID_ARG, "camera " + std::to_string(v) + " is invalid");
        tiles += (long long)((cams[v].width + kTileEdge - 1) / kTileEdge) * ((cams[v].height + kTileEdge - 1) / kTileEdge);
    }
    if (tiles > kMaxTiles) return reject(DS_ERR_INVALID_ARG, "the views exceed the no-alloc limit of 65536 tiles");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return reject(DS_ERR_CUDA, "cudaGetDevice failed");
    bool dev_ok = on_current_device(verts, dev) && on_current_device(tex, dev);
    for (int v = 0; v < n_views && dev_ok; ++v)
        dev_ok = on_current_device(out[v].gbuf, dev) && on_current_device(out[v].color, dev) &&
                 (!out[v].n_front || on_current_device(out[v].n_front, dev));
    if (!dev_ok) return reject(DS_ERR_INVALID_ARG, "an input or output is not device memory of the current device");

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return reject(DS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    // ---- views and soup over the scratch array
    ds::ViewTable& vt = t_vt;
    const ds_tuning tu{kTileEdge, 0, 0, ds::kChunk};
    ds::build_table(vt, tu, cams, seeds, n_views, S, out, nullptr);
    const int tile_base = vt.v[n_views - 1].tile_base + vt.v[n_views - 1].tiles_x * vt.v[n_views - 1].tiles_y;

    ds::SoupDev sd;
    sd.verts = verts;
    sd.tex = tex;
    sd.act = reinterpret_cast<float*>(base + kOffAct);
    sd.act_a = reinterpret_cast<float*>(base + kOffActA);
    sd.T = T;
    sd.N = grid_n;
    sd.C = C;
    sd.V = V;
    auto* recs = reinterpret_cast<ds::SetupRec*>(base + kOffRecs);
    auto* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    auto* offs = reinterpret_cast<uint32_t*>(base + kOffOffs);
    auto* tbox = reinterpret_cast<int4*>(base + kOffBox);
    auto* zkeys = reinterpret_cast<uint32_t*>(base + kOffZkeys);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(base + kOffKeys0), reinterpret_cast<uint32_t*>(base + kOffKeys1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(base + kOffVals0), reinterpret_cast<uint32_t*>(base + kOffVals1)};
    auto* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    auto* hist_scan = reinterpret_cast<uint32_t*>(base + kOffHistScan);
    auto* ranges = reinterpret_cast<uint2*>(base + kOffRanges);
    int* misc = reinterpret_cast<int*>(base + kOffMisc);
    int* status = misc;
    int* counter = misc + 4;
    uint32_t* dK = reinterpret_cast<uint32_t*>(misc + 12);

    // scan levels for inputs up to max(n_views * T, 256 * sort blocks) = 2^16 items
    ds::ScanScratch sc;
    int64_t sizes[6] = {0};
    sc.levels = ds::scan_levels(kMaxViewTris > 256 * kMaxSortBlocks ? kMaxViewTris : 256 * kMaxSortBlocks, sizes);
    uint32_t* sp = reinterpret_cast<uint32_t*>(base + kOffScan);
    for (int i = 0; i < sc.levels; ++i) {
        sc.level_n[i] = sizes[i];
        sc.level[i] = sp;
        sp += sizes[i];
        sc.level_out[i] = sp;
        sp += sizes[i];
    }

#define NA_TRY(call)                                                                                         \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return reject(DS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    // ---- the forward pipeline of ds_raster_forward, on the scratch array.
    // The array keeps the previous call's contents: the status word, the work
    // counters and the tile ranges are cleared here.
    const size_t nvt = (size_t)n_views * T;
    NA_TRY(cudaMemsetAsync(misc, 0, 256, st));
    NA_TRY(ds::launch_activate(sd, st));
    ds::set_view_soups(vt, sd);
    NA_TRY(ds::launch_setup(vt, recs, counts, tbox, zkeys, st));
    NA_TRY(ds::scan_exclusive(counts, offs, (int64_t)nvt, dK, sc, st));
    uint32_t K = 0;   // the one data-dependent size, read back into host stack memory
    NA_TRY(cudaMemcpyAsync(&K, dK, sizeof(K), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if ((long long)K > kMaxPairs)
        return reject(DS_ERR_CAPACITY, "binning produced " + std::to_string(K) +
                                           " (tile, triangle) pairs; the no-alloc limit is 524288");
    int tile_bits = 0;
    while (tile_bits < 32 && (1ull << tile_bits) < (unsigned long long)tile_base) ++tile_bits;
    const int DB = tile_bits <= 16 ? 16 : 32 - tile_bits;
    NA_TRY(ds::launch_emit(vt, recs, counts, offs, tbox, zkeys, DB, keys[0], vals[0], (uint32_t)kMaxPairs, status, st));
    cudaError_t se = cudaSuccess;
    const int res = ds::radix_sort_pairs(keys[0], vals[0], keys[1], vals[1], dK, K, tile_bits + DB, hist, hist_scan, sc,
                                         st, &se);
    NA_TRY(se);
    NA_TRY(cudaMemsetAsync(ranges, 0, 8 * (size_t)tile_base, st));
    NA_TRY(ds::launch_tile_ranges(keys[res], dK, K, DB, ranges, st));
    ds::Bg b{};
    for (int i = 0; i < C - 1; ++i) b.c[i] = bg[i];
    const int grid = 0;
    NA_TRY(ds::launch_raster_fwd(vt, sd, recs, keys[res], vals[res], ranges, DB, mode, b, counter, grid, st));
    bool want_front = false;
    for (int v = 0; v < n_views; ++v) want_front = want_front || out[v].n_front;
    if (want_front)
        NA_TRY(ds::launch_raster_count(vt, sd, recs, keys[res], vals[res], ranges, DB, 0, nullptr, counter + 1, grid, st));
#undef NA_TRY
    return DS_OK;
}
