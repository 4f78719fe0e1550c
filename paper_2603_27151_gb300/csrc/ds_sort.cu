// ds_sort.cu -- device-wide exclusive scan and a stable LSD radix sort of
// (key, value) pairs with 8-bit digits, used to bin triangles into tiles.
#include "ds_internal.h"

namespace ds {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- scan
// Each block scans kScanBlock items (1024 threads x 4 consecutive items) and
// writes its total; higher levels scan the block totals.
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int64_t n, uint32_t* __restrict__ block_sum) {
    __shared__ uint32_t warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + 4 * tid;
    uint32_t x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = base + k < n ? in[base + k] : 0u;
    const uint32_t tsum = x[0] + x[1] + x[2] + x[3];
    uint32_t inc = tsum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += o;
        }
        warp_tot[lane] = wi - w;   // exclusive prefix of warp totals
        if (lane == 31 && block_sum) block_sum[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + inc - tsum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += x[k];
    }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ block_off) {
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t add = block_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i + 1024 * k < n) out[i + 1024 * k] += add;
}

__global__ void k_scan_total(const uint32_t* __restrict__ in, const uint32_t* __restrict__ out, int64_t n,
                             uint32_t* __restrict__ total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

int scan_levels(int64_t n, int64_t sizes[6]) {
    int lv = 0;
    int64_t m = n;
    while (m > kScanBlock && lv < 6) {
        m = (m + kScanBlock - 1) / kScanBlock;
        sizes[lv++] = m;
    }
    return lv;
}

static cudaError_t scan_rec(const uint32_t* in, uint32_t* out, int64_t n, const ScanScratch& sc, int lv,
                            cudaStream_t st) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb <= 1) {
        k_scan_block<<<1, 1024, 0, st>>>(in, out, n, nullptr);
        note_launches(1);
        return cudaGetLastError();
    }
    if (lv >= sc.levels) return cudaErrorInvalidValue;
    k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in, out, n, sc.level[lv]);
    cudaError_t e = scan_rec(sc.level[lv], sc.level_out[lv], nb, sc, lv + 1, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, n, sc.level_out[lv]);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, const ScanScratch& sc,
                           cudaStream_t st) {
    if (n > 0) {
        cudaError_t e = scan_rec(in, out, n, sc, 0, st);
        if (e != cudaSuccess) return e;
    }
    if (total) {
        k_scan_total<<<1, 1, 0, st>>>(in, out, n, total);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortRounds = kSortBlock / kSortThreads;   // 16

// Digit histogram of one block's keys, stored digit-major: hist[d * nblk + b].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ count, uint32_t kcap,
                                                             int shift, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const uint32_t K = min(*count, kcap);
    const uint32_t base = blockIdx.x * kSortBlock;
    for (int r = 0; r < kSortRounds; ++r) {
        const uint32_t i = base + r * kSortThreads + tid;
        if (i < K) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)tid * gridDim.x + blockIdx.x] = h[tid];
}

// Stable scatter: keys are taken in their input order, 256 per round; the
// rank of a key among equal digits is (keys of earlier rounds) + (keys of
// earlier warps in this round) + (earlier lanes of its warp).
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ count, uint32_t kcap, int shift,
    const uint32_t* __restrict__ hist_scan) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_w[kWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t K = min(*count, kcap);
    const uint32_t base = blockIdx.x * kSortBlock;
    s_base[tid] = hist_scan[(size_t)tid * gridDim.x + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        if (base + r * kSortThreads >= K) break;   // uniform across the block
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s_w[w][tid] = 0;
        __syncthreads();
        const uint32_t i = base + r * kSortThreads + tid;
        const bool valid = i < K;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t wrank = __popc(peers & lt);
        if (valid && wrank == 0) s_w[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s_base[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_w[w][tid];
                s_w[w][tid] = run;
                run += c;
            }
            s_base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_w[warp][d] + wrank;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* count,
                     uint32_t kcap, int nbits, uint32_t* hist, uint32_t* hist_scan, const ScanScratch& sc,
                     cudaStream_t st, cudaError_t* err) {
    *err = cudaSuccess;
    if (kcap == 0 || nbits <= 0) return 0;
    const unsigned nblk = (kcap + kSortBlock - 1) / kSortBlock;
    uint32_t* ks[2] = {k0, k1};
    uint32_t* vs[2] = {v0, v1};
    int cur = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_radix_hist<<<nblk, kSortThreads, 0, st>>>(ks[cur], count, kcap, shift, hist);
        cudaError_t e = scan_exclusive(hist, hist_scan, (int64_t)256 * nblk, nullptr, sc, st);
        if (e == cudaSuccess) {
            k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(ks[cur], vs[cur], ks[cur ^ 1], vs[cur ^ 1], count, kcap,
                                                           shift, hist_scan);
            note_launches(2);   // histogram + scatter
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            *err = e;
            return cur;
        }
        cur ^= 1;
    }
    return cur;
}

}  // namespace ds
