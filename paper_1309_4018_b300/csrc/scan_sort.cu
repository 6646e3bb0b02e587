// Device-wide exclusive scan and key/index sort used by the setup phase.
#include <cooperative_groups.h>

#include <algorithm>
#include <utility>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pb {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename TIn>
__global__ void scan_tiles_kernel(const TIn *__restrict__ in, int64_t *__restrict__ out,
                                  int64_t *__restrict__ tile_sums, int64_t n) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t x = (base + i < n) ? (int64_t)in[base + i] : 0;
        v[i] = run;
        run += x;
    }
    // inclusive scan of per-thread totals across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const int64_t excl = incl - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] = v[i] + excl;
    if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = excl + run;
}

// Sum of the block's values (every thread gets it).
__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int64_t t = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    return t;
}

// The whole scan in one cooperative launch: every block takes a contiguous
// run of tiles; it sums its run, and after a grid-wide barrier adds the sums
// of the blocks before it and scans its tiles in order with a running carry.
// Block 0 writes the total into out[n].  Integer sums: the result does not
// depend on the grid.
template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) scan_coop_kernel(const TIn *__restrict__ in, int64_t *__restrict__ out,
                                                                 int64_t n, int64_t *__restrict__ block_sums) {
    cg::grid_group grid = cg::this_grid();
    __shared__ int64_t warp_tot[kScanThreads / 32];
    __shared__ int64_t red[kScanThreads / 32];
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per * kScanTile, b1 = min(n, b0 + per * kScanTile);
    int64_t local = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kScanThreads) local += (int64_t)in[i];
    local = block_sum(local, red);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = local;
    grid.sync();
    int64_t before = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kScanThreads) before += block_sums[b];
    before = block_sum(before, red);
    if (blockIdx.x == 0) {
        int64_t all = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kScanThreads) all += block_sums[b];
        all = block_sum(all, red);
        if (threadIdx.x == 0) out[n] = all;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = before;
    for (int64_t t0 = b0; t0 < b1; t0 += kScanTile) {
        const int64_t base = t0 + threadIdx.x * kScanItems;
        int64_t v[kScanItems];
        int64_t run = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t x = (base + i < b1) ? (int64_t)in[base + i] : 0;
            v[i] = run;
            run += x;
        }
        int64_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int64_t wbefore = 0, tile_total = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) {
            if (w < warp) wbefore += warp_tot[w];
            tile_total += warp_tot[w];
        }
        const int64_t excl = carry + wbefore + incl - run;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i)
            if (base + i < b1) out[base + i] = v[i] + excl;
        carry += tile_total;
    }
}

int scan_grid(int64_t ntiles) {
    static int cap = 0;
    if (!cap) {
        int per_sm = 0, nsm = 0, dev = 0;
        PB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_coop_kernel<int64_t>, kScanThreads, 0));
        int per_sm32 = 0;
        PB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, scan_coop_kernel<int32_t>, kScanThreads, 0));
        PB_CUDA_TRY(cudaGetDevice(&dev));
        PB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        cap = std::max(1, nsm * std::min(2, std::min(per_sm, per_sm32)));
    }
    return (int)std::min<int64_t>(cap, ntiles);
}

template <typename TIn>
void scan_impl(const TIn *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        PB_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    if (n <= kScanTile) {  // one tile: its total lands in out[n]
        scan_tiles_kernel<TIn><<<1, kScanThreads, 0, s>>>(in, out, out + n, n);
        PB_LAUNCH_CHECK();
        return;
    }
    const int grid = scan_grid((n + kScanTile - 1) / kScanTile);
    TmpBuf<int64_t> sums(grid, s);
    const TIn *a_in = in;
    int64_t *a_out = out, *a_sums = sums.p;
    int64_t a_n = n;
    void *args[] = {&a_in, &a_out, &a_n, &a_sums};
    PB_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)scan_coop_kernel<TIn>, grid, kScanThreads, args, 0, s));
    PB_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- merge sort
// (key, idx) pairs in one total order: by key, then by idx.
__device__ __forceinline__ bool pair_less(uint64_t ka, int32_t ia, uint64_t kb, int32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

constexpr int kSortBlock = 2048;   // elements per tile sorted in shared memory (1024 threads)
constexpr int kMergeItems = 8;     // outputs per thread of a merge round

// Copies n pairs and pads to n2 (a multiple of kSortBlock) with pairs that
// order after every real one.
__global__ void pad_kernel(uint64_t *k, int32_t *v, const uint64_t *kin, const int32_t *vin, int64_t n, int64_t n2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    if (i < n) { k[i] = kin[i]; v[i] = vin[i]; }
    else { k[i] = ~0ull; v[i] = 0x7fffffff; }
}

// Every tile of kSortBlock pairs sorted ascending in shared memory (bitonic network).
__global__ void __launch_bounds__(1024) tile_sort_kernel(uint64_t *__restrict__ k, int32_t *__restrict__ v) {
    __shared__ uint64_t sk[kSortBlock];
    __shared__ int32_t sv[kSortBlock];
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
        sk[t] = k[base + t];
        sv[t] = v[base + t];
    }
    __syncthreads();
    for (int st = 2; st <= kSortBlock; st <<= 1)
        for (int j = st >> 1; j > 0; j >>= 1) {
            const int i = threadIdx.x;   // kSortBlock / 2 compare-exchanges
            const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
            const int hi = lo + j;
            const bool asc = (lo & st) == 0;
            const uint64_t ka = sk[lo], kb = sk[hi];
            const int32_t ia = sv[lo], ib = sv[hi];
            if (pair_less(kb, ib, ka, ia) == asc) {
                sk[lo] = kb; sk[hi] = ka;
                sv[lo] = ib; sv[hi] = ia;
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
        k[base + t] = sk[t];
        v[base + t] = sv[t];
    }
}

// One merge round: the sorted runs of width w of (ka, va) merged pairwise into
// (kb, vb); only the first nout outputs are written.  Each thread finds where
// its first output lies on the merge path of its two runs (binary search),
// then merges kMergeItems outputs.  Within the total order no two real pairs
// are equal, so the result is the unique sorted order.
__global__ void merge_round_kernel(const uint64_t *__restrict__ ka, const int32_t *__restrict__ va,
                                   uint64_t *__restrict__ kb, int32_t *__restrict__ vb, int64_t n, int64_t nout,
                                   int64_t w) {
    const int64_t o0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kMergeItems;
    if (o0 >= nout) return;
    const int64_t s = o0 / (2 * w) * (2 * w);
    const int64_t a0 = s, na = min(w, n - s);
    const int64_t b0 = s + na, nb = max((int64_t)0, min(w, n - s - na));
    const int64_t d = o0 - s;
    int64_t lo = max((int64_t)0, d - nb), hi = min(d, na);
    while (lo < hi) {   // smallest i with B[d - i - 1] < A[i]
        const int64_t i = (lo + hi) >> 1;
        const int64_t j = d - i - 1;
        if (pair_less(ka[b0 + j], va[b0 + j], ka[a0 + i], va[a0 + i])) hi = i;
        else lo = i + 1;
    }
    int64_t i = lo, j = d - lo;
    const int64_t end = min(o0 + kMergeItems, min(nout, s + na + nb));
    for (int64_t o = o0; o < end; ++o) {
        const bool take_a = j >= nb || (i < na && !pair_less(ka[b0 + j], va[b0 + j], ka[a0 + i], va[a0 + i]));
        if (take_a) { kb[o] = ka[a0 + i]; vb[o] = va[a0 + i]; ++i; }
        else { kb[o] = ka[b0 + j]; vb[o] = va[b0 + j]; ++j; }
    }
}

}  // namespace

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int32_t>(in, out, n, s); }

// Tiles of kSortBlock pairs sorted in shared memory, then merge rounds doubling
// the sorted run width; the last round writes into (keys, idx).
void sort_key_index(uint64_t *keys, int32_t *idx, int64_t n, cudaStream_t s) {
    if (n <= 1) return;
    const int64_t n2 = (n + kSortBlock - 1) / kSortBlock * kSortBlock;
    TmpBuf<uint64_t> k0(n2, s), k1(n2, s);
    TmpBuf<int32_t> v0(n2, s), v1(n2, s);
    pad_kernel<<<div_up(n2, 256), 256, 0, s>>>(k0.p, v0.p, keys, idx, n, n2);
    PB_LAUNCH_CHECK();
    tile_sort_kernel<<<(unsigned)(n2 / kSortBlock), 1024, 0, s>>>(k0.p, v0.p);
    PB_LAUNCH_CHECK();
    uint64_t *ka = k0.p, *kb = k1.p;
    int32_t *va = v0.p, *vb = v1.p;
    for (int64_t w = kSortBlock; w < n2; w <<= 1) {
        const bool last = 2 * w >= n2;
        uint64_t *ko = last ? keys : kb;
        int32_t *vo = last ? idx : vb;
        const int64_t nout = last ? n : n2;
        merge_round_kernel<<<div_up(div_up(nout, kMergeItems), 256), 256, 0, s>>>(ka, va, ko, vo, n2, nout, w);
        PB_LAUNCH_CHECK();
        if (last) return;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    // a single tile: copy the sorted pairs back
    PB_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    PB_CUDA_TRY(cudaMemcpyAsync(idx, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
}

}  // namespace pb
