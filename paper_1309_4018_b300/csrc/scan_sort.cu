// Device-wide exclusive scan and key/index sort used by the setup phase.
#include "common.cuh"

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

__global__ void scan_add_kernel(int64_t *__restrict__ out, const int64_t *__restrict__ tile_off, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

__global__ void write_total_kernel(int64_t *out, const int64_t *tile_off, int64_t ntiles, int64_t n) {
    out[n] = tile_off[ntiles];
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
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    TmpBuf<int64_t> sums(ntiles, s), offs(ntiles + 1, s);
    scan_tiles_kernel<TIn><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, sums.p, n);
    PB_LAUNCH_CHECK();
    scan_impl<int64_t>(sums.p, offs.p, ntiles, s);
    scan_add_kernel<<<div_up(n, 256), 256, 0, s>>>(out, offs.p, n);
    PB_LAUNCH_CHECK();
    write_total_kernel<<<1, 1, 0, s>>>(out, offs.p, ntiles, n);
    PB_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- bitonic sort
__device__ __forceinline__ bool pair_greater(uint64_t ka, int32_t ia, uint64_t kb, int32_t ib) {
    return ka > kb || (ka == kb && ia > ib);
}

__global__ void bitonic_global_kernel(uint64_t *__restrict__ k, int32_t *__restrict__ v, int64_t half,
                                      int64_t j, int64_t stage) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const int64_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
    const int64_t hi = lo + j;
    const bool asc = (lo & stage) == 0;
    uint64_t ka = k[lo], kb = k[hi];
    int32_t ia = v[lo], ib = v[hi];
    if (pair_greater(ka, ia, kb, ib) == asc) {
        k[lo] = kb; k[hi] = ka;
        v[lo] = ib; v[hi] = ia;
    }
}

constexpr int kSortBlock = 2048;  // elements per block in shared memory (1024 threads)

// Runs every step j <= jmax of the given stage (or of all stages up to kSortBlock
// when stage == 0) inside one block's shared tile.
__global__ void __launch_bounds__(1024) bitonic_shared_kernel(uint64_t *__restrict__ k, int32_t *__restrict__ v,
                                                              int64_t stage, int64_t jmax) {
    __shared__ uint64_t sk[kSortBlock];
    __shared__ int32_t sv[kSortBlock];
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
        sk[t] = k[base + t];
        sv[t] = v[base + t];
    }
    __syncthreads();
    auto step = [&](int64_t st, int64_t j) {
        const int i = threadIdx.x;  // kSortBlock / 2 compare-exchanges
        const int lo = ((i & ~(int)(j - 1)) << 1) | (i & (int)(j - 1));
        const int hi = lo + (int)j;
        const bool asc = ((base + lo) & st) == 0;
        uint64_t ka = sk[lo], kb = sk[hi];
        int32_t ia = sv[lo], ib = sv[hi];
        if (pair_greater(ka, ia, kb, ib) == asc) {
            sk[lo] = kb; sk[hi] = ka;
            sv[lo] = ib; sv[hi] = ia;
        }
        __syncthreads();
    };
    if (stage == 0) {
        for (int64_t st = 2; st <= kSortBlock; st <<= 1)
            for (int64_t j = st >> 1; j > 0; j >>= 1) step(st, j);
    } else {
        for (int64_t j = jmax; j > 0; j >>= 1) step(stage, j);
    }
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
        k[base + t] = sk[t];
        v[base + t] = sv[t];
    }
}

__global__ void pad_kernel(uint64_t *k, int32_t *v, const uint64_t *kin, const int32_t *vin, int64_t n, int64_t n2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    if (i < n) { k[i] = kin[i]; v[i] = vin[i]; }
    else { k[i] = ~0ull; v[i] = 0x7fffffff; }
}

}  // namespace

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int32_t>(in, out, n, s); }

void sort_key_index(uint64_t *keys, int32_t *idx, int64_t n, cudaStream_t s) {
    if (n <= 1) return;
    int64_t n2 = kSortBlock;
    while (n2 < n) n2 <<= 1;
    TmpBuf<uint64_t> k(n2, s);
    TmpBuf<int32_t> v(n2, s);
    pad_kernel<<<div_up(n2, 256), 256, 0, s>>>(k.p, v.p, keys, idx, n, n2);
    PB_LAUNCH_CHECK();
    const unsigned nblk = (unsigned)(n2 / kSortBlock);
    bitonic_shared_kernel<<<nblk, 1024, 0, s>>>(k.p, v.p, 0, 0);
    PB_LAUNCH_CHECK();
    for (int64_t stage = 2 * kSortBlock; stage <= n2; stage <<= 1) {
        int64_t j = stage >> 1;
        for (; j >= kSortBlock; j >>= 1) {
            bitonic_global_kernel<<<div_up(n2 / 2, 256), 256, 0, s>>>(k.p, v.p, n2 / 2, j, stage);
            PB_LAUNCH_CHECK();
        }
        bitonic_shared_kernel<<<nblk, 1024, 0, s>>>(k.p, v.p, stage, j);
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaMemcpyAsync(keys, k.p, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    PB_CUDA_TRY(cudaMemcpyAsync(idx, v.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
}

}  // namespace pb
