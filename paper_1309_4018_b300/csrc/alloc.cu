// Caching allocator of the library's device and page-locked host blocks.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "common.cuh"

namespace pb {

namespace {

constexpr size_t kDeviceCacheBytes = size_t(16) << 30;   // per device
constexpr size_t kHostCacheBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

struct Pool {
    std::multimap<size_t, void *> free;   // size -> block
    size_t held = 0;
};

std::mutex g_mu;
Pool g_dev[kMaxDevices];
Pool g_host;

// Smallest cached block of at least `bytes` and at most twice that.
void *take(Pool &pl, size_t bytes, size_t *got) {
    auto it = pl.free.lower_bound(bytes);
    if (it == pl.free.end() || it->first > 2 * bytes) return nullptr;
    void *p = it->second;
    *got = it->first;
    pl.held -= it->first;
    pl.free.erase(it);
    return p;
}

size_t round_up(size_t b) { return (b + 255) / 256 * 256; }

// Host-side fault injection for tests of the error paths: with the environment
// variable PB_FAULT=alloc:N set when the library is loaded, the N-th device
// allocation request (counted from 1 over the whole process) fails with
// PB_ENOMEM as if cudaMalloc had run out of memory.  Nothing reaches the GPU.
long long fault_alloc_at() {
    const char *e = std::getenv("PB_FAULT");
    if (!e || std::strncmp(e, "alloc:", 6) != 0) return 0;
    return std::atoll(e + 6);
}
const long long g_fault_at = fault_alloc_at();
std::atomic<long long> g_alloc_requests{0};

}  // namespace

void *cached_device_alloc(size_t bytes, size_t *got) {
    if (g_fault_at > 0 && g_alloc_requests.fetch_add(1) + 1 == g_fault_at)
        throw Error{PB_ENOMEM, "injected allocation failure (PB_FAULT=alloc:" + std::to_string(g_fault_at) + ")"};
    int dev = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    bytes = round_up(bytes);
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (void *p = take(g_dev[dev], bytes, got)) return p;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        // give the cached blocks back to the driver and try once more
        cudaGetLastError();
        if (dev >= 0 && dev < kMaxDevices) {
            std::lock_guard<std::mutex> lk(g_mu);
            for (auto &kv : g_dev[dev].free) cudaFree(kv.second);
            g_dev[dev].free.clear();
            g_dev[dev].held = 0;
        }
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{PB_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
        }
    }
    *got = bytes;
    return p;
}

void cached_device_free(void *p, size_t bytes) {
    if (!p) return;
    int dev = -1;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess) dev = at.device;
    else cudaGetLastError();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (dev >= 0 && dev < kMaxDevices && g_dev[dev].held + bytes <= kDeviceCacheBytes) {
            g_dev[dev].free.emplace(bytes, p);
            g_dev[dev].held += bytes;
            return;
        }
    }
    cudaFree(p);
}

void *cached_host_alloc(size_t bytes, size_t *got) {
    bytes = round_up(bytes);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (void *p = take(g_host, bytes, got)) return p;
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw Error{PB_ENOMEM, "cudaMallocHost failed"};
    }
    *got = bytes;
    return p;
}

void cached_host_free(void *p, size_t bytes) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_host.held + bytes <= kHostCacheBytes) {
            g_host.free.emplace(bytes, p);
            g_host.held += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

namespace {

// Page-locked staging area of a host thread (HostReads), grown on demand.
struct Staging {
    unsigned char *p = nullptr;
    size_t cap = 0, top = 0;
    ~Staging() {
        if (p) cached_host_free(p, cap);
    }
};
thread_local Staging t_staging;
constexpr size_t kStagingBytes = 64 << 10;

}  // namespace

HostReads::HostReads(cudaStream_t s) : s_(s), begin_(t_staging.top), end_(t_staging.top) {}

HostReads::~HostReads() { t_staging.top = begin_; }

void *HostReads::take(size_t bytes) {
    Staging &st = t_staging;
    if (!st.p) {
        size_t got = 0;
        st.p = static_cast<unsigned char *>(cached_host_alloc(kStagingBytes, &got));
        st.cap = got;
    }
    if (end_ != st.top) fail(PB_EINVAL, "internal: host staging area used out of order");
    const size_t at = (end_ + 15) / 16 * 16;
    if (at + bytes > st.cap) fail(PB_EINVAL, "internal: host staging area exhausted");
    end_ = at + bytes;
    st.top = end_;
    return st.p + at;
}

}  // namespace pb
