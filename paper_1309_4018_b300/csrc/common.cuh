// Shared definitions of the pbbem CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/pbbem.h"

namespace pb {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * kPi);
// e^2 N_A / (4 pi eps0 * 1 Angstrom) / 1000 in kJ/mol (CODATA 2018)
constexpr double kKjPerMol = 1389.3545764;
constexpr int kMaxLevel = 21;
constexpr int kMaxP = 12;
constexpr int kRadialMaxP = 8;      // the FP32 M2P uses the radial form up to this order
constexpr int kMaxTerms1 = (kMaxP + 2) * (kMaxP + 3) * (kMaxP + 4) / 6;   // terms up to order kMaxP + 1

// Four doubles, 32-byte aligned (one vector load).
struct alignas(32) dvec4 {
    double x, y, z, w;
};

inline int nterms(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// ---------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

#define PB_CUDA_TRY(call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            throw ::pb::Error{PB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};   \
    } while (0)

// Every kernel launch of the library is followed by PB_LAUNCH_CHECK, which
// also counts it (pb_launch_count).
extern std::atomic<long long> g_launches;
#define PB_LAUNCH_CHECK()                            \
    do {                                             \
        ::pb::g_launches.fetch_add(1, std::memory_order_relaxed); \
        PB_CUDA_TRY(cudaGetLastError());             \
    } while (0)

inline void fail(int code, const std::string &m) { throw Error{code, m}; }

// ---------------------------------------------------------------- caching allocator
// Library-owned device and page-locked host blocks are recycled: a released
// block goes to a per-device free list (bounded; beyond the bound it is freed)
// and a later request of at most its size takes it back, so a problem built
// again (or a new one of similar size) allocates nothing from the driver.
// Blocks are only released when no queued work uses them: every entry point
// synchronises its stream before returning.  *got receives the block's size.
void *cached_device_alloc(size_t bytes, size_t *got);
void cached_device_free(void *p, size_t bytes);
void *cached_host_alloc(size_t bytes, size_t *got);
void cached_host_free(void *p, size_t bytes);

// ---------------------------------------------------------------- device buffer
// Device array owned by the library.  alloc() keeps the existing allocation
// when it is large enough (a re-setup of the same geometry allocates nothing).
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0, cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n), cap(o.cap) { o.p = nullptr; o.n = 0; o.cap = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; cap = o.cap; o.p = nullptr; o.n = 0; o.cap = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cached_device_free(p, cap * sizeof(T));
        p = nullptr;
        n = 0;
        cap = 0;
    }
    void alloc(size_t count) {
        if (p && count <= cap && count > 0) {
            n = count;
            return;
        }
        release();
        if (count == 0) return;
        size_t got = 0;
        p = static_cast<T *>(cached_device_alloc(count * sizeof(T), &got));
        n = count;
        cap = got / sizeof(T);
    }
    void zero(cudaStream_t s) {
        if (n) PB_CUDA_TRY(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void upload(const T *h, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) PB_CUDA_TRY(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void download(T *h, size_t count, cudaStream_t s) const {
        if (count) PB_CUDA_TRY(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
};

// Page-locked host scalars (asynchronous device-to-host reads).
template <typename T>
struct PinnedBuf {
    T *p = nullptr;
    size_t cap = 0;
    PinnedBuf() = default;
    PinnedBuf(const PinnedBuf &) = delete;
    PinnedBuf &operator=(const PinnedBuf &) = delete;
    PinnedBuf(PinnedBuf &&o) noexcept : p(o.p), cap(o.cap) { o.p = nullptr; o.cap = 0; }
    PinnedBuf &operator=(PinnedBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; cap = o.cap; o.p = nullptr; o.cap = 0; }
        return *this;
    }
    ~PinnedBuf() { release(); }
    void release() {
        if (p) cached_host_free(p, cap * sizeof(T));
        p = nullptr;
        cap = 0;
    }
    void alloc(size_t count) {
        if (p && count <= cap) return;
        release();
        size_t got = 0;
        p = static_cast<T *>(cached_host_alloc(count * sizeof(T), &got));
        cap = got / sizeof(T);
    }
};

// Small device-to-host reads gathered into one stream synchronisation.  The
// values land in a page-locked staging area of the calling host thread (a
// copy into pageable memory would wait for the stream inside cudaMemcpyAsync
// and pass through a driver buffer): add() queues a copy and returns where it
// will be, valid after wait() and until the HostReads is destroyed.  Objects
// on one thread must be destroyed in reverse order of creation.
class HostReads {
  public:
    explicit HostReads(cudaStream_t s);
    ~HostReads();
    HostReads(const HostReads &) = delete;
    HostReads &operator=(const HostReads &) = delete;
    template <typename T>
    const T *add(const T *d, size_t n = 1) {
        return add_on(s_, d, n);
    }
    // The copy queued on stream `on` instead (wait() then synchronises it too).
    template <typename T>
    const T *add_on(cudaStream_t on, const T *d, size_t n = 1) {
        void *h = take(n * sizeof(T));
        PB_CUDA_TRY(cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, on));
        if (on != s_) {
            bool seen = false;
            for (int i = 0; i < nother_; ++i) seen = seen || other_[i] == on;
            if (!seen) {
                if (nother_ == kOther) fail(PB_EINVAL, "internal: too many streams in one host read");
                other_[nother_++] = on;
            }
        }
        return static_cast<const T *>(h);
    }
    void wait() {
        PB_CUDA_TRY(cudaStreamSynchronize(s_));
        for (int i = 0; i < nother_; ++i) PB_CUDA_TRY(cudaStreamSynchronize(other_[i]));
    }

  private:
    static constexpr int kOther = 4;
    void *take(size_t bytes);
    cudaStream_t s_;
    size_t begin_, end_;
    cudaStream_t other_[kOther] = {};
    int nother_ = 0;
};
// One value read from the device (a stream synchronisation).
template <typename T>
T read_device(const T *d, cudaStream_t s) {
    HostReads r(s);
    const T *h = r.add(d);
    r.wait();
    return *h;
}

// Stream-ordered temporary: allocated and freed on the stream that uses it,
// so its release waits for the kernels queued before it.
template <typename T>
struct TmpBuf {
    T *p = nullptr;
    cudaStream_t s = 0;
    TmpBuf(size_t count, cudaStream_t st) : s(st) {
        if (count) {
            cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), st);
            if (e != cudaSuccess) {
                p = nullptr;
                throw Error{PB_ENOMEM, "cudaMallocAsync of " + std::to_string(count * sizeof(T)) + " bytes failed"};
            }
        }
    }
    TmpBuf(const TmpBuf &) = delete;
    TmpBuf &operator=(const TmpBuf &) = delete;
    ~TmpBuf() {
        if (p) cudaFreeAsync(p, s);
    }
};

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- primitives (scan_sort.cu)
// out[i] = sum_{j < i} in[j]; out has n + 1 entries (out[n] = total).  Deterministic.
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
void exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Sort (key, idx) pairs ascending by key then idx (a total order: equals a
// stable sort by key when idx is the input position).  n arbitrary.
void sort_key_index(uint64_t *keys, int32_t *idx, int64_t n, cudaStream_t s);

}  // namespace pb
