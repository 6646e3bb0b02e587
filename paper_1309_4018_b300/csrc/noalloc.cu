// Coulomb energy of a set of point charges computed without allocating any
// device memory.
//
// Who needs it: callers that manage every byte of device memory themselves
// (a host application with its own memory pool or a strict memory budget) or
// that cannot afford the device-wide synchronisation that cudaMalloc and
// cudaFree may imply inside a tight loop.  They hand in device pointers for
// the charges and the result and get the energy without the library touching
// the allocator.
//
// The per-charge row sums that the pb_coulomb_energy path keeps in a
// stream-ordered temporary live here in a file-scope device array instead.
// Every process that loads the library holds that array (2 MiB per GPU it
// touches) until exit.
#include <mutex>

#include "gmres.cuh"

namespace {

constexpr int64_t kNoAllocMaxCharges = 262144;   // 2 MiB of FP64 row sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_coulomb_rows[kNoAllocMaxCharges];

std::mutex g_mutex;
double *g_rows_addr[kMaxDevices] = {};   // device address of g_coulomb_rows, per device

// Device address of the scratch array on `device` (which must be current).
// cudaGetSymbolAddress is called once per device; the name itself is only a
// host-side stand-in and must never be handed to a kernel.
int rows_address(int device, double **out, const char **err) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_rows_addr[device]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_coulomb_rows) != cudaSuccess || !p) {
            if (err) *err = "cudaGetSymbolAddress of the scratch array failed";
            return PB_ECUDA;
        }
        g_rows_addr[device] = p;
    }
    *out = g_rows_addr[device];
    return PB_OK;
}

}  // namespace

extern "C" int pb_coulomb_energy_noalloc(int device, const double *xyz, const double *q, int64_t nc, double eps,
                                         double *energy, void *stream, const char **err) {
    if (err) *err = "";
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices) {
        if (err) *err = "no such CUDA device";
        return PB_EINVAL;
    }
    if (nc < 0 || nc > kNoAllocMaxCharges) {
        if (err) *err = "charge count outside 0..262144, the capacity of the static scratch array";
        return PB_EINVAL;
    }
    if (!energy || (nc > 0 && (!xyz || !q)) || !(eps > 0.0)) {
        if (err) *err = "null device pointer or eps <= 0";
        return PB_EINVAL;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) {
        if (err) *err = "cudaSetDevice failed";
        return PB_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = PB_OK;
    try {
        if (nc == 0) {
            PB_CUDA_TRY(cudaMemsetAsync(energy, 0, sizeof(double), s));
        } else {
            double *rows = nullptr;
            rc = rows_address(device, &rows, err);
            if (rc == PB_OK) {
                // rows[0..nc) are all rewritten before they are read; nothing needs clearing
                pb::coulomb_rows(xyz, q, nc, rows, s);
                pb::weighted_sum(q, rows, nc, 0.5 * pb::kKjPerMol / eps, energy, s);
            }
        }
    } catch (const pb::Error &e) {
        if (err) *err = "a CUDA launch failed";
        rc = e.code;
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
