// noalloc.cu -- ads_apply_noalloc: the operators of ads_apply for callers
// that must not allocate device memory while they run.
//
// ads_apply allocates two interior scratch fields per call.  Some callers
// cannot allow that: a host application whose device memory is all handed
// out up front (a memory pool owned by another framework, a fixed budget
// per process), or a loop that cannot take the device-wide synchronisation
// and latency cudaMalloc/cudaFree may cost.  This variant uses a fixed
// scratch array compiled into the library instead; it allocates nothing.
#include <cuda_runtime.h>

#include <atomic>

#include "ads.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocFieldMax = (size_t)1 << 19;   // doubles per scratch field (4 MiB)

// Two scratch fields, 8 MiB in all; every GPU that loads the library keeps it
// until the process exits.  Shared by all calls, it keeps the last call's
// contents (each call clears what it reads before writing it).
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocFieldMax];

// Device address of the array, resolved once per device (host threads that
// race on the first call store the same value).  In host code the symbol's
// name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::atomic<double *> g_scratch_ptr[kMaxDevices];

// the scratch of device `dev`, which must be the current device
int scratch_for_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return ads_internal_fail(ADS_ERR_UNSUPPORTED, "ads_apply_noalloc: device ordinal beyond the scratch table");
    double *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        if (e != cudaSuccess || !q) {
            cudaGetLastError();
            return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: cudaGetSymbolAddress of the scratch failed");
        }
        p = (double *)q;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return ADS_OK;
}

// true when ptr is memory the simulation's device reads directly
bool on_device(const void *ptr, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int ads_apply_noalloc(ads_sim_t *sim, int op, const double *in, double *out, size_t count)
{
    if (!sim || !in || !out) return ads_internal_fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: null argument");
    const size_t need = ads_internal_interior_count(sim);
    if (need > kNoallocFieldMax)
        return ads_internal_fail(ADS_ERR_UNSUPPORTED,
                                 "ads_apply_noalloc: the space has more interior coefficients (padded layout) than "
                                 "the fixed scratch holds (524288 per field); use ads_apply");
    const int sdev = ads_internal_sim_device(sim);
    if (!on_device(in, sdev) || !on_device(out, sdev))
        return ads_internal_fail(ADS_ERR_INVALID_ARG,
                                 "ads_apply_noalloc: in and out must be device memory of the simulation's device");
    // the one place that selects the simulation's device (the scratch address
    // is resolved with it current) and restores the caller's afterwards
    int dev0 = 0;
    if (cudaGetDevice(&dev0) != cudaSuccess) {
        cudaGetLastError();
        return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: cudaGetDevice failed");
    }
    if (sdev != dev0 && cudaSetDevice(sdev) != cudaSuccess) {
        cudaGetLastError();
        return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: cannot select the simulation's device");
    }
    double *base = nullptr;
    int rc = scratch_for_device(sdev, &base);
    if (rc == ADS_OK) rc = ads_internal_apply_scratch(sim, op, in, out, count, base, base + kNoallocFieldMax);
    if (sdev != dev0) cudaSetDevice(dev0);
    return rc;
}
