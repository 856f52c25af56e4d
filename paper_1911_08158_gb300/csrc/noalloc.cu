// noalloc.cu -- ads_apply_noalloc: the operators of ads_apply for callers
// that must not allocate device memory while they run.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they need an operator: code that runs while a CUDA stream is
// being captured into a graph, or a real-time loop whose memory is fixed
// up front.  ads_apply allocates two interior scratch fields per call; this
// variant uses a fixed scratch array compiled into the library instead.
#include <cuda_runtime.h>

#include "ads.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocFieldMax = (size_t)1 << 19;   // doubles per scratch field (4 MiB)

// Two scratch fields, 8 MiB in all; every GPU that loads the library keeps it
// until the process exits.  Shared by all calls, it keeps the last call's
// contents (each call clears what it reads before writing it).
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocFieldMax];

// Device address of the array, resolved once per device.  In host code the
// symbol's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: no current CUDA device");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: cudaGetSymbolAddress of the scratch failed");
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return ADS_OK;
}

}  // namespace

extern "C" int ads_apply_noalloc(ads_sim_t *sim, int op, const double *in, double *out, size_t count)
{
    if (!sim) return ads_internal_fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: null sim");
    const size_t need = ads_internal_interior_count(sim);
    if (need > kNoallocFieldMax)
        return ads_internal_fail(ADS_ERR_UNSUPPORTED,
                                 "ads_apply_noalloc: the space has more interior coefficients (padded layout) than "
                                 "the fixed scratch holds (524288 per field); use ads_apply");
    // the scratch address is resolved with the simulation's device current
    int dev0 = 0;
    cudaGetDevice(&dev0);
    const int sdev = ads_internal_sim_device(sim);
    if (sdev != dev0 && cudaSetDevice(sdev) != cudaSuccess)
        return ads_internal_fail(ADS_ERR_CUDA, "ads_apply_noalloc: cannot select the simulation's device");
    double *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc == ADS_OK) rc = ads_internal_apply_scratch(sim, op, in, out, count, base, base + kNoallocFieldMax);
    if (sdev != dev0) cudaSetDevice(dev0);
    return rc;
}
