// common.cuh -- small device/host helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>

namespace ads {

// Ricker wavelet r(t) = (1 - 2 a) exp(-a), a = (pi f (t - t0))^2: time profile of the
// source term F_{n+1} = (f(t_{n+1}), w) of Sec. 2
__device__ __forceinline__ double ricker_dev(double f, double t0, double t)
{
    const double pi = 3.141592653589793238462643;
    double a = pi * pi * f * f * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}

// elements of one line-table image: fac [m][2p+1] | phi, psi [m][p] | Phi, Psi [S][p][p]
__host__ __device__ __forceinline__ int line_image_elems_dev(int p, int m, int S)
{
    return m * (2 * p + 1) + 2 * m * p + 2 * S * p * p;
}

}  // namespace ads
