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

// Shared-memory plan of one K1 CTA (host and device use the same one).
// Row tiles: ty rows of one z-plane.  Fused: ty = my, the y sweep runs in
// the CTA.  Pair: a 2-CTA cluster holds one z-plane, CTA h its rows
// [h * ycut, ...) (ycut a multiple of 32), and the y sweep of columns
// [h * xcut, ...) reads the partner's rows through distributed shared memory.
struct RhsPlan {
    int rows;        // row capacity of S1 / S2
    int RS;          // row stride (odd)
    int rows_pad;    // rows rounded to whole warps
    int cols_pad;    // columns of this CTA's y sweep rounded to whole warps
    int cld;         // slot stride of the carry buffers
    int Smax;        // segments of the longer swept axis
    int ycut, xcut;  // pair split points (0 otherwise)
    bool fuse;
};

__host__ __device__ inline int pair_cut(int n)
{
    int c = ((n / 2) + 31) & ~31;
    return c < n ? c : n;
}

__host__ __device__ inline RhsPlan rhs_plan(int mx, int my, int ty, int pair, int Sx, int Sy)
{
    RhsPlan q;
    q.RS = ((mx + 1) & ~1) | 1;
    q.fuse = pair || ty == my;
    q.ycut = pair ? pair_cut(my) : 0;
    q.xcut = pair ? pair_cut(mx) : 0;
    q.rows = pair ? (q.ycut > my - q.ycut ? q.ycut : my - q.ycut) : ty;
    q.rows_pad = (q.rows + 31) & ~31;
    const int xs = pair ? (q.xcut > mx - q.xcut ? q.xcut : mx - q.xcut) : mx;
    q.cols_pad = (xs + 31) & ~31;
    q.cld = (q.fuse && q.cols_pad > q.rows_pad) ? q.cols_pad : q.rows_pad;
    q.Smax = (q.fuse && Sy > Sx) ? Sy : Sx;
    return q;
}

}  // namespace ads
