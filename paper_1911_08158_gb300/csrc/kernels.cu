// kernels.cu -- set-up, boundary, operator and diagnostic kernels (sm_103a),
// the table-size helpers of the hot-path kernels and the non-templated
// launch wrappers.  The hot-path kernels themselves (K1 k_rhs, K2/K3 k_col)
// live in sweep.cuh and are instantiated in rhs_f32.cu, rhs_f64.cu,
// col_f32.cu and col_f64.cu.
#include "kernels.cuh"

#include <cstdio>
#include <cstring>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "tma.cuh"

namespace ads {

std::atomic<unsigned long long> g_launches{0};

std::mutex &attr_mutex()
{
    static std::mutex m;
    return m;
}

namespace {

// ---------------------------------------------------------------- helpers
template <typename T, int P>
__global__ void k_axis_apply(const T *__restrict__ band, int axis, const T *__restrict__ in, T *__restrict__ out,
                             Dims d, T alpha, T beta, int transpose)
{
    constexpr int W = 2 * P + 1;
    const long long n = d.count();
    const long long plane = d.plane();
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / plane);
        const long long rem = idx - (long long)z * plane;
        const int y = (int)(rem / d.sx);
        const int x = (int)(rem - (long long)y * d.sx);
        if (x >= d.mx) {   // row padding stays zero, so dot products may span it
            out[idx] = T(0);
            continue;
        }
        int i, m;
        long long st;
        if (axis == 0) { i = x; m = d.mx; st = 1; }
        else if (axis == 1) { i = y; m = d.my; st = d.sx; }
        else { i = z; m = d.mz; st = plane; }
        T acc = T(0);
#pragma unroll
        for (int k = -P; k <= P; ++k) {
            const int j = i + k;
            if (j < 0 || j >= m) continue;
            // (A^T)[i][j] = A[j][i] = band[j][i-j]
            const T c = transpose ? band[j * W + (-k + P)] : band[i * W + (k + P)];
            acc += c * in[idx + (long long)k * st];
        }
        out[idx] = (beta == T(0) ? T(0) : beta * out[idx]) + alpha * acc;
    }
}

// Sum of Kronecker products, one CTA per (z-plane, tile of ty rows): the
// terms are applied one after another through two staging buffers
// (z-contraction, y-contraction) and accumulated into a third, which is
// stored once.
template <typename T, int P>
__global__ void __launch_bounds__(256) k_kron_sum(const __grid_constant__ KronSum<T> ks, T *out, Dims d, int ty)
{
    constexpr int W = 2 * P + 1;
    extern __shared__ __align__(16) unsigned char ksum_smem[];
    const int sx = d.sx, mx = d.mx, my = d.my, mz = d.mz;
    T *Tz = reinterpret_cast<T *>(ksum_smem);   // [(ty + 2P)][sx]
    T *Uy = Tz + (size_t)(ty + 2 * P) * sx;     // [ty][sx]
    T *O = Uy + (size_t)ty * sx;                // [ty][sx] accumulator
    const int z = blockIdx.y, y0 = blockIdx.x * ty;
    const int tye = min(ty, my - y0);
    const long long plane = d.plane();
    const long long base = (long long)z * plane + (long long)y0 * sx;
    for (int idx = threadIdx.x; idx < tye * mx; idx += blockDim.x) {
        const int l = idx / mx, x = idx - l * mx;
        O[(size_t)l * sx + x] = ks.beta == T(0) ? T(0) : ks.beta * out[base + (long long)l * sx + x];
    }
    for (int t = 0; t < ks.nt; ++t) {
        const KronTerm<T> &tm = ks.t[t];
        if (tm.plain) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < tye * mx; idx += blockDim.x) {
                const int l = idx / mx, x = idx - l * mx;
                O[(size_t)l * sx + x] += tm.alpha * tm.in[base + (long long)l * sx + x];
            }
            continue;
        }
        T cz[W];
        bool zok[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            cz[k] = tm.bz[z * W + k];
            zok[k] = z + k - P >= 0 && z + k - P < mz;
        }
        __syncthreads();   // previous term's reads of Tz / Uy are done
        const int nr = tye + 2 * P;
        for (int idx = threadIdx.x; idx < nr * mx; idx += blockDim.x) {
            const int r = idx / mx, x = idx - r * mx;
            const int y = y0 - P + r;
            T acc = T(0);
            if (y >= 0 && y < my) {
                const T *src = tm.in + (long long)(z - P) * plane + (long long)y * sx + x;
#pragma unroll
                for (int k = 0; k < W; ++k)
                    if (zok[k]) acc += cz[k] * src[(long long)k * plane];
            }
            Tz[(size_t)r * sx + x] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < tye * mx; idx += blockDim.x) {
            const int l = idx / mx, x = idx - l * mx;
            const T *row = tm.by + (size_t)(y0 + l) * W;
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < W; ++q) acc += row[q] * Tz[(size_t)(l + q) * sx + x];
            Uy[(size_t)l * sx + x] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < tye * mx; idx += blockDim.x) {
            const int l = idx / mx, x = idx - l * mx;
            const T *row = tm.bx + (size_t)x * W;
            const T *u = Uy + (size_t)l * sx;
            T acc = T(0);
#pragma unroll
            for (int r = 0; r < W; ++r) {
                const int xx = x + r - P;
                if (xx >= 0 && xx < mx) acc += row[r] * u[xx];
            }
            O[(size_t)l * sx + x] += tm.alpha * acc;
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < tye * sx; idx += blockDim.x) {
        const int l = idx / sx, x = idx - l * sx;
        out[base + (long long)l * sx + x] = x < mx ? O[(size_t)l * sx + x] : T(0);
    }
}

template <typename T, int P>
__global__ void k_solve_x(const T *__restrict__ F, T *data, Dims d)
{
    constexpr int W = 2 * P + 1;
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= d.my * d.mz) return;
    T *row = data + (long long)line * d.sx;   // lines are rows: (z*my + y)*sx
    T wp[P];
#pragma unroll
    for (int k = 0; k < P; ++k) wp[k] = T(0);
    for (int j = 0; j < d.mx; ++j) {
        T w = row[j];
#pragma unroll
        for (int k = 1; k <= P; ++k) w -= F[j * W + P - k] * wp[k - 1];
        row[j] = w;
#pragma unroll
        for (int k = P - 1; k > 0; --k) wp[k] = wp[k - 1];
        wp[0] = w;
    }
    T xp[P];
#pragma unroll
    for (int k = 0; k < P; ++k) xp[k] = T(0);
    for (int j = d.mx - 1; j >= 0; --j) {
        T v = row[j];
#pragma unroll
        for (int k = 1; k <= P; ++k) v -= F[j * W + P + k] * xp[k - 1];
        v *= F[j * W + P];
        row[j] = v;
#pragma unroll
        for (int k = P - 1; k > 0; --k) xp[k] = xp[k - 1];
        xp[0] = v;
    }
}

template <typename T>
__global__ void k_pack(const double *__restrict__ full, T *__restrict__ in, Dims d, double scale)
{
    const long long n = d.count();
    const long long plane = d.plane();
    const int o = d.off, oz = d.offz;
    const int nx = d.mx + 2 * o, ny = d.my + 2 * o;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / plane);
        const long long rem = idx - (long long)z * plane;
        const int y = (int)(rem / d.sx);
        const int x = (int)(rem - (long long)y * d.sx);
        T v = T(0);
        if (x < d.mx) v = (T)(scale * full[((long long)(z + oz) * ny + (y + o)) * nx + (x + o)]);
        in[idx] = v;
    }
}

template <typename T>
__global__ void k_unpack(const T *__restrict__ in, double *__restrict__ full, Dims d)
{
    const int o = d.off, oz = d.offz;
    const int nx = d.mx + 2 * o, ny = d.my + 2 * o, nz = d.mz + 2 * oz;
    const long long n = (long long)nx * ny * nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / ((long long)nx * ny));
        const long long rem = idx - (long long)z * nx * ny;
        const int y = (int)(rem / nx);
        const int x = (int)(rem - (long long)y * nx);
        double v = 0.0;
        if (x >= o && x < d.mx + o && y >= o && y < d.my + o && z >= oz && z < d.mz + oz)
            v = (double)in[(long long)(z - oz) * d.plane() + (long long)(y - o) * d.sx + (x - o)];
        full[idx] = v;
    }
}

template <typename T>
__global__ void k_uva_to_pq(const double *__restrict__ u, const double *__restrict__ v,
                            const double *__restrict__ acc, T *P, T *Q, T *A, long long n, double tau)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double tv = tau * v[i], aa = acc[i];
        P[i] = (T)(u[i] + tv + 0.25 * tau * tau * aa);
        Q[i] = (T)(tv + 0.5 * tau * tau * aa);
        A[i] = (T)aa;
    }
}

template <typename T>
__global__ void k_pq_to_uva(const T *P, const T *Q, const T *A, double *u, double *v, double *acc, long long n,
                            double tau)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double p = (double)P[i], q = (double)Q[i], aa = (double)A[i];
        if (u) u[i] = p - q + 0.25 * tau * tau * aa;
        if (v) v[i] = (q - 0.5 * tau * tau * aa) / tau;
        if (acc) acc[i] = aa;
    }
}

__global__ void k_outer(const double *gx, const double *gy, const double *gz, double amp, double *out, Dims d)
{
    const long long n = d.count();
    const long long plane = d.plane();
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / plane);
        const long long rem = idx - (long long)z * plane;
        const int y = (int)(rem / d.sx);
        const int x = (int)(rem - (long long)y * d.sx);
        out[idx] = x < d.mx ? amp * gz[z] * gy[y] * gx[x] : 0.0;
    }
}

__global__ void k_axpby(double a, const double *x, double b, double *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void k_convert(const T *x, double *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

template <typename T>
__global__ void k_convert_from(const double *x, T *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)x[i];
}

// Neumaier-compensated (sum, correction) pairs, combined by two-sum.
__device__ __forceinline__ void two_sum_add(double &s, double &c, double v)
{
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

__global__ void k_dot_partial(const double *x, const double *y, long long n, double *partial)
{
    __shared__ double ss[256], sc[256];
    double s = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        two_sum_add(s, c, x[i] * y[i]);
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            double s1 = ss[threadIdx.x], c1 = sc[threadIdx.x];
            two_sum_add(s1, c1, ss[threadIdx.x + h]);
            ss[threadIdx.x] = s1;
            sc[threadIdx.x] = c1 + sc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = ss[0];
        partial[2 * blockIdx.x + 1] = sc[0];
    }
}

__global__ void k_dot_final(const double *partial, int nb, double *result)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nb; ++b) {
        two_sum_add(s, c, partial[2 * b]);
        c += partial[2 * b + 1];
    }
    result[0] = s + c;
}

template <typename T>
__global__ void k_lincomb(T *out, T a, const T *x, T b, const T *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : T(0));
}

template <typename T>
__global__ void k_atm_update(T *U, T *Up, const T *d, long long n, long long *step)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && step) step[0] += 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T u = U[i];
        U[i] = T(2) * u - Up[i] + d[i];
        Up[i] = u;
    }
}

// One CTA waits on an mbarrier whose transaction bytes never arrive (no
// copy is issued): the bounded wait must run out and record the timeout.
__global__ void k_wait_selftest(long long cycles, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, 16);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, err, cycles))) return;
    if (threadIdx.x == 0) atomicExch(err + 1, 1);   // the wait completed (not expected)
}

__global__ void k_delay(unsigned long long ns)
{
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    t = t0;
    while (t - t0 < ns) {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    }
}

template <typename T>
__global__ void k_pq_update(T *P, T *Q, T *A, const T *x, long long n, T tau2, int write_a, long long *step)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && step) step[0] += 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T a = x[i];
        const T q = Q[i] + tau2 * a;
        Q[i] = q;
        P[i] += q;
        if (write_a) A[i] = a;
    }
}

template <typename T>
__global__ void k_add_converted(const T *x, double *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += (double)x[i];
}

template <typename T>
__global__ void k_add_source(T *out, Dims d, const T *fx, const T *fy, const T *fz, double scale, double freq,
                             double t0, const long long *step, int toff, double tau)
{
    __shared__ T s_c;
    if (threadIdx.x == 0) s_c = (T)(scale * ricker_dev(freq, t0, (double)(step[0] + toff) * tau));
    __syncthreads();
    const T c = s_c;
    const long long n = d.count();
    const long long plane = d.plane();
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / plane);
        const long long rem = idx - (long long)z * plane;
        const int y = (int)(rem / d.sx);
        const int x = (int)(rem - (long long)y * d.sx);
        if (x < d.mx) out[idx] += c * fz[z] * fy[y] * fx[x];
    }
}

template <typename T>
__global__ void k_add_field(T *out, const T *field, long long n, double scale, double freq, double t0,
                            const long long *step, int toff, double tau)
{
    __shared__ T s_c;
    if (threadIdx.x == 0) s_c = (T)(scale * ricker_dev(freq, t0, (double)(step[0] + toff) * tau));
    __syncthreads();
    const T c = s_c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] += c * field[i];
}

template <typename T>
__global__ void k_el_to_uv(const T *U, const T *Up, double *u, double *v, long long n, double tau)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = (double)U[i], b = (double)Up[i];
        if (u) u[i] = a;
        if (v) v[i] = (a - b) / tau;
    }
}

inline int grid_for(long long n, int bs)
{
    long long g = (n + bs - 1) / bs;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3D map over an interior field [z][y][x] (dims mx, my, mz; row pitch sx)
bool make_map(CUtensorMap *m, const void *base, int elem, const Dims &d, int b0, int b1, int b2)
{
    auto fn = encode_fn();
    if (!fn || !base || ((uintptr_t)base & 15) || (((size_t)d.sx * elem) & 15)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)d.mx, (cuuint64_t)d.my, (cuuint64_t)d.mz};
    cuuint64_t strides[2] = {(cuuint64_t)d.sx * elem, (cuuint64_t)d.sx * d.my * elem};
    cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                    const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool make_update_maps(ColMaps *m, const void *P, const void *Q, int elem, const Dims &d, int axis)
{
    const int len = axis == 1 ? d.my : d.mz;
    const int box = col_box(len);
    const int b1 = axis == 1 ? box : 1, b2 = axis == 1 ? 1 : box;
    std::memset(m, 0, sizeof(*m));
    return make_map(&m->P, P, elem, d, 32, b1, b2) && make_map(&m->Q, Q, elem, d, 32, b1, b2);
}

namespace {
}  // namespace

size_t line_image_elems(int p, int S, int seg) { return (size_t)line_image_elems_dev(p, S * seg, S); }

size_t rhs_image_elems(int p, const Dims &d, int Sx, int Sy, int seg)
{
    const int W = 2 * p + 1, mxp = Sx * seg, myp = Sy * seg;
    (void)d;
    return 2 * (size_t)mxp * W + 2 * (size_t)myp * W + mxp + myp + line_image_elems(p, Sx, seg) +
           line_image_elems(p, Sy, seg);
}

size_t rhs_smem_bytes(int p, int elem, const Dims &d, int ty, int Sx, int Sy, int seg, int pair, int planes)
{
    const RhsPlan q = rhs_plan(d.mx, d.my, ty, pair, Sx, Sy);
    size_t n = (size_t)planes * q.rows * q.RS + 2 * (size_t)q.Smax * p * q.cld;
    size_t img = rhs_image_elems(p, d, Sx, Sy, seg);
    if (planes == 3) img += (size_t)Sx * seg * (2 * p + 1);   // Bx
    return n * elem + 32 + ((img * elem + 15) & ~(size_t)15);   // alignment of the carry buffers and tables
}

namespace {
// rounds of line groups (32 lines x S segment warps) in a CTA of `warps` warps
int line_rounds(int lines, int S, int warps)
{
    const int per = warps / S;
    if (per < 1) return 1 << 20;
    const int groups = (lines + 31) / 32;
    return (groups + per - 1) / per;
}
}  // namespace

int choose_seg(const int *m, int elem)
{
    int n32 = 0, n33 = 0;
    for (int a = 0; a < 3; ++a) {
        n32 += (m[a] + kSeg - 1) / kSeg;
        n33 += (m[a] + kSegAlt - 1) / kSegAlt;
    }
    int best = n33 < n32 ? kSegAlt : kSeg;
    // K1 (whole plane per CTA) runs the x sweep over my lines and the y sweep
    // over mx lines, line groups in rounds; a round lasts about one segment
    // of recurrences.  m = 129 (128 elements, p = 3): 33-row segments need
    // two rounds per sweep, 44-row segments one.
    const int warps = rhs_threads(elem) / 32;
    auto cost = [&](int seg) {
        const int Sx = (m[0] + seg - 1) / seg, Sy = (m[1] + seg - 1) / seg;
        if (Sx > 16 || Sy > 16) return 1 << 30;
        return seg * (line_rounds(m[1], Sx, warps) + line_rounds(m[0], Sy, warps));
    };
    // 44-row lines take at most 8 segments: K1 at 44 rows exists in the
    // single-CTA layout only, whose FP64 CTA (the set-up and residual sweeps
    // of every simulation) has 8 warps
    const int S44[3] = {(m[0] + kSegLong - 1) / kSegLong, (m[1] + kSegLong - 1) / kSegLong,
                        (m[2] + kSegLong - 1) / kSegLong};
    if (S44[0] <= 8 && S44[1] <= 8 && S44[2] <= 16 && cost(kSegLong) < cost(best)) best = kSegLong;
    return best;
}

int rhs_threads(int elem) { return elem == 8 ? 256 : 512; }

size_t col_smem_bytes(int p, int elem, int len, int S, int seg)
{
    (void)len;
    size_t n = 2 * (size_t)S * p * 32;
    return n * elem + 16 + ((line_image_elems(p, S, seg) * elem + 15) & ~(size_t)15);
}

#define ADS_DISPATCH_P(p, CALL)                      \
    switch (p) {                                     \
    case 1: return CALL(1);                          \
    case 2: return CALL(2);                          \
    case 3: return CALL(3);                          \
    case 4: return CALL(4);                          \
    default: return cudaErrorInvalidValue;           \
    }

template <typename T>
cudaError_t launch_rhs_group(int p, const RhsArgs<T> *a, int n, cudaStream_t s)
{
    if (!a || n <= 0 || p < 1 || p > 4) return cudaErrorInvalidValue;
    bool has[3] = {false, false, false};
    for (int i = 0; i < n; ++i) {
        const int seg = a[i].lx.seg;
        if (!seg_supported(seg)) return cudaErrorInvalidValue;
        // the cluster pair: FP32, at most 8 segments per line, 32- or 33-row segments
        if (a[i].pair && (sizeof(T) != 4 || a[i].lx.S > 8 || a[i].ly.S > 8 || seg == kSegLong))
            return cudaErrorInvalidValue;
        has[seg == kSeg ? 0 : seg == kSegAlt ? 1 : 2] = true;
    }
    cudaError_t e = cudaSuccess;
    if (has[0] && (e = launch_rhs_seg<T, kSeg>(p, a, n, s)) != cudaSuccess) return e;
    if (has[1] && (e = launch_rhs_seg<T, kSegAlt>(p, a, n, s)) != cudaSuccess) return e;
    if (has[2] && (e = launch_rhs_seg<T, kSegLong>(p, a, n, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_rhs(int p, int seg, const RhsArgs<T> &a, cudaStream_t s)
{
    if (!seg_supported(seg)) return cudaErrorInvalidValue;
    return launch_rhs_group<T>(p, &a, 1, s);
}

template <typename T>
cudaError_t launch_col(int p, int seg, const ColArgs<T> &a, cudaStream_t s)
{
    if (!seg_supported(seg)) return cudaErrorInvalidValue;
    return launch_col_group<T>(p, &a, nullptr, 1, s);
}

template <typename T>
cudaError_t launch_axis_apply(int p, const T *band, int axis, const T *in, T *out, Dims d, T alpha, T beta,
                              int transpose, cudaStream_t s)
{
    const int bs = 256;
    const int g = grid_for(d.count(), bs);
    ++g_launches;
#define C(P) (k_axis_apply<T, P><<<g, bs, 0, s>>>(band, axis, in, out, d, alpha, beta, transpose), cudaGetLastError())
    ADS_DISPATCH_P(p, C)
#undef C
}

template <typename T, int P>
cudaError_t kron_sum_impl(dim3 grid, size_t smem, cudaStream_t s, const KronSum<T> &ks, T *out, Dims d, int ty)
{
    static std::atomic<size_t> smem_set{48 * 1024};   // per instantiation (raised outside capture)
    cudaError_t e = raise_dyn_smem(k_kron_sum<T, P>, smem_set, smem);
    if (e != cudaSuccess) return e;
    k_kron_sum<T, P><<<grid, 256, smem, s>>>(ks, out, d, ty);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kron_sum(int p, const KronSum<T> &ks, T *out, Dims d, cudaStream_t s)
{
    if (ks.nt < 0 || ks.nt > kMaxKronTerms) return cudaErrorInvalidValue;
    // rows per tile: three buffers within 120 KB of shared memory
    const size_t row = (size_t)d.sx * sizeof(T);
    int ty = (int)((120 * 1024 / row - 2 * p) / 3);
    if (ty > 16) ty = 16;
    if (ty < 1) ty = 1;
    if (ty > d.my) ty = d.my;
    const size_t smem = (size_t)(3 * ty + 2 * p) * row;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    dim3 grid((d.my + ty - 1) / ty, d.mz);
    ++g_launches;
#define C(P) kron_sum_impl<T, P>(grid, smem, s, ks, out, d, ty)
    ADS_DISPATCH_P(p, C)
#undef C
}

template <typename T>
cudaError_t launch_solve_x(int p, const T *fac, T *data, Dims d, cudaStream_t s)
{
    const int bs = 128;
    const int g = (d.my * d.mz + bs - 1) / bs;
    ++g_launches;
#define C(P) (k_solve_x<T, P><<<g, bs, 0, s>>>(fac, data, d), cudaGetLastError())
    ADS_DISPATCH_P(p, C)
#undef C
}

template <typename T>
cudaError_t launch_pack(const double *full, T *in, Dims d, double scale, cudaStream_t s)
{
    ++g_launches;
    k_pack<T><<<grid_for(d.count(), 256), 256, 0, s>>>(full, in, d, scale);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(const T *in, double *full, Dims d, cudaStream_t s)
{
    ++g_launches;
    long long n = (long long)(d.mx + 2 * d.off) * (d.my + 2 * d.off) * (d.mz + 2 * d.offz);
    k_unpack<T><<<grid_for(n, 256), 256, 0, s>>>(in, full, d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_uva_to_pq(const double *u, const double *v, const double *a, T *P, T *Q, T *A, Dims d,
                             double tau, cudaStream_t s)
{
    ++g_launches;
    k_uva_to_pq<T><<<grid_for(d.count(), 256), 256, 0, s>>>(u, v, a, P, Q, A, d.count(), tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pq_to_uva(const T *P, const T *Q, const T *A, double *u, double *v, double *a, Dims d,
                             double tau, cudaStream_t s)
{
    ++g_launches;
    k_pq_to_uva<T><<<grid_for(d.count(), 256), 256, 0, s>>>(P, Q, A, u, v, a, d.count(), tau);
    return cudaGetLastError();
}

cudaError_t launch_outer(const double *gx, const double *gy, const double *gz, double amp, double *out, Dims d,
                         cudaStream_t s)
{
    ++g_launches;
    k_outer<<<grid_for(d.count(), 256), 256, 0, s>>>(gx, gy, gz, amp, out, d);
    return cudaGetLastError();
}

cudaError_t launch_axpby(double a, const double *x, double b, double *y, long long n, cudaStream_t s)
{
    ++g_launches;
    k_axpby<<<grid_for(n, 256), 256, 0, s>>>(a, x, b, y, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert(const T *x, double *y, long long n, cudaStream_t s)
{
    ++g_launches;
    k_convert<T><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_from(const double *x, T *y, long long n, cudaStream_t s)
{
    ++g_launches;
    k_convert_from<T><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_dot(const double *x, const double *y, long long n, double *partial, int nblocks, double *result,
                       cudaStream_t s)
{
    g_launches += 2;
    k_dot_partial<<<nblocks, 256, 0, s>>>(x, y, n, partial);
    k_dot_final<<<1, 32, 0, s>>>(partial, nblocks, result);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lincomb(T *out, T a, const T *x, T b, const T *y, long long n, cudaStream_t s)
{
    ++g_launches;
    k_lincomb<T><<<grid_for(n, 256), 256, 0, s>>>(out, a, x, b, y, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_atm_update(T *U, T *Up, const T *d, long long n, long long *step, cudaStream_t s)
{
    ++g_launches;
    k_atm_update<T><<<grid_for(n, 256), 256, 0, s>>>(U, Up, d, n, step);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long cycles, int *err, cudaStream_t s)
{
    k_wait_selftest<<<1, 64, 0, s>>>(cycles, err);
    return cudaGetLastError();
}

cudaError_t launch_delay(unsigned long long ns, cudaStream_t s)
{
    k_delay<<<1, 1, 0, s>>>(ns);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pq_update(T *P, T *Q, T *A, const T *x, long long n, T tau2, int write_a, long long *step,
                             cudaStream_t s)
{
    ++g_launches;
    k_pq_update<T><<<grid_for(n, 256), 256, 0, s>>>(P, Q, A, x, n, tau2, write_a, step);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_converted(const T *x, double *y, long long n, cudaStream_t s)
{
    ++g_launches;
    k_add_converted<T><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_source(T *out, Dims d, const T *fx, const T *fy, const T *fz, double scale, double freq,
                              double t0, const long long *step, int toff, double tau, cudaStream_t s)
{
    ++g_launches;
    k_add_source<T><<<grid_for(d.count(), 256), 256, 0, s>>>(out, d, fx, fy, fz, scale, freq, t0, step, toff, tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_field(T *out, const T *field, long long n, double scale, double freq, double t0,
                             const long long *step, int toff, double tau, cudaStream_t s)
{
    ++g_launches;
    k_add_field<T><<<grid_for(n, 256), 256, 0, s>>>(out, field, n, scale, freq, t0, step, toff, tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_el_to_uv(const T *U, const T *Up, double *u, double *v, long long n, double tau, cudaStream_t s)
{
    ++g_launches;
    k_el_to_uv<T><<<grid_for(n, 256), 256, 0, s>>>(U, Up, u, v, n, tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs_el(int p, const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s)
{
    switch (a.lx.seg) {
    case kSeg: return launch_rhs_el_seg<T, kSeg>(p, a, el, s);
    case kSegAlt: return launch_rhs_el_seg<T, kSegAlt>(p, a, el, s);
    case kSegLong: return launch_rhs_el_seg<T, kSegLong>(p, a, el, s);
    default: return cudaErrorInvalidValue;
    }
}

#define ADS_INST(T)                                                                                                \
    template cudaError_t launch_rhs<T>(int, int, const RhsArgs<T> &, cudaStream_t);                                \
    template cudaError_t launch_rhs_group<T>(int, const RhsArgs<T> *, int, cudaStream_t);                         \
    template cudaError_t launch_rhs_el<T>(int, const RhsArgs<T> &, const RhsElas<T> &, cudaStream_t);             \
    template cudaError_t launch_col<T>(int, int, const ColArgs<T> &, cudaStream_t);                                \
    template cudaError_t launch_axis_apply<T>(int, const T *, int, const T *, T *, Dims, T, T, int, cudaStream_t); \
    template cudaError_t launch_solve_x<T>(int, const T *, T *, Dims, cudaStream_t);                               \
    template cudaError_t launch_kron_sum<T>(int, const KronSum<T> &, T *, Dims, cudaStream_t);                     \
    template cudaError_t launch_pack<T>(const double *, T *, Dims, double, cudaStream_t);                          \
    template cudaError_t launch_unpack<T>(const T *, double *, Dims, cudaStream_t);                                \
    template cudaError_t launch_uva_to_pq<T>(const double *, const double *, const double *, T *, T *, T *, Dims,  \
                                             double, cudaStream_t);                                                \
    template cudaError_t launch_pq_to_uva<T>(const T *, const T *, const T *, double *, double *, double *, Dims,  \
                                             double, cudaStream_t);                                                \
    template cudaError_t launch_convert<T>(const T *, double *, long long, cudaStream_t);                          \
    template cudaError_t launch_convert_from<T>(const double *, T *, long long, cudaStream_t);                      \
    template cudaError_t launch_lincomb<T>(T *, T, const T *, T, const T *, long long, cudaStream_t);              \
    template cudaError_t launch_atm_update<T>(T *, T *, const T *, long long, long long *, cudaStream_t);          \
    template cudaError_t launch_pq_update<T>(T *, T *, T *, const T *, long long, T, int, long long *, cudaStream_t); \
    template cudaError_t launch_add_converted<T>(const T *, double *, long long, cudaStream_t);                     \
    template cudaError_t launch_add_source<T>(T *, Dims, const T *, const T *, const T *, double, double, double,   \
                                              const long long *, int, double, cudaStream_t);                       \
    template cudaError_t launch_add_field<T>(T *, const T *, long long, double, double, double, const long long *, \
                                             int, double, cudaStream_t);                                           \
    template cudaError_t launch_el_to_uv<T>(const T *, const T *, double *, double *, long long, double, cudaStream_t);

ADS_INST(float)
ADS_INST(double)

}  // namespace ads
