// kernels.cu -- device kernels of the ADS/IGA time step (sm_103a).
//
// Hot path of one scalar-wave step (Sec. 2, eq. pwave2; Appendix):
//   K1  k_rhs   : sum-factorised RHS  F(t_{n+1}) - K p_n  on a tile of x-lines,
//                 then the x-direction banded forward/back substitution of
//                 (Mx + eta Kx) on every line of the tile (thread per line),
//                 optionally also the y-direction sweep when a tile spans the
//                 whole y extent (then K2 is skipped);
//   K2  k_col(y): y-direction sweep, thread per x column, coalesced rows;
//   K3  k_col(z): z-direction sweep + Newmark update of the (p, q) state.
// The remaining kernels serve set-up, the boundary and diagnostics.
#include "kernels.cuh"

#include <cstdio>
#include <cstring>

#include <cudaTypedefs.h>

#include "tma.cuh"

namespace ads {

unsigned long long g_launches = 0;

namespace {

constexpr int kSeg = 32;   // rows per register segment of the line solves

__device__ __forceinline__ double ricker_dev(double f, double t0, double t)
{
    const double pi = 3.141592653589793238462643;
    double a = pi * pi * f * f * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}


// ---------------------------------------------------------------- shared helpers

// cooperative copy of n elements global -> shared
template <typename T>
__device__ __forceinline__ void stage(T *dst, const T *src, int n, int tid, int nt)
{
    for (int i = tid; i < n; i += nt) dst[i] = src[i];
}

// Shared-memory image of the tables of one directional factor set.
template <typename T>
struct LineSm {
    T *fac, *phi, *psi, *Phi, *Psi;
    int S;
};

template <typename T, int P>
__host__ __device__ __forceinline__ size_t line_sm_elems(int m, int S)
{
    return (size_t)m * (2 * P + 1) + 2 * (size_t)m * P + 2 * (size_t)S * P * P;
}

// pointers into a shared-memory copy of a LineDev buffer (m = S * SEG rows)
template <typename T, int P>
__device__ __forceinline__ LineSm<T> line_carve(T *base, int m, int S)
{
    LineSm<T> l;
    l.S = S;
    l.fac = base; base += (size_t)m * (2 * P + 1);
    l.phi = base; base += (size_t)m * P;
    l.psi = base; base += (size_t)m * P;
    l.Phi = base; base += (size_t)S * P * P;
    l.Psi = base;
    return l;
}

__host__ __device__ __forceinline__ int line_image_elems_dev(int p, int m, int S)
{
    return m * (2 * p + 1) + 2 * m * p + 2 * S * p * p;
}

// ------------------------------------------------ segment-parallel solve
//
// A line of length m is cut into segments of SEG rows (the last may be
// shorter).  The thread owning segment s keeps its rows in registers
// v[0..SEG) (rows s*SEG + k; v[k] = 0 past the line end) and runs:
//   pass 1  local forward substitution with zero carry-in
//   (carry)  c_s = sum over earlier segments through the transfer matrices Phi
//   pass 2  forward correction v += sum_k c_s[k] phi[.][k], fused with the
//           local backward substitution (zero carry-in from below)
//   (carry)  e_s through Psi from later segments
//   pass 3  backward correction v += sum_k e_s[k] psi[.][k]
// which equals plain forward/back substitution of the banded LU (Appendix)
// up to rounding order.  Every loop is fully unrolled over SEG, so each
// element of v is a register.

// The 1D tables are padded to whole segments (identity factor rows, zero
// fundamental solutions beyond the line end), so every segment is full and
// the passes need no predicates.  fb/pb: the segment's rows of fac/phi.
template <typename T, int P, int SEG>
__device__ __forceinline__ void seg_pass1(const T *fb, T (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        T w = v[k];
#pragma unroll
        for (int q = 1; q <= P; ++q)
            if (k - q >= 0) w -= fb[k * W + P - q] * v[k - q];
        v[k] = w;
    }
}

template <typename T, int P, int SEG>
__device__ __forceinline__ void seg_pass2(const T *fb, const T *pb, const T (&c)[P], T (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
#pragma unroll
    for (int k = SEG - 1; k >= 0; --k) {
        T w = v[k];
#pragma unroll
        for (int q = 0; q < P; ++q) w += c[q] * pb[k * P + q];
#pragma unroll
        for (int q = 1; q <= P; ++q)
            if (k + q < SEG) w -= fb[k * W + P + q] * v[k + q];
        v[k] = w * fb[k * W + P];
    }
}

template <typename T, int P, int SEG>
__device__ __forceinline__ void seg_pass3(const T *qb, const T (&e)[P], T (&v)[SEG])
{
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        T x = v[k];
#pragma unroll
        for (int q = 0; q < P; ++q) x += e[q] * qb[k * P + q];
        v[k] = x;
    }
}

template <typename T, int P>
__device__ __forceinline__ void carry_fwd(const T *Phi, int s, const T *CT, int ld, int j, T (&c)[P])
{
#pragma unroll
    for (int k = 0; k < P; ++k) c[k] = T(0);
    for (int q = 0; q < s; ++q) {
        T n[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            T acc = CT[(q * P + k) * ld + j];
#pragma unroll
            for (int r = 0; r < P; ++r) acc += Phi[(q * P + k) * P + r] * c[r];
            n[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < P; ++k) c[k] = n[k];
    }
}

template <typename T, int P>
__device__ __forceinline__ void carry_bwd(const T *Psi, int S, int s, const T *CH, int ld, int j, T (&e)[P])
{
#pragma unroll
    for (int k = 0; k < P; ++k) e[k] = T(0);
    for (int q = S - 1; q > s; --q) {
        T n[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            T acc = CH[(q * P + k) * ld + j];
#pragma unroll
            for (int r = 0; r < P; ++r) acc += Psi[(q * P + k) * P + r] * e[r];
            n[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < P; ++k) e[k] = n[k];
    }
}

// Passes 2-3 with the two carry exchanges, after pass 1 left v in
// registers.  All threads of the block call it (it synchronises); `on`
// marks threads that own a segment.  CT/CH: [S][P][ld], slot j.
template <typename T, int P, int SEG>
__device__ __forceinline__ void seg_finish(const LineSm<T> &L, bool on, int s, int j, int ld, T *CT, T *CH,
                                           T (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
    const int b0 = s * SEG;
    if (on) {
#pragma unroll
        for (int k = 0; k < P; ++k) CT[(s * P + k) * ld + j] = v[SEG - 1 - k];
    }
    __syncthreads();
    if (on) {
        T c[P];
        carry_fwd<T, P>(L.Phi, s, CT, ld, j, c);
        seg_pass2<T, P, SEG>(L.fac + b0 * W, L.phi + b0 * P, c, v);
#pragma unroll
        for (int k = 0; k < P; ++k) CH[(s * P + k) * ld + j] = v[k];
    }
    __syncthreads();
    if (on) {
        T e[P];
        carry_bwd<T, P>(L.Psi, L.S, s, CH, ld, j, e);
        seg_pass3<T, P, SEG>(L.psi + b0 * P, e, v);
    }
}

// band row of a Toeplitz-interior band: registers inside [lo, hi), table outside
template <typename T, int W>
__device__ __forceinline__ void band_row(const T *tab, int lo, int hi, const T (&mid)[W], int i, T (&r)[W])
{
    if (i >= lo && i < hi) {
#pragma unroll
        for (int k = 0; k < W; ++k) r[k] = mid[k];
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) r[k] = tab[i * W + k];
    }
}

// Phase 1 of K1 for the column pair (x, x+1) and output rows [yb, ye):
// stream the rows yp = yb-P .. ye+P-1, z-contract each (t1 = Mz p,
// t2 = Kz p) into a ring of W slots, and y-contract every complete window
// into s1, s2.  The loop is unrolled by W so that ring slots are static
// registers.  GUARD: rows or planes may fall outside the grid (zero);
// INTERIOR: every output row lies in the Toeplitz range (band rows from
// registers).  Column x+1 may be the zero padding of the row (x+1 = mx).
template <typename T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };

template <typename T, int P, bool GUARD, bool INTERIOR>
__device__ __forceinline__ void phase1_chunk(const T *col0, long long plane, int sx, int my, const bool (&zok)[2 * P + 1],
                                             const T (&cm)[2 * P + 1], const T (&ck)[2 * P + 1],
                                             const T (&mym)[2 * P + 1], const T (&myk)[2 * P + 1], const T *bMy,
                                             const T *bKy, int ylo, int yhi, int yb, int ye, T *s1col, T *s2col, int RS)
{
    constexpr int W = 2 * P + 1;
    using V2 = typename Vec2<T>::type;
    T r1[W][2], r2[W][2];
#pragma unroll
    for (int k = 0; k < W; ++k) r1[k][0] = r1[k][1] = r2[k][0] = r2[k][1] = T(0);
    const int n = ye - yb + 2 * P;
    const T *rowp = col0 + (long long)(yb - P) * sx;
    for (int r0 = 0; r0 < n; r0 += W) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int r = r0 + j;
            const int yp = yb - P + r;
            const bool ok = GUARD ? ((r < n) && yp >= 0 && yp < my) : (r < n);
            const T *c = rowp + (long long)r * sx;
            V2 v[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const bool okk = GUARD ? (ok && zok[k]) : ok;
                v[k] = okk ? *reinterpret_cast<const V2 *>(c + (long long)k * plane) : V2{T(0), T(0)};
            }
            T t10 = T(0), t11 = T(0), t20 = T(0), t21 = T(0);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                t10 += cm[k] * v[k].x;
                t11 += cm[k] * v[k].y;
                t20 += ck[k] * v[k].x;
                t21 += ck[k] * v[k].y;
            }
            r1[j][0] = t10; r1[j][1] = t11;
            r2[j][0] = t20; r2[j][1] = t21;
            if (r >= 2 * P && r < n) {
                const int y = yb + r - 2 * P;
                T bm[W], bk[W];
                if (INTERIOR) {
#pragma unroll
                    for (int q = 0; q < W; ++q) { bm[q] = mym[q]; bk[q] = myk[q]; }
                } else {
                    band_row<T, W>(bMy, ylo, yhi, mym, y, bm);
                    band_row<T, W>(bKy, ylo, yhi, myk, y, bk);
                }
                T a0 = T(0), a1 = T(0), c0 = T(0), c1 = T(0);
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    // window row y-P+q = stream index r-2P+q  ->  ring slot (j-2P+q) mod W
                    const int sl = (j - 2 * P + q + 2 * W) % W;
                    a0 += bm[q] * r1[sl][0];
                    a1 += bm[q] * r1[sl][1];
                    c0 += bk[q] * r1[sl][0] + bm[q] * r2[sl][0];
                    c1 += bk[q] * r1[sl][1] + bm[q] * r2[sl][1];
                }
                s1col[(size_t)y * RS] = a0;
                s1col[(size_t)y * RS + 1] = a1;
                s2col[(size_t)y * RS] = c0;
                s2col[(size_t)y * RS + 1] = c1;
            }
        }
    }
}

// Phase 2 of K1, pass 1 for one row segment [b0, b0+n): form
//   R = F - c2 (Kx s1 + Mx s2)
// from the s1, s2 rows with a static register window and run the local
// forward substitution on it.  FAST: a full segment inside the Toeplitz
// range (no predicates, band rows in registers).
// Segment kinds of the x-direction pass 1.
enum { kSegMiddle = 0, kSegFirst = 1, kSegLast = 2, kSegGeneral = 3 };
constexpr int kHeadRows = 8;   // leading rows of the first segment read from the band table (>= Toeplitz lo)

template <typename T, int P, int SEG, int MODE>
__device__ __forceinline__ void phase2_fwd(const T *row1, const T *row2, int mx, int b0, const T (&mxm)[2 * P + 1],
                                           const T (&mxk)[2 * P + 1], const T *bMx, const T *bKx, int xlo, int xhi,
                                           const T *fb, const T *fx, T rowF, T c2, T (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
    T a1[SEG + 2 * P], a2[SEG + 2 * P];   // window positions b0-P .. b0+SEG+P-1 (static after unrolling)
#pragma unroll
    for (int j = 0; j < SEG + 2 * P; ++j) {
        const int xx = b0 - P + j;
        bool in_;
        if (MODE == kSegMiddle) in_ = true;
        else if (MODE == kSegFirst) in_ = j >= P;                  // x < 0 is outside
        else if (MODE == kSegLast) in_ = xx < mx;                  // b0 - P >= 0 here
        else in_ = xx >= 0 && xx < mx;
        a1[j] = in_ ? row1[xx] : T(0);
        a2[j] = in_ ? row2[xx] : T(0);
    }
    const T *fxb = fx ? fx + b0 : nullptr;
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        const int x = b0 + k;
        T bm[W], bk[W];
        const bool table = MODE == kSegLast || (MODE == kSegFirst && k < kHeadRows);
        if (MODE == kSegGeneral) {
            band_row<T, W>(bMx, xlo, xhi, mxm, x, bm);   // rows past the line end are zero
            band_row<T, W>(bKx, xlo, xhi, mxk, x, bk);
        } else if (table) {
#pragma unroll
            for (int q = 0; q < W; ++q) { bm[q] = bMx[x * W + q]; bk[q] = bKx[x * W + q]; }
        } else {
#pragma unroll
            for (int q = 0; q < W; ++q) { bm[q] = mxm[q]; bk[q] = mxk[q]; }
        }
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < W; ++q) acc += bk[q] * a1[k + q] + bm[q] * a2[k + q];
        T w = (fxb ? rowF * fxb[k] : T(0)) - c2 * acc;
#pragma unroll
        for (int q = 1; q <= P; ++q)
            if (k - q >= 0) w -= fb[k * W + P - q] * v[k - q];
        v[k] = w;
    }
}

// ---------------------------------------------------------------- K1
//
// One CTA per (z-plane, y-tile of ty rows).  Shared memory: S1, S2 [ty][RS]
// (RS odd), carry buffers and the 1D tables.  Phases:
//  1. z- then y-contraction of p, thread per x, streaming along y with a
//     register window (loads prefetched two rows ahead):
//        s1 = (My.Mz) p,   s2 = (Ky.Mz + My.Kz) p       (K p = Kx s1 + Mx s2)
//  2. x-direction, thread per (row, segment of SEG): R = F - c2 (Kx s1 + Mx s2)
//     is formed in registers while the local forward pass runs, then the
//     carry exchange and passes 2-3; the row is written back to S1.
//  3. whole plane in the tile: y-direction solve, thread per (x, segment).
//  4. coalesced store.
template <typename T>
struct RhsThreads {
    static constexpr int value = sizeof(T) == 8 ? 256 : 512;   // FP64: more registers per thread
};

template <typename T, int P>
__global__ void __launch_bounds__(RhsThreads<T>::value, 1) k_rhs(const RhsArgs<T> a)
{
    constexpr int W = 2 * P + 1;
    constexpr int SEG = kSeg;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_r;
    const int mx = a.d.mx, my = a.d.my, mz = a.d.mz, sx = a.d.sx;
    const long long plane = (long long)sx * my;
    const int RS = ((mx + 1) & ~1) | 1;   // odd, holds every column pair
    const int ty = a.ty;
    const int y0 = blockIdx.x * ty, z = blockIdx.y;
    const int tye = min(ty, my - y0);
    const bool fuse_y = (ty == my);
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
    const int rows_pad = (ty + 31) & ~31, cols_pad = (mx + 31) & ~31;
    const int cld = (fuse_y && cols_pad > rows_pad) ? cols_pad : rows_pad;

    __shared__ __align__(8) uint64_t bar;
    T *S1 = reinterpret_cast<T *>(smem_raw);
    T *S2 = S1 + (size_t)ty * RS;
    const int Smax = (fuse_y && a.ly.S > a.lx.S) ? a.ly.S : a.lx.S;
    T *CT = S2 + (size_t)ty * RS;
    T *CH = CT + (size_t)Smax * P * cld;
    // the 1D tables arrive as one bulk copy into a 16-byte aligned region
    T *tb = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(CH + (size_t)Smax * P * cld) + 15) & ~(uintptr_t)15);
    const int mxp = a.lx.S * SEG, myp = a.ly.S * SEG;   // padded table lengths
    T *bMx = tb;
    T *bKx = bMx + mxp * W;
    T *bMy = bKx + mxp * W;
    T *bKy = bMy + myp * W;
    T *sfx = bKy + myp * W;
    T *sfy = sfx + mxp;
    T *lxb = sfy + myp;
    T *lyb = lxb + line_image_elems_dev(P, mxp, a.lx.S);
    const LineSm<T> LX = line_carve<T, P>(lxb, mxp, a.lx.S);
    const LineSm<T> LY = line_carve<T, P>(lyb, myp, a.ly.S);
    const bool has_src = a.src.fx != nullptr;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (uint32_t)a.img_bytes);
        bulk_load(tb, a.img, (uint32_t)a.img_bytes, &bar);
        T r = T(0);
        if (has_src) {   // overlaps the copy
            double t = (double)(a.step[0] + a.toff) * a.tau;
            r = (T)(a.src.amp * ricker_dev(a.src.freq, a.src.t0, t));
        }
        s_r = r;
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, a.err)) return;   // error recorded for the host

    // ---- phase 1
    {
        T cm[W], ck[W], mym[W], myk[W];
        const int ylo = a.bandM[1].lo, yhi = a.bandM[1].hi;   // K shares M's interior range
        bool zok[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            cm[k] = a.bandM[2].v[z * W + k];
            ck[k] = a.bandK[2].v[z * W + k];
            const int mid = ylo < yhi ? ylo : 0;
            mym[k] = bMy[mid * W + k];
            myk[k] = bKy[mid * W + k];
            zok[k] = (z + k - P >= 0) && (z + k - P < mz);
        }
        const int npair = (mx + 1) >> 1;          // column pairs (the last may end in padding)
        const int XG = (npair + 31) >> 5;
        int YC = nwarps / XG;
        if (YC < 1) YC = 1;
        const int rows_per = (tye + YC - 1) / YC;
        const bool zin = z >= P && z + P < mz;
        for (int item = warp; item < XG * YC; item += nwarps) {
            const int xg = item % XG, yc = item / XG;
            const int pr = xg * 32 + lane;
            const int x = 2 * pr;
            const int yb = y0 + yc * rows_per;
            int ye = yb + rows_per;
            if (ye > y0 + tye) ye = y0 + tye;
            if (yb >= ye || pr >= npair) continue;
            const T *col0 = a.in + x + (long long)(z - P) * plane;   // plane z-P, row 0, column x
            T *c1 = S1 + x - (size_t)y0 * RS, *c2 = S2 + x - (size_t)y0 * RS;
            const bool guard = !zin || yb - P < 0 || ye + P > my;
            const bool inter = yb >= ylo && ye <= yhi;
            if (!guard && inter)
                phase1_chunk<T, P, false, true>(col0, plane, sx, my, zok, cm, ck, mym, myk, bMy, bKy, ylo, yhi, yb, ye, c1, c2, RS);
            else if (!guard)
                phase1_chunk<T, P, false, false>(col0, plane, sx, my, zok, cm, ck, mym, myk, bMy, bKy, ylo, yhi, yb, ye, c1, c2, RS);
            else
                phase1_chunk<T, P, true, false>(col0, plane, sx, my, zok, cm, ck, mym, myk, bMy, bKy, ylo, yhi, yb, ye, c1, c2, RS);
        }
    }
    __syncthreads();

    // ---- phase 2: x-direction, thread per (row, segment); rounds of row groups
    const int RG = rows_pad >> 5;
    const int gpr2 = nwarps / LX.S > 0 ? nwarps / LX.S : 1;
    for (int g0 = 0; g0 < RG; g0 += gpr2) {
        const int gi = warp / LX.S, s = warp % LX.S;
        const int g = g0 + gi;
        const int l = g * 32 + lane;
        const bool on = gi < gpr2 && g < RG && l < tye;
        const int b0 = s * SEG;
        const int n = on ? min(SEG, mx - b0) : 0;
        T v[SEG];
#pragma unroll
        for (int k = 0; k < SEG; ++k) v[k] = T(0);
        if (on) {
            const T *row1 = S1 + (size_t)l * RS;
            const T *row2 = S2 + (size_t)l * RS;
            const int y = y0 + l;
            const T rowF = has_src ? s_r * sfy[y] * a.src.fz[z] : T(0);
            const T c2 = a.c2;
            const int xlo = a.bandM[0].lo, xhi = a.bandM[0].hi;
            T mxm[W], mxk[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int mid = xlo < xhi ? xlo : 0;
                mxm[k] = bMx[mid * W + k];
                mxk[k] = bKx[mid * W + k];
            }
            const T *srcF = has_src ? sfx : nullptr;
            const T *fb = LX.fac + b0 * W;
            // kinds: interior segments take bands from registers; the first reads its
            // head rows (< kHeadRows >= Toeplitz lo) from the table; the last reads
            // every row from the table (its rows past hi are not Toeplitz)
            const bool regular = LX.S >= 2 && xlo <= kHeadRows && xhi >= (LX.S - 1) * SEG && mx >= (LX.S - 1) * SEG + P;
            if (regular && s > 0 && s < LX.S - 1)
                phase2_fwd<T, P, SEG, kSegMiddle>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else if (regular && s == 0)
                phase2_fwd<T, P, SEG, kSegFirst>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else if (regular)
                phase2_fwd<T, P, SEG, kSegLast>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else
                phase2_fwd<T, P, SEG, kSegGeneral>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
        }
        seg_finish<T, P, SEG>(LX, on, s, l, cld, CT, CH, v);   // reads of S1/S2 are done (its first barrier)
        if (on) {
            T *row1 = S1 + (size_t)l * RS;
#pragma unroll
            for (int k = 0; k < SEG; ++k)
                if (k < n) row1[b0 + k] = v[k];
        }
        __syncthreads();
    }

    // ---- phase 3: y-direction (whole plane), thread per (x, segment); rounds of column groups
    if (fuse_y) {
        const int CG = cols_pad >> 5;
        const int gpr3 = nwarps / LY.S > 0 ? nwarps / LY.S : 1;
        for (int g0 = 0; g0 < CG; g0 += gpr3) {
            const int gi = warp / LY.S, s = warp % LY.S;
            const int x = (g0 + gi) * 32 + lane;
            const bool on = gi < gpr3 && x < mx;
            const int b0 = s * SEG;
            const int n = on ? min(SEG, my - b0) : 0;
            T v[SEG];
#pragma unroll
            for (int k = 0; k < SEG; ++k) v[k] = (k < n) ? S1[(size_t)(b0 + k) * RS + x] : T(0);
            if (on) seg_pass1<T, P, SEG>(LY.fac + b0 * W, v);
            seg_finish<T, P, SEG>(LY, on, s, x, cld, CT, CH, v);
            if (on) {
#pragma unroll
                for (int k = 0; k < SEG; ++k)
                    if (k < n) S1[(size_t)(b0 + k) * RS + x] = v[k];
            }
            __syncthreads();
        }
    }

    // ---- phase 4: store
    {
        T *dst0 = a.out + (long long)z * plane + (long long)y0 * sx;
        for (int l = warp; l < tye; l += nwarps) {
            const T *src = S1 + (size_t)l * RS;
            T *dst = dst0 + (long long)l * sx;
            for (int x = lane; x < mx; x += 32) dst[x] = src[x];
        }
    }
}

// ---------------------------------------------------------------- K2/K3
//
// 32 x-columns per CTA (lane = column), one warp per line segment of SEG
// rows held in registers (coalesced direct loads: a warp reads 32
// consecutive values of each row).  Epilogue: plain store, or the Newmark
// update of the (p, q) state, whose p and q tiles [len][32] are fetched by
// TMA at kernel start (overlapping the solve), updated in shared memory and
// written back by TMA stores.
struct ColMaps {
    CUtensorMap P, Q;
};

template <typename T, int P>
__global__ void __launch_bounds__(512) k_col(const __grid_constant__ ColMaps maps, const ColArgs<T> a, int box)
{
    constexpr int SEG = kSeg;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const Dims d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, s = tid >> 5;
    const int x0 = blockIdx.x * 32, x = x0 + lane;
    const int o = blockIdx.y;
    int len;
    long long stride, base;
    if (a.axis == 1) {
        len = d.my;
        stride = d.sx;
        base = (long long)o * d.plane();
    } else {
        len = d.mz;
        stride = d.plane();
        base = (long long)o * d.sx;
    }
    __shared__ __align__(8) uint64_t bar_tab;
    const bool upd = a.mode == 1;
    const int nch = upd ? (len + box - 1) / box : 0;
    const int rows = nch * box;
    unsigned char *sm = align128(smem_raw);   // the host reserves 128 spare bytes
    T *bufP = reinterpret_cast<T *>(sm);
    T *bufQ = bufP + (size_t)rows * 32;
    T *CT = bufQ + (size_t)rows * 32;
    T *CH = CT + (size_t)a.ln.S * P * 32;
    T *lb = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(CH + (size_t)a.ln.S * P * 32) + 15) & ~(uintptr_t)15);
    auto coords = [&](int c, int &c0, int &c1, int &c2) {
        c0 = x0;
        if (a.axis == 1) { c1 = c * box; c2 = o; }
        else { c1 = o; c2 = c * box; }
    };
    if (tid == 0) {
        mbar_init(&bar_tab, 1);
        if (upd) mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar_tab, (uint32_t)a.ln.bytes);
        bulk_load(lb, a.ln.base, (uint32_t)a.ln.bytes, &bar_tab);
        if (upd) {
            mbar_expect_tx(&bar, 2u * nch * 32u * box * sizeof(T));
            for (int c = 0; c < nch; ++c) {
                int c0, c1, c2;
                coords(c, c0, c1, c2);
                tma_load_3d(bufP + (size_t)c * box * 32, &maps.P, &bar, c0, c1, c2);
                tma_load_3d(bufQ + (size_t)c * box * 32, &maps.Q, &bar, c0, c1, c2);
            }
            if (blockIdx.x == 0 && blockIdx.y == 0) a.step[0] += 1;
        }
    }
    const bool on = x < d.mx && s < a.ln.S;
    const int b0 = s * SEG;
    const int n = on ? min(SEG, len - b0) : 0;
    T v[SEG];
    const T *__restrict__ in = a.in + base + x + (long long)b0 * stride;
#pragma unroll
    for (int k = 0; k < SEG; ++k) v[k] = (k < n) ? in[(long long)k * stride] : T(0);
    const LineSm<T> L = line_carve<T, P>(lb, a.ln.S * SEG, a.ln.S);
    __syncthreads();   // barriers initialised
    if (!mbar_wait_bounded(&bar_tab, 0, a.err)) return;
    if (on) seg_pass1<T, P, SEG>(L.fac + b0 * (2 * P + 1), v);
    seg_finish<T, P, SEG>(L, on, s, lane, 32, CT, CH, v);
    const long long off = base + x + (long long)b0 * stride;
    if (!upd) {
        if (!on) return;
        T *__restrict__ out = a.out + off;
#pragma unroll
        for (int k = 0; k < SEG; ++k)
            if (k < n) out[(long long)k * stride] = v[k];
        return;
    }
    if (!mbar_wait_bounded(&bar, 0, a.err)) return;   // error recorded for the host
    if (on) {
        const T tau2 = a.tau2;
#pragma unroll
        for (int k = 0; k < SEG; ++k) {
            if (k < n) {
                const int idx = (b0 + k) * 32 + lane;
                const T q = bufQ[idx] + tau2 * v[k];
                bufQ[idx] = q;
                bufP[idx] += q;
            }
        }
        if (a.write_a) {
            T *__restrict__ Ap = a.A + off;
#pragma unroll
            for (int k = 0; k < SEG; ++k)
                if (k < n) Ap[(long long)k * stride] = v[k];
        }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
        for (int c = 0; c < nch; ++c) {
            int c0, c1, c2;
            coords(c, c0, c1, c2);
            tma_store_3d(&maps.P, bufP + (size_t)c * box * 32, c0, c1, c2);
            tma_store_3d(&maps.Q, bufQ + (size_t)c * box * 32, c0, c1, c2);
        }
        tma_store_commit();
        tma_store_wait_read();
    }
}

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
    const int nx = d.mx + 2, ny = d.my + 2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / plane);
        const long long rem = idx - (long long)z * plane;
        const int y = (int)(rem / d.sx);
        const int x = (int)(rem - (long long)y * d.sx);
        T v = T(0);
        if (x < d.mx) v = (T)(scale * full[((long long)(z + 1) * ny + (y + 1)) * nx + (x + 1)]);
        in[idx] = v;
    }
}

template <typename T>
__global__ void k_unpack(const T *__restrict__ in, double *__restrict__ full, Dims d)
{
    const int nx = d.mx + 2, ny = d.my + 2, nz = d.mz + 2;
    const long long n = (long long)nx * ny * nz;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(idx / ((long long)nx * ny));
        const long long rem = idx - (long long)z * nx * ny;
        const int y = (int)(rem / nx);
        const int x = (int)(rem - (long long)y * nx);
        double v = 0.0;
        if (x >= 1 && x <= d.mx && y >= 1 && y <= d.my && z >= 1 && z <= d.mz)
            v = (double)in[(long long)(z - 1) * d.plane() + (long long)(y - 1) * d.sx + (x - 1)];
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

template <typename T, int P>
cudaError_t rhs_impl(const RhsArgs<T> &a, cudaStream_t s)
{
    const size_t smem = rhs_smem_bytes(P, sizeof(T), a.d, a.ty, a.lx.S, a.ly.S);
    static size_t smem_set = 48 * 1024;   // per instantiation: opt-in dynamic shared memory
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rhs<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    if (a.lx.S > 16 || a.ly.S > 16 || a.lx.S * kSeg < a.d.mx || !a.img || (a.img_bytes & 15) ||
        ((uintptr_t)a.img & 15))
        return cudaErrorInvalidValue;
    dim3 grid((a.d.my + a.ty - 1) / a.ty, a.d.mz);
    k_rhs<T, P><<<grid, RhsThreads<T>::value, smem, s>>>(a);
    ++g_launches;
    return cudaGetLastError();
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

template <typename T, int P>
cudaError_t col_impl(const ColArgs<T> &a, cudaStream_t s)
{
    const int len = a.axis == 1 ? a.d.my : a.d.mz;
    const int outer = a.axis == 1 ? a.d.mz : a.d.my;
    if (a.ln.S * kSeg < len || a.ln.S > 16 || !a.ln.base || (a.ln.bytes & 15) || ((uintptr_t)a.ln.base & 15))
        return cudaErrorInvalidValue;
    const int nch = (len + 255) / 256;
    const int box = (len + nch - 1) / nch;
    ColMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    size_t tiles = 0;
    if (a.mode == 1) {
        const int b1 = a.axis == 1 ? box : 1, b2 = a.axis == 1 ? 1 : box;
        if (!make_map(&maps.P, a.P, sizeof(T), a.d, 32, b1, b2) || !make_map(&maps.Q, a.Q, sizeof(T), a.d, 32, b1, b2))
            return cudaErrorInvalidValue;
        tiles = 2 * (size_t)nch * box * 32 * sizeof(T);
    }
    const size_t smem = 128 + tiles + col_smem_bytes(P, sizeof(T), len, a.ln.S);
    static size_t smem_set = 48 * 1024;
    if (smem > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(k_col<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    dim3 grid((a.d.mx + 31) / 32, outer);
    k_col<T, P><<<grid, 32 * a.ln.S, smem, s>>>(maps, a, box);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace

static size_t line_elems(int p, int m, int S) { return (size_t)m * (2 * p + 1) + 2 * (size_t)m * p + 2 * (size_t)S * p * p; }

size_t line_image_elems(int p, int S) { return (size_t)line_image_elems_dev(p, S * kSeg, S); }

size_t rhs_image_elems(int p, const Dims &d, int Sx, int Sy)
{
    const int W = 2 * p + 1, mxp = Sx * kSeg, myp = Sy * kSeg;
    (void)d;
    return 2 * (size_t)mxp * W + 2 * (size_t)myp * W + mxp + myp + line_image_elems(p, Sx) + line_image_elems(p, Sy);
}

size_t rhs_smem_bytes(int p, int elem, const Dims &d, int ty, int Sx, int Sy)
{
    const int RS = ((d.mx + 1) & ~1) | 1;
    const int rows_pad = (ty + 31) & ~31, cols_pad = (d.mx + 31) & ~31;
    const bool fuse = ty == d.my;
    const int cld = (fuse && cols_pad > rows_pad) ? cols_pad : rows_pad;
    const int Smax = (fuse && Sy > Sx) ? Sy : Sx;
    size_t n = 2 * (size_t)ty * RS + 2 * (size_t)Smax * p * cld;
    return n * elem + 16 + ((rhs_image_elems(p, d, Sx, Sy) * elem + 15) & ~(size_t)15);
}

int rhs_threads(int elem) { return elem == 8 ? 256 : 512; }

size_t col_smem_bytes(int p, int elem, int len, int S)
{
    (void)len;
    size_t n = 2 * (size_t)S * p * 32;
    return n * elem + 16 + ((line_image_elems(p, S) * elem + 15) & ~(size_t)15);
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
cudaError_t launch_rhs(int p, int seg, const RhsArgs<T> &a, cudaStream_t s)
{
    if (seg != kSeg) return cudaErrorInvalidValue;
#define C(P) rhs_impl<T, P>(a, s)
    ADS_DISPATCH_P(p, C)
#undef C
}

template <typename T>
cudaError_t launch_col(int p, int seg, const ColArgs<T> &a, cudaStream_t s)
{
    if (seg != kSeg) return cudaErrorInvalidValue;
#define C(P) col_impl<T, P>(a, s)
    ADS_DISPATCH_P(p, C)
#undef C
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
    long long n = (long long)(d.mx + 2) * (d.my + 2) * (d.mz + 2);
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

template <typename T>
cudaError_t launch_add_source(T *out, Dims d, const T *fx, const T *fy, const T *fz, double scale, double freq,
                              double t0, const long long *step, int toff, double tau, cudaStream_t s)
{
    ++g_launches;
    k_add_source<T><<<grid_for(d.count(), 256), 256, 0, s>>>(out, d, fx, fy, fz, scale, freq, t0, step, toff, tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_el_to_uv(const T *U, const T *Up, double *u, double *v, long long n, double tau, cudaStream_t s)
{
    ++g_launches;
    k_el_to_uv<T><<<grid_for(n, 256), 256, 0, s>>>(U, Up, u, v, n, tau);
    return cudaGetLastError();
}

#define ADS_INST(T)                                                                                                \
    template cudaError_t launch_rhs<T>(int, int, const RhsArgs<T> &, cudaStream_t);                                \
    template cudaError_t launch_col<T>(int, int, const ColArgs<T> &, cudaStream_t);                                \
    template cudaError_t launch_axis_apply<T>(int, const T *, int, const T *, T *, Dims, T, T, int, cudaStream_t); \
    template cudaError_t launch_solve_x<T>(int, const T *, T *, Dims, cudaStream_t);                               \
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
    template cudaError_t launch_add_source<T>(T *, Dims, const T *, const T *, const T *, double, double, double,   \
                                              const long long *, int, double, cudaStream_t);                       \
    template cudaError_t launch_el_to_uv<T>(const T *, const T *, double *, double *, long long, double, cudaStream_t);

ADS_INST(float)
ADS_INST(double)

}  // namespace ads
