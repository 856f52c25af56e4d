// sweep.cuh -- the hot-path kernels of the scalar-wave step (sm_103a) and
// their grouped launchers.  Included only by the translation units that
// instantiate them (rhs_f32.cu, rhs_f64.cu, col_f32.cu, col_f64.cu).
//
// Hot path of one scalar-wave step (Sec. 2, eq. pwave2; Appendix):
//   K1  k_rhs   : sum-factorised RHS  F(t_{n+1}) - K p_n  on a tile of x-lines,
//                 then the x-direction banded forward/back substitution of
//                 (Mx + eta Kx) on every line of the tile, and the y-direction
//                 sweep when a tile spans the whole y extent (then K2 is skipped);
//   K2  k_col(y): y-direction sweep, 32 x-columns per CTA, coalesced rows;
//   K3  k_col(z): z-direction sweep + Newmark update of the (p, q) state.
// Every kernel takes a group of up to NB independent simulations (same
// degree and precision, any grid): the flat block index is split into
// per-simulation ranges (RhsGroup::off / ColGroup::off), so one launch
// advances a whole batch; NB = 1 is the single-simulation launch.
#pragma once
#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace ads {
namespace {


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
// The recurrences below subtract the oldest neighbour first and the newest
// (v[k-1], resp. v[k+1]) last, so only one FMA per row sits on the chain
// that runs through the segment; everything else overlaps it.
// Value type V of the line values: T (one line per thread), or float2 for
// FP32 lines handled in pairs (two lines of the same 1D operator share every
// coefficient load, and one packed FFMA2 does both lines' multiply-add).
// c + a v and v a with a coefficient a of the 1D tables:
__device__ __forceinline__ float madd(float a, float v, float c) { return fmaf(a, v, c); }
__device__ __forceinline__ double madd(double a, double v, double c) { return fma(a, v, c); }
__device__ __forceinline__ float2 madd(float a, float2 v, float2 c) { return __ffma2_rn(make_float2(a, a), v, c); }
__device__ __forceinline__ float mulc(float v, float a) { return v * a; }
__device__ __forceinline__ double mulc(double v, double a) { return v * a; }
__device__ __forceinline__ float2 mulc(float2 v, float a) { return __fmul2_rn(v, make_float2(a, a)); }
template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float vzero<float>() { return 0.0f; }
template <>
__device__ __forceinline__ double vzero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.0f, 0.0f); }

template <typename T, int P, int SEG, typename V = T>
__device__ __forceinline__ void seg_pass1(const T *fb, V (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        V w = v[k];
#pragma unroll
        for (int q = P; q >= 1; --q)
            if (k - q >= 0) w = madd(-fb[k * W + P - q], v[k - q], w);
        v[k] = w;
    }
}

template <typename T, int P, int SEG, typename V = T>
__device__ __forceinline__ void seg_pass2(const T *fb, const T *pb, const V (&c)[P], V (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
    // forward correction first: independent per row, off the chain
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        V w = v[k];
#pragma unroll
        for (int q = 0; q < P; ++q) w = madd(pb[k * P + q], c[q], w);
        v[k] = w;
    }
#pragma unroll
    for (int k = SEG - 1; k >= 0; --k) {
        V w = v[k];
#pragma unroll
        for (int q = P; q >= 1; --q)
            if (k + q < SEG) w = madd(-fb[k * W + P + q], v[k + q], w);
        v[k] = mulc(w, fb[k * W + P]);
    }
}

template <typename T, int P, int SEG, typename V = T>
__device__ __forceinline__ void seg_pass3(const T *qb, const V (&e)[P], V (&v)[SEG])
{
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        V x = v[k];
#pragma unroll
        for (int q = 0; q < P; ++q) x = madd(qb[k * P + q], e[q], x);
        v[k] = x;
    }
}

template <typename T, int P, typename V = T>
__device__ __forceinline__ void carry_fwd(const T *Phi, int s, const V *CT, int ld, int j, V (&c)[P])
{
#pragma unroll
    for (int k = 0; k < P; ++k) c[k] = vzero<V>();
    for (int q = 0; q < s; ++q) {
        V n[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            V acc = CT[(q * P + k) * ld + j];
#pragma unroll
            for (int r = 0; r < P; ++r) acc = madd(Phi[(q * P + k) * P + r], c[r], acc);
            n[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < P; ++k) c[k] = n[k];
    }
}

template <typename T, int P, typename V = T>
__device__ __forceinline__ void carry_bwd(const T *Psi, int S, int s, const V *CH, int ld, int j, V (&e)[P])
{
#pragma unroll
    for (int k = 0; k < P; ++k) e[k] = vzero<V>();
    for (int q = S - 1; q > s; --q) {
        V n[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            V acc = CH[(q * P + k) * ld + j];
#pragma unroll
            for (int r = 0; r < P; ++r) acc = madd(Psi[(q * P + k) * P + r], e[r], acc);
            n[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < P; ++k) e[k] = n[k];
    }
}

// Barrier of the warps that share lines: the whole block (id 0), or a named
// barrier of `nthreads` threads (the S warps of one line group).
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    if (id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Passes 2-3 with the two carry exchanges, after pass 1 left v in
// registers.  Every thread of the synchronising group calls it (barrier id
// 0: the whole block; else the named barrier of one line group); `on` marks
// threads that own a segment.  CT/CH: [S][P][ld], slot j.
template <typename T, int P, int SEG, typename V = T>
__device__ __forceinline__ void seg_finish(const LineSm<T> &L, bool on, int s, int j, int ld, V *CT, V *CH,
                                           V (&v)[SEG], int bar_id = 0, int bar_threads = 0)
{
    constexpr int W = 2 * P + 1;
    const int b0 = s * SEG;
    if (on) {
#pragma unroll
        for (int k = 0; k < P; ++k) CT[(s * P + k) * ld + j] = v[SEG - 1 - k];
    }
    group_sync(bar_id, bar_threads);
    if (on) {
        V c[P];
        carry_fwd<T, P, V>(L.Phi, s, CT, ld, j, c);
        seg_pass2<T, P, SEG, V>(L.fac + b0 * W, L.phi + b0 * P, c, v);
#pragma unroll
        for (int k = 0; k < P; ++k) CH[(s * P + k) * ld + j] = v[k];
    }
    group_sync(bar_id, bar_threads);
    if (on) {
        V e[P];
        carry_bwd<T, P, V>(L.Psi, L.S, s, CH, ld, j, e);
        seg_pass3<T, P, SEG, V>(L.psi + b0 * P, e, v);
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
// registers.  Rows and planes outside the grid are read clamped and meet
// zero band entries (see phase1_chunk).  Column x+1 may be the zero padding
// of the row (x+1 = mx).
template <typename T>
struct Vec2;
template <>
struct Vec2<float> { using type = float2; };
template <>
struct Vec2<double> { using type = double2; };

__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// c + a * b on a pair of columns: one packed FP32 FMA (FFMA2) for float
__device__ __forceinline__ float2 fma2(float a, float2 b, float2 c) { return __ffma2_rn(make_float2(a, a), b, c); }
__device__ __forceinline__ double2 fma2(double a, double2 b, double2 c)
{
    return make_double2(fma(a, b.x, c.x), fma(a, b.y, c.y));
}

constexpr int kPhase1Lookahead = 1;   // stream rows whose loads are in flight ahead of the one contracted

// Rows and planes outside the grid need no predicates: the band rows of M
// and K hold zeros outside the matrix, so the loads read a clamped (valid)
// row or plane and the zero coefficient drops its value.  zoff[k]: element
// offset of plane clamp(z-P+k) (uniform over the CTA).
// SC (the elastic K1): s2 = cy (Ky t1) + cz (My t2), the two contractions
// scaled after they are formed.
// MASS (the elastic K1's upper blocks, cy = cz = 0): only s1 = My Mz p; s2 = 0.
template <typename T, int P, bool INTERIOR, bool SC = false, bool MASS = false, int PF = kPhase1Lookahead>
__device__ __forceinline__ void phase1_chunk(const T *colx, const long long (&zoff)[2 * P + 1], int sx, int my,
                                             const T (&cm)[2 * P + 1], const T (&ck)[2 * P + 1],
                                             const T (&mym)[2 * P + 1], const T (&myk)[2 * P + 1], const T *bMy,
                                             const T *bKy, int ylo, int yhi, int yb, int ye, T *s1col, T *s2col, int RS,
                                             T cy = T(1), T cz = T(1))
{
    constexpr int W = 2 * P + 1;
    using V2 = typename Vec2<T>::type;
    V2 r1[W], r2[W];   // ring of z-contracted rows (t1 = Mz p, t2 = Kz p) for the column pair
#pragma unroll
    for (int k = 0; k < W; ++k) r1[k] = r2[k] = V2{T(0), T(0)};
    const int n = ye - yb + 2 * P;
    // the W plane values of stream row r (row clamped into the grid: rows
    // outside it, and those past the chunk, meet zero band entries or none)
    auto load_row = [&](int r, V2(&dst)[W]) {
        const int yp = min(max(yb - P + r, 0), my - 1);
        const T *c = colx + (long long)yp * sx;
#pragma unroll
        for (int k = 0; k < W; ++k) dst[k] = *reinterpret_cast<const V2 *>(c + zoff[k]);
    };
    // rows r .. r+PF-1 in flight: row r+PF's loads are issued before row r is contracted
    V2 pf[PF][W];
#pragma unroll
    for (int d = 0; d < PF; ++d) load_row(d, pf[d]);
    // one block of W stream rows (ring slots static after unrolling); TAIL:
    // the last, partial block stops at the stream end (a check that full
    // blocks do without: it would keep the next row's loads from being
    // hoisted)
    auto block = [&](int r0, auto tail) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int r = r0 + j;
            if constexpr (decltype(tail)::value) {
                if (r >= n) break;
            }
            V2 nv[W];
            load_row(r + PF, nv);
            const V2(&v)[W] = pf[0];
            V2 t1 = V2{T(0), T(0)}, t2 = V2{T(0), T(0)};
#pragma unroll
            for (int k = 0; k < W; ++k) {
                t1 = fma2(cm[k], v[k], t1);
                if (!MASS) t2 = fma2(ck[k], v[k], t2);
            }
            r1[j] = t1;
            r2[j] = t2;
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
                V2 a = V2{T(0), T(0)}, c = V2{T(0), T(0)}, c2 = V2{T(0), T(0)};
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    // window row y-P+q = stream index r-2P+q  ->  ring slot (j-2P+q) mod W
                    const int sl = (j - 2 * P + q + 2 * W) % W;
                    a = fma2(bm[q], r1[sl], a);
                    if (MASS) continue;
                    c = fma2(bk[q], r1[sl], c);
                    if (SC) c2 = fma2(bm[q], r2[sl], c2);
                    else c = fma2(bm[q], r2[sl], c);
                }
                if (SC) {
                    c.x = cy * c.x + cz * c2.x;
                    c.y = cy * c.y + cz * c2.y;
                }
                s1col[(size_t)y * RS] = a.x;
                s1col[(size_t)y * RS + 1] = a.y;
                s2col[(size_t)y * RS] = c.x;
                s2col[(size_t)y * RS + 1] = c.y;
            }
#pragma unroll
            for (int d = 0; d + 1 < PF; ++d)
#pragma unroll
                for (int k = 0; k < W; ++k) pf[d][k] = pf[d + 1][k];
#pragma unroll
            for (int k = 0; k < W; ++k) pf[PF - 1][k] = nv[k];
        }
    };
    int r0 = 0;
    for (; r0 + W <= n; r0 += W) block(r0, std::false_type{});
    if (r0 < n) block(r0, std::true_type{});
}

// Phase 1 of the elastic K1, one extra Kronecker term for the column pair
// (x, x+1) and output rows [yb, ye): stream the rows yp = yb-P .. ye+P-1,
// z-contract each with the term's z band (coefficients cz of this plane)
// into a ring of W slots, y-contract every complete window with the term's
// y band (rows read from global memory) and add coef times the result to the
// plane column scol (or write it: init).  Rows and planes outside the grid
// are read clamped and meet zero band entries, as in phase1_chunk.
template <typename T, int P>
__device__ __forceinline__ void phase1_extra(const T *colx, const long long (&zoff)[2 * P + 1], int sx, int my,
                                             const T *bz, const T *by, int yb, int ye, T *scol, int RS, T coef,
                                             bool init)
{
    constexpr int W = 2 * P + 1;
    using V2 = typename Vec2<T>::type;
    T cz[W];
#pragma unroll
    for (int k = 0; k < W; ++k) cz[k] = bz[k];
    V2 r[W];
#pragma unroll
    for (int k = 0; k < W; ++k) r[k] = V2{T(0), T(0)};
    const int n = ye - yb + 2 * P;
    auto load_row = [&](int rr, V2(&dst)[W]) {
        const int yp = min(max(yb - P + rr, 0), my - 1);
        const T *c = colx + (long long)yp * sx;
#pragma unroll
        for (int k = 0; k < W; ++k) dst[k] = *reinterpret_cast<const V2 *>(c + zoff[k]);
    };
    V2 pf[W];
    load_row(0, pf);
    auto block = [&](int r0, auto tail) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int rr = r0 + j;
            if constexpr (decltype(tail)::value) {
                if (rr >= n) break;
            }
            V2 nv[W];
            load_row(rr + 1, nv);
            V2 t = V2{T(0), T(0)};
#pragma unroll
            for (int k = 0; k < W; ++k) t = fma2(cz[k], pf[k], t);
            r[j] = t;
            if (rr >= 2 * P && rr < n) {
                const int y = yb + rr - 2 * P;
                const T *brow = by + (size_t)y * W;
                V2 a = V2{T(0), T(0)};
#pragma unroll
                for (int q = 0; q < W; ++q) a = fma2(brow[q], r[(j - 2 * P + q + 2 * W) % W], a);
                T *d = scol + (size_t)y * RS;
                if (init) {
                    d[0] = coef * a.x;
                    d[1] = coef * a.y;
                } else {
                    d[0] += coef * a.x;
                    d[1] += coef * a.y;
                }
            }
#pragma unroll
            for (int k = 0; k < W; ++k) pf[k] = nv[k];
        }
    };
    int r0 = 0;
    for (; r0 + W <= n; r0 += W) block(r0, std::false_type{});
    if (r0 < n) block(r0, std::true_type{});
}

// Phase 2 of K1, pass 1 for one row segment [b0, b0+n): form
//   R = F - c2 (Kx s1 + Mx s2)
// from the s1, s2 rows with a static register window and run the local
// forward substitution on it.  MODE, the segment kind: kSegMiddle, every row
// inside the Toeplitz range (band rows in registers, no predicates);
// kSegFirst, the first segment (its kHeadRows head rows read from the band
// table); kSegLast / kSegLastAll, the last segment (its kTailRows tail rows,
// or every row, from the table); kSegGeneral, any segment (each row checks
// the Toeplitz range).
enum { kSegMiddle = 0, kSegFirst = 1, kSegLast = 2, kSegGeneral = 3, kSegLastAll = 4 };
constexpr int kHeadRows = 8;   // leading rows of the first segment read from the band table (>= Toeplitz lo)
constexpr int kTailRows = 8;   // trailing rows of the last segment read from the table (>= its rows from Toeplitz hi)

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
        else if (MODE == kSegLast || MODE == kSegLastAll) in_ = xx < mx;   // b0 - P >= 0 here
        else in_ = xx >= 0 && xx < mx;
        a1[j] = in_ ? row1[xx] : T(0);
        a2[j] = in_ ? row2[xx] : T(0);
    }
    const T *fxb = fx ? fx + b0 : nullptr;
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        const int x = b0 + k;
        T bm[W], bk[W];
        const bool table = MODE == kSegLastAll || (MODE == kSegLast && k >= SEG - kTailRows) ||
                           (MODE == kSegFirst && k < kHeadRows);
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
        T acc1 = T(0), acc2 = T(0);   // two independent chains
#pragma unroll
        for (int q = 0; q < W; ++q) {
            acc1 += bk[q] * a1[k + q];
            acc2 += bm[q] * a2[k + q];
        }
        // a general load vector (global row) is read only inside the line; the
        // separable one (shared memory) is padded with zeros
        const bool fin = MODE == kSegMiddle || MODE == kSegFirst || x < mx;
        v[k] = (fxb && fin ? rowF * fxb[k] : T(0)) - c2 * (acc1 + acc2);
    }
    seg_pass1<T, P, SEG>(fb, v);   // rows are independent above; the chain is here
}

// Phase 2 of the elastic K1, pass 1 for one row segment: form
//   R = F - c2 (X1 s1 + X2 s2 [+ X3 s3])
// with a window of 2p+1 positions per plane that slides along the segment
// (the band rows of every position from the table), then the local forward
// substitution.  Rows past the line end meet zero band rows and F = 0.
// TOEP: the whole segment lies in the Toeplitz interior rows, whose band rows
// x1m, x2m, x3m are held in registers (else every row is read from the table).
template <typename T, int P, int SEG, bool HAS3, bool TOEP>
__device__ __forceinline__ void phase2_fwd_el(const T *row1, const T *row2, const T *row3, int mx, int b0,
                                              const T *bX1, const T *bX2, const T *bX3, const T (&x1m)[2 * P + 1],
                                              const T (&x2m)[2 * P + 1], const T (&x3m)[2 * P + 1], const T *fb,
                                              const T *fx, T rowF, T c2, T cx, T (&v)[SEG])
{
    constexpr int W = 2 * P + 1;
    T w1[W], w2[W], w3[W];
    auto ld = [&](const T *row, int xx) { return (xx >= 0 && xx < mx) ? row[xx] : T(0); };
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) {
        const int xx = b0 - P + j;
        w1[j] = ld(row1, xx);
        w2[j] = ld(row2, xx);
        w3[j] = HAS3 ? ld(row3, xx) : T(0);
    }
#pragma unroll
    for (int k = 0; k < SEG; ++k) {
        const int xn = b0 - P + k + 2 * P;   // the position entering the window
        w1[(k + 2 * P) % W] = ld(row1, xn);
        w2[(k + 2 * P) % W] = ld(row2, xn);
        if (HAS3) w3[(k + 2 * P) % W] = ld(row3, xn);
        const int x = b0 + k;
        T acc1 = T(0), acc2 = T(0), acc3 = T(0);   // independent chains
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int sl = (k + q) % W;
            acc1 += (TOEP ? x1m[q] : bX1[x * W + q]) * w1[sl];
            acc2 += (TOEP ? x2m[q] : bX2[x * W + q]) * w2[sl];
            if (HAS3) acc3 += (TOEP ? x3m[q] : bX3[x * W + q]) * w3[sl];
        }
        v[k] = (fx && x < mx ? rowF * fx[x] : T(0)) - c2 * (cx * acc1 + (acc2 + acc3));
    }
    seg_pass1<T, P, SEG>(fb, v);
}

// ---------------------------------------------------------------- K1
//
// One CTA per (z-plane, y-tile of ty rows).  Shared memory: S1, S2 [ty][RS]
// (RS odd), carry buffers and the 1D tables (one bulk copy, waited for
// after phase 1).  Phases:
//  1. z- then y-contraction of p, thread per (column pair, row chunk),
//     streaming along y with a register ring (y bands from global memory):
//        s1 = (My.Mz) p,   s2 = (Ky.Mz + My.Kz) p       (K p = Kx s1 + Mx s2)
//  2. x-direction, thread per (row, segment of SEG): R = F - c2 (Kx s1 + Mx s2)
//     is formed in registers while the local forward pass runs, then the
//     carry exchange and passes 2-3; the row is written back to S1.
//  3. whole plane in the tile: y-direction solve, thread per (x, segment)
//     (FP32: per pair of columns x, x + H and segment, H half the CTA's
//     columns, with packed FP32 instructions), results stored from registers
//     to global memory.
//  4. row tiles only: coalesced store of S1.
// K1 CTA layouts: one CTA per tile, the 2-CTA cluster pair (FP32), or the
// wide FP64 CTA for lines of more than 8 segments (every segment of a line
// needs a warp of its own in the same round).
enum { kLayoutSingle = 0, kLayoutPair = 1, kLayoutWide = 2 };

template <typename T, int LAYOUT>
struct RhsThreads {
    // FP64: more registers per thread; a pair CTA holds half a plane, two per SM
    static constexpr int value =
        LAYOUT == kLayoutWide ? 512 : (sizeof(T) == 8 ? 256 : 512) / (LAYOUT == kLayoutPair ? 2 : 1);
    static constexpr int per_sm = LAYOUT == kLayoutPair ? 2 : 1;
};

// index of the simulation that owns block b: off[i] <= b < off[i+1]
__device__ __forceinline__ int group_find(const int *off, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The body of K1 for block lb of one simulation (arguments a); EL: the
// elastic K1, whose right-hand side also holds el's extra terms (phase 1
// accumulates them into planes 2 and 3, phase 2 contracts plane 3 with Bx).
template <typename T, int P, int SEG, int LAYOUT, bool EL>
__device__ __forceinline__ void rhs_body(const RhsArgs<T> &a, const RhsElas<T> *el, const int lb)
{
    constexpr bool PAIR = LAYOUT == kLayoutPair;
    constexpr int W = 2 * P + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T s_r;
    const int mx = a.d.mx, my = a.d.my, mz = a.d.mz, sx = a.d.sx;
    const long long plane = (long long)sx * my;
    const RhsPlan q = rhs_plan(mx, my, a.ty, PAIR ? 1 : 0, a.lx.S, a.ly.S);
    const int RS = q.RS;   // odd, holds every column pair
    // this CTA's rows [y0, y0 + tye) of plane z; a pair splits the plane at
    // q.ycut (rank 0 below, rank 1 above; cluster ranks are consecutive blocks)
    int y0, z, tye, half = 0;
    if (PAIR) {
        half = lb & 1;
        z = lb >> 1;
        y0 = half ? q.ycut : 0;
        tye = half ? my - q.ycut : q.ycut;
    } else {
        const int ty = a.ty;
        const int nty = (my + ty - 1) / ty;
        y0 = (lb % nty) * ty;
        z = lb / nty;
        tye = min(ty, my - y0);
    }
    const bool fuse_y = q.fuse;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
    const int rows_pad = (tye + 31) & ~31;
    const int cld = q.cld;
    // every segment of a line needs its own warp in one round; the host never
    // launches fewer, but a launch that did would compute wrong lines: report it
    // (all threads of the block, and both CTAs of a pair, take this exit alike)
    if (nwarps < a.lx.S || (fuse_y && nwarps < a.ly.S)) {
        if (tid == 0) atomicExch(a.err, kDevErrConfig);
        return;
    }

    __shared__ __align__(8) uint64_t bar;
    T *S1 = reinterpret_cast<T *>(smem_raw);
    T *S2 = S1 + (size_t)q.rows * RS;
    T *S3 = S2 + (size_t)q.rows * RS;   // elastic K1 with a B plane only
    const int Smax = q.Smax;
    // carry buffers 8-byte aligned (the y sweep of line pairs keeps float2 carries)
    T *CT = reinterpret_cast<T *>(
        (reinterpret_cast<uintptr_t>(S3 + ((EL && el->s3) ? (size_t)q.rows * RS : 0)) + 7) & ~(uintptr_t)7);
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
    const T *bBx = lyb + line_image_elems_dev(P, myp, a.ly.S);   // elastic images end with Bx
    const bool has_src = a.src.fx != nullptr || a.srcfield != nullptr;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (uint32_t)a.img_bytes);
        bulk_load(tb, a.img, (uint32_t)a.img_bytes, &bar);
    }
    if (!a.direct && warp == nwarps - 1) {
        // the y band rows outside the Toeplitz range [lo, hi) are read from
        // global memory by the boundary row chunks of phase 1: bring their
        // cache lines into L1 now, so those reads do not wait on L2/DRAM
        constexpr int LINE = 128 / sizeof(T);
        const int lo = a.bandM[1].lo, hi = a.bandM[1].hi;
        const int h = (lo < hi ? lo : my) * W, t0 = (lo < hi ? hi : my) * W, t1 = my * W;
        const int nh = (h + LINE - 1) / LINE, nt = (t1 - t0 + LINE - 1) / LINE;
        for (int i = lane; i < 2 * (nh + nt); i += 32) {
            const T *band = (i & 1) ? a.bandK[1].v : a.bandM[1].v;
            const int l = i >> 1;
            prefetch_l1(band + (l < nh ? l * LINE : t0 + (l - nh) * LINE));
        }
    }
    __syncthreads();   // barrier initialised
    // everything above reads static tables only; p, the step counter and the
    // output buffer belong to the previous kernels of the stream
    griddep_wait();
    // the wavelet value r(t) (a step-counter load and FP64 arithmetic) is
    // first read in phase 2, after the barrier that ends phase 1: one thread
    // of a middle row chunk (whose phase-1 item has no boundary work)
    // computes it while the others start
    if (tid == NT / 2) {
        T r = T(0);
        if (has_src) {
            double t = (double)(a.step[0] + a.toff) * a.tau;
            r = (T)(a.src.amp * ricker_dev(a.src.freq, a.src.t0, t));
        }
        s_r = r;
    }

    if (a.direct) {
        // ---- phase 1 (direct mode): the RHS is given; stage its rows into S1
        const T *src0 = a.in + (long long)z * plane + (long long)y0 * sx;
        for (int l = warp; l < tye; l += nwarps) {
            const T *src = src0 + (long long)l * sx;
            T *dst = S1 + (size_t)l * RS;
            for (int x = lane; x < mx; x += 32) dst[x] = src[x];
        }
    } else {
        // ---- phase 1 (overlaps the table copy: its y bands are read from global memory)
        const T *gMy = a.bandM[1].v, *gKy = a.bandK[1].v;
        T cm[W], ck[W], mym[W], myk[W];
        const int ylo = a.bandM[1].lo, yhi = a.bandM[1].hi;   // K shares M's interior range
        long long zoff[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            cm[k] = a.bandM[2].v[z * W + k];   // zero for planes outside the grid
            ck[k] = a.bandK[2].v[z * W + k];
            const int mid = ylo < yhi ? ylo : 0;
            mym[k] = gMy[mid * W + k];
            myk[k] = gKy[mid * W + k];
            zoff[k] = (long long)min(max(z + k - P, 0), mz - 1) * plane;
        }
        // work items (column pair, row chunk) spread over all lanes of the
        // CTA: as many chunks as keep every lane busy, whatever mx is
        const int npair = (mx + 1) >> 1;          // column pairs (the last may end in padding)
        int YC = NT / npair;
        if (YC < 1) YC = 1;
        if (YC > tye) YC = tye;
        const int rows_per = (tye + YC - 1) / YC;
        for (int item = tid; item < npair * YC; item += NT) {
            const int pr = item % npair, yc = item / npair;
            const int x = 2 * pr;
            const int yb = y0 + yc * rows_per;
            int ye = yb + rows_per;
            if (ye > y0 + tye) ye = y0 + tye;
            const bool live = yb < ye;
            const bool inter = !live || (yb >= ylo && ye <= yhi);
            // one variant per warp (lanes of two row chunks may share a warp)
            const bool winter = __all_sync(__activemask(), inter);
            if (!live) continue;
            T *c1 = S1 + x - (size_t)y0 * RS, *c2 = S2 + x - (size_t)y0 * RS;
            if constexpr (EL) {
                const bool mass = el->cy == T(0) && el->cz == T(0);   // uniform over the launch
                if (mass && winter)
                    phase1_chunk<T, P, true, true, true>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi,
                                                         yb, ye, c1, c2, RS, el->cy, el->cz);
                else if (mass)
                    phase1_chunk<T, P, false, true, true>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi,
                                                          yb, ye, c1, c2, RS, el->cy, el->cz);
                else if (winter)
                    phase1_chunk<T, P, true, true>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi, yb,
                                                   ye, c1, c2, RS, el->cy, el->cz);
                else
                    phase1_chunk<T, P, false, true>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi, yb,
                                                    ye, c1, c2, RS, el->cy, el->cz);
            } else if (winter)
                phase1_chunk<T, P, true>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi, yb, ye, c1, c2, RS);
            else
                phase1_chunk<T, P, false>(a.in + x, zoff, sx, my, cm, ck, mym, myk, gMy, gKy, ylo, yhi, yb, ye, c1, c2, RS);
            if constexpr (EL) {
                // the extra terms of the same cells, after this thread's own
                // writes of them (no barrier needed)
                for (int t = 0; t < el->n; ++t) {
                    const ExtraTerm<T> &e = el->ex[t];
                    T *sc = (e.slot == 3 ? S3 : S2) + x - (size_t)y0 * RS;
                    phase1_extra<T, P>(e.in + x, zoff, sx, my, e.bz + (size_t)z * W, e.by, yb, ye, sc, RS, e.coef,
                                       e.init != 0);
                }
            }
        }
    }
    // tables in shared memory from here on; every thread leaves together if
    // the copy did not arrive (the error word tells the host); a pair CTA
    // still meets its partner at both cluster barriers first
    if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, a.err))) {
        if (PAIR) {
            cooperative_groups::this_cluster().sync();
            cooperative_groups::this_cluster().sync();
        }
        return;
    }

    // ---- phase 2: x-direction, thread per (row, segment); rounds of row groups
    // line groups (32 rows x S segments, S warps) run their rounds
    // independently: each synchronises on a named barrier of its own (ids
    // 1..15); rows and carry slots of different groups never overlap
    const int RG = rows_pad >> 5;
    const int gpr2 = min(nwarps / LX.S, 15);
    for (int g0 = 0; g0 < RG; g0 += gpr2) {
        const int gi = warp / LX.S, s = warp % LX.S;
        const int g = g0 + gi;
        if (gi >= gpr2 || g >= RG) continue;   // the whole group skips alike
        const int l = g * 32 + lane;
        const bool on = l < tye;
        const int b0 = s * SEG;
        const int n = on ? min(SEG, mx - b0) : 0;
        T v[SEG];
#pragma unroll
        for (int k = 0; k < SEG; ++k) v[k] = T(0);
        if (on && a.direct) {
            const T *row1 = S1 + (size_t)l * RS;
#pragma unroll
            for (int k = 0; k < SEG; ++k) v[k] = (k < n) ? row1[b0 + k] : T(0);
            seg_pass1<T, P, SEG>(LX.fac + b0 * W, v);
        } else if (on) {
            const T *row1 = S1 + (size_t)l * RS;
            const T *row2 = S2 + (size_t)l * RS;
            const int y = y0 + l;
            const T rowF = !has_src ? T(0) : (a.srcfield ? s_r : s_r * sfy[y] * a.src.fz[z]);
            const T c2 = a.c2;
            const int xlo = a.bandM[0].lo, xhi = a.bandM[0].hi;
            T mxm[W], mxk[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int mid = xlo < xhi ? xlo : 0;
                mxm[k] = bMx[mid * W + k];
                mxk[k] = bKx[mid * W + k];
            }
            const T *srcF = !has_src ? nullptr
                                     : (a.srcfield ? a.srcfield + (long long)z * plane + (long long)y * sx : sfx);
            const T *fb = LX.fac + b0 * W;
            // kinds: interior segments take bands from registers; the first reads its
            // head rows (< kHeadRows >= Toeplitz lo) from the table, the last its
            // tail rows (the last kTailRows of the padded line, when they hold
            // every row from Toeplitz hi on, padding included), else every row
            const bool regular = LX.S >= 2 && xlo <= kHeadRows && xhi >= (LX.S - 1) * SEG && mx >= (LX.S - 1) * SEG + P;
            const bool tail = xhi >= LX.S * SEG - kTailRows;
            if constexpr (EL) {
                T x1m[W], x2m[W], x3m[W];
                const int mid = xlo < xhi ? xlo : 0;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    x1m[k] = bKx[mid * W + k];
                    x2m[k] = bMx[mid * W + k];
                    x3m[k] = el->s3 ? bBx[mid * W + k] : T(0);
                }
                const bool toep = b0 >= xlo && b0 + SEG <= xhi;   // uniform over the warp
                const T *r3 = el->s3 ? S3 + (size_t)l * RS : nullptr;
                if (el->s3 && toep)
                    phase2_fwd_el<T, P, SEG, true, true>(row1, row2, r3, mx, b0, bKx, bMx, bBx, x1m, x2m, x3m, fb,
                                                         srcF, rowF, c2, el->cx, v);
                else if (el->s3)
                    phase2_fwd_el<T, P, SEG, true, false>(row1, row2, r3, mx, b0, bKx, bMx, bBx, x1m, x2m, x3m, fb,
                                                          srcF, rowF, c2, el->cx, v);
                else if (toep)
                    phase2_fwd_el<T, P, SEG, false, true>(row1, row2, r3, mx, b0, bKx, bMx, bBx, x1m, x2m, x3m, fb,
                                                          srcF, rowF, c2, el->cx, v);
                else
                    phase2_fwd_el<T, P, SEG, false, false>(row1, row2, r3, mx, b0, bKx, bMx, bBx, x1m, x2m, x3m, fb,
                                                           srcF, rowF, c2, el->cx, v);
            } else if (regular && s > 0 && s < LX.S - 1)
                phase2_fwd<T, P, SEG, kSegMiddle>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else if (regular && s == 0)
                phase2_fwd<T, P, SEG, kSegFirst>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else if (regular && tail)
                phase2_fwd<T, P, SEG, kSegLast>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else if (regular)
                phase2_fwd<T, P, SEG, kSegLastAll>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
            else
                phase2_fwd<T, P, SEG, kSegGeneral>(row1, row2, mx, b0, mxm, mxk, bMx, bKx, xlo, xhi, fb, srcF, rowF, c2, v);
        }
        // the group's reads of its S1/S2 rows are done at seg_finish's first barrier
        seg_finish<T, P, SEG>(LX, on, s, l, cld, CT, CH, v, 1 + gi, 32 * LX.S);
        if (on) {
            T *row1 = S1 + (size_t)l * RS;
#pragma unroll
            for (int k = 0; k < SEG; ++k)
                if (k < n) row1[b0 + k] = v[k];
        }
    }
    __syncthreads();   // phase 3 reads every row

    // ---- phase 3: y-direction (whole plane), thread per (x, segment); rounds of column groups
    if (fuse_y) {
        // a pair sweeps columns [c0, c1) over the rows of both CTAs: rows below
        // q.ycut live in rank 0's S1, the others in rank 1's (read through
        // distributed shared memory once both have finished phase 2)
        int c0 = 0, c1 = mx;
        const T *Slo = S1, *Shi = S1;
        if (PAIR) {
            cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
            cl.sync();
            const T *peer = cl.map_shared_rank(S1, half ^ 1);
            Slo = half ? peer : S1;
            Shi = half ? S1 : peer;
            c0 = half ? q.xcut : 0;
            c1 = half ? mx : q.xcut;
        }
        const int ycut = PAIR ? q.ycut : my;
        // FP32: the y sweep runs on line pairs (one packed instruction for two
        // columns; 8-11 % faster K1 than a line per thread)
        constexpr bool Y2 = sizeof(T) == 4;
        if constexpr (Y2) {
            // line pairs: thread xl holds columns x0 = c0 + xl and x0 + H (H =
            // half the columns, rounded up), both solved by the same packed
            // instructions; slot xl of the carry buffers holds the pair
            const int ncol = c1 - c0, H = (ncol + 1) >> 1;
            const int CG = (H + 31) >> 5;
            const int gpr3 = min(nwarps / LY.S, 15);
            float2 *CT2 = reinterpret_cast<float2 *>(CT), *CH2 = reinterpret_cast<float2 *>(CH);
            for (int g0 = 0; g0 < CG; g0 += gpr3) {
                const int gi = warp / LY.S, s = warp % LY.S;
                if (gi >= gpr3 || g0 + gi >= CG) continue;   // the whole column group skips alike
                const int xl = (g0 + gi) * 32 + lane;
                const bool on = xl < H, on1 = xl + H < ncol;
                const int x0 = c0 + xl;
                const int b0 = s * SEG;
                const int n = on ? min(SEG, my - b0) : 0;
                float2 v[SEG];
#pragma unroll
                for (int k = 0; k < SEG; ++k) {
                    const int r = b0 + k;   // a pair's rows below ycut live in rank 0's S1
                    const T *row =
                        (PAIR ? (r < ycut ? Slo + (size_t)r * RS : Shi + (size_t)(r - ycut) * RS) : S1 + (size_t)r * RS) +
                        x0;
                    v[k] = (k < n) ? make_float2(row[0], on1 ? row[H] : 0.0f) : make_float2(0.0f, 0.0f);
                }
                if (on) seg_pass1<T, P, SEG, float2>(LY.fac + b0 * W, v);
                seg_finish<T, P, SEG, float2>(LY, on, s, xl, cld >> 1, CT2, CH2, v, 1 + gi, 32 * LY.S);
                if (on) {
                    T *dst = a.out + (long long)z * plane + (long long)b0 * sx + x0;
#pragma unroll
                    for (int k = 0; k < SEG; ++k) {
                        if (k < n) {
                            dst[(long long)k * sx] = v[k].x;
                            if (on1) dst[(long long)k * sx + H] = v[k].y;
                        }
                    }
                }
            }
        }
        const int CG = Y2 ? 0 : (c1 - c0 + 31) >> 5;
        const int gpr3 = min(nwarps / LY.S, 15);
        for (int g0 = 0; g0 < CG; g0 += gpr3) {
            const int gi = warp / LY.S, s = warp % LY.S;
            if (gi >= gpr3 || g0 + gi >= CG) continue;   // the whole column group skips alike
            const int xl = (g0 + gi) * 32 + lane;   // column slot within this CTA's range
            const int x = c0 + xl;
            const bool on = x < c1;
            const int b0 = s * SEG;
            const int n = on ? min(SEG, my - b0) : 0;
            T v[SEG];
            if constexpr (PAIR) {
#pragma unroll
                for (int k = 0; k < SEG; ++k) {
                    const int r = b0 + k;
                    v[k] = (k < n) ? (r < ycut ? Slo[(size_t)r * RS + x] : Shi[(size_t)(r - ycut) * RS + x]) : T(0);
                }
            } else {
#pragma unroll
                for (int k = 0; k < SEG; ++k) v[k] = (k < n) ? S1[(size_t)(b0 + k) * RS + x] : T(0);
            }
            if (on) seg_pass1<T, P, SEG>(LY.fac + b0 * W, v);
            seg_finish<T, P, SEG>(LY, on, s, xl, cld, CT, CH, v, 1 + gi, 32 * LY.S);
            // finished columns go straight to global memory (lanes = consecutive
            // x: one coalesced row segment per k); the next round reads other
            // columns of S1 and its carry writes follow seg_finish's barriers
            if (on) {
                T *dst = a.out + (long long)z * plane + (long long)b0 * sx + x;
#pragma unroll
                for (int k = 0; k < SEG; ++k)
                    if (k < n) dst[(long long)k * sx] = v[k];
            }
        }
        // the partner may still be reading this CTA's S1
        if (PAIR) cooperative_groups::this_cluster().sync();
    }

    // ---- phase 4: store (row tiles; the fused path stored in phase 3)
    if (!fuse_y) {
        T *dst0 = a.out + (long long)z * plane + (long long)y0 * sx;
        for (int l = warp; l < tye; l += nwarps) {
            const T *src = S1 + (size_t)l * RS;
            T *dst = dst0 + (long long)l * sx;
            for (int x = lane; x < mx; x += 32) dst[x] = src[x];
        }
    }
}

template <typename T, int P, int NB, int SEG, int LAYOUT>
__global__ void __launch_bounds__(RhsThreads<T, LAYOUT>::value, RhsThreads<T, LAYOUT>::per_sm)
    k_rhs(const __grid_constant__ RhsGroup<T, NB> g)
{
    const int gs = NB > 1 ? group_find(g.off, g.n, blockIdx.x) : 0;
    rhs_body<T, P, SEG, LAYOUT, false>(g.a[gs], nullptr, blockIdx.x - g.off[gs]);   // block within the simulation
}

// the elastic K1 of one simulation
template <typename T, int P, int SEG, int LAYOUT>
__global__ void __launch_bounds__(RhsThreads<T, LAYOUT>::value, RhsThreads<T, LAYOUT>::per_sm)
    k_rhs_el(const __grid_constant__ RhsElGroup<T> g)
{
    rhs_body<T, P, SEG, LAYOUT, true>(g.a, &g.el, blockIdx.x);
}

// ---------------------------------------------------------------- K2/K3
//
// 32 x-columns per CTA (lane = column), one warp per line segment of SEG
// rows held in registers (coalesced direct loads: a warp reads 32
// consecutive values of each row).  Epilogue: plain store, or the Newmark
// update of the (p, q) state, whose p and q tiles [len][32] are fetched by
// TMA at kernel start (overlapping the solve), updated in shared memory and
// written back by TMA stores.
template <typename T, int P, int NB, int SEG>
__global__ void __launch_bounds__(512) k_col(const __grid_constant__ ColGroup<T, NB> g)
{
    const int gs = NB > 1 ? group_find(g.off, g.n, blockIdx.x) : 0;
    const ColArgs<T> &a = g.a[gs];
    const ColMaps &maps = g.maps[gs];
    const int box = g.box[gs];
    const int blk = blockIdx.x - g.off[gs];   // block within this simulation
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const Dims d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, s = tid >> 5;
    const int ntx = (d.mx + 31) >> 5;
    const int x0 = (blk % ntx) * 32, x = x0 + lane;
    const int o = blk / ntx;
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
    // update through TMA-staged p, q tiles, or (tiles too large for shared
    // memory: long FP64 lines) straight from global memory after the solve
    const bool staged = upd && g.tma[gs];
    const int nch = staged ? (len + box - 1) / box : 0;
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
        if (staged) mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar_tab, (uint32_t)a.ln.bytes);
        bulk_load(lb, a.ln.base, (uint32_t)a.ln.bytes, &bar_tab);   // static line tables
    }
    // the input line, p, q and the step counter belong to the previous kernels of the stream
    griddep_wait();
    if (tid == 0) {
        if (upd && blk == 0) a.step[0] += 1;
        if (staged) {
            mbar_expect_tx(&bar, 2u * nch * 32u * box * sizeof(T));
            for (int c = 0; c < nch; ++c) {
                int c0, c1, c2;
                coords(c, c0, c1, c2);
                tma_load_3d(bufP + (size_t)c * box * 32, &maps.P, &bar, c0, c1, c2);
                tma_load_3d(bufQ + (size_t)c * box * 32, &maps.Q, &bar, c0, c1, c2);
            }
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
    if (!__syncthreads_and(mbar_wait_bounded(&bar_tab, 0, a.err))) return;
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
    if (!staged) {
        if (!on) return;
        const T tau2 = a.tau2;
        T *__restrict__ Pp = a.P + off;
        T *__restrict__ Qp = a.Q + off;
#pragma unroll
        for (int k = 0; k < SEG; ++k) {
            if (k < n) {
                const long long o = (long long)k * stride;
                const T q = Qp[o] + tau2 * v[k];
                Qp[o] = q;
                Pp[o] += q;
            }
        }
        if (a.write_a) {
            T *__restrict__ Ap = a.A + off;
#pragma unroll
            for (int k = 0; k < SEG; ++k)
                if (k < n) Ap[(long long)k * stride] = v[k];
        }
        return;
    }
    if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, a.err))) return;   // error recorded for the host
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


// ---------------------------------------------------------------- launchers

template <typename T>
bool rhs_entry_ok(const RhsArgs<T> &a, int seg)
{
    return a.d.mx > 0 && a.d.my > 0 && a.d.mz > 0 && a.ty > 0 && a.ty <= a.d.my && a.lx.S <= 16 &&
           a.ly.S <= 16 && a.lx.seg == seg && a.ly.seg == seg && a.lx.S * seg >= a.d.mx &&
           a.ly.S * seg >= a.d.my && a.img && !(a.img_bytes & 15) && !((uintptr_t)a.img & 15);
}

template <typename T>
int rhs_blocks(const RhsArgs<T> &a)
{
    return a.pair ? 2 * a.d.mz : (a.d.my + a.ty - 1) / a.ty * a.d.mz;
}

// one launch of up to NB simulations, entries a[order[0..n)]
template <typename T, int P, int NB, int SEG, int LAYOUT>
cudaError_t rhs_group_p(const RhsArgs<T> *a, const int *order, int n, cudaStream_t s)
{
    constexpr bool PAIR = LAYOUT == kLayoutPair;
    RhsGroup<T, NB> g;
    std::memset(&g, 0, sizeof(g));
    size_t smem = 0;
    long long blocks = 0;
    for (int k = 0; k < n; ++k) {
        const RhsArgs<T> &e = a[order[k]];
        if (!rhs_entry_ok(e, SEG) || (e.pair != 0) != PAIR) return cudaErrorInvalidValue;
        if (std::max(e.lx.S, (PAIR || e.ty == e.d.my) ? e.ly.S : 0) > RhsThreads<T, LAYOUT>::value / 32)
            return cudaErrorInvalidValue;   // a segment without a warp
        g.a[k] = e;
        g.off[k] = (int)blocks;
        blocks += rhs_blocks(e);
        smem = std::max(smem, rhs_smem_bytes(P, sizeof(T), e.d, e.ty, e.lx.S, e.ly.S, SEG, PAIR ? 1 : 0));
    }
    if (blocks <= 0 || blocks > (1ll << 30)) return cudaErrorInvalidValue;
    g.off[n] = (int)blocks;
    g.n = n;
    static std::atomic<size_t> smem_set{48 * 1024};   // per instantiation: opt-in dynamic shared memory
    if (cudaError_t e = raise_dyn_smem(k_rhs<T, P, NB, SEG, LAYOUT>, smem_set, smem); e != cudaSuccess) return e;
    ++g_launches;
    // programmatic dependent launch: the kernel's prologue overlaps the tail
    // of the previous kernel of the stream (it waits for that kernel before
    // touching its data); pairs: two CTAs per cluster, the halves of one
    // z-plane (every simulation's block range has an even length, so
    // clusters never straddle two)
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(RhsThreads<T, LAYOUT>::value, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    std::memset(attr, 0, sizeof(attr));
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_rhs<T, P, NB, SEG, LAYOUT>, g);
}

// A single simulation is a group of one: one instantiation per (T, P, SEG,
// layout) serves both (its parameters are read with a run-time index, which
// keeps them out of the register budget of the sweeps).  Pairs are FP32
// only and need at most 8 segments per line; FP64 lines of more than 8
// segments take the wide (512-thread) CTA.
template <typename T>
int rhs_layout(const RhsArgs<T> &e)
{
    if (e.pair) return kLayoutPair;
    const bool fuse = e.ty == e.d.my;
    const int smax = std::max(e.lx.S, fuse ? e.ly.S : 0);
    return (sizeof(T) == 8 && smax > RhsThreads<T, kLayoutSingle>::value / 32) ? kLayoutWide : kLayoutSingle;
}

template <typename T, int P, int SEG, int LAYOUT>
cudaError_t rhs_group_chunks(const RhsArgs<T> *a, std::vector<int> &order, cudaStream_t s)
{
    // heaviest blocks first (rows x columns of a tile) so that the tail of
    // the launch holds the short ones
    auto cost = [&](int i) {
        const int rows = a[i].pair ? (a[i].d.my + 1) / 2 : a[i].ty;
        return (long long)rows * a[i].d.mx;
    };
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return cost(i) > cost(j); });
    const int m = (int)order.size();
    for (int k0 = 0; k0 < m; k0 += kBatch) {
        cudaError_t e = rhs_group_p<T, P, kBatch, SEG, LAYOUT>(a, order.data() + k0, std::min(kBatch, m - k0), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// the entries of segment length SEG, one grouped launch series per layout;
// 44-row segments take the single-CTA layout only
template <typename T, int P, int SEG>
cudaError_t rhs_seg_p(const RhsArgs<T> *a, int n, cudaStream_t s)
{
    for (int layout : {kLayoutSingle, kLayoutPair, kLayoutWide}) {
        std::vector<int> order;
        for (int i = 0; i < n; ++i)
            if (a[i].lx.seg == SEG && rhs_layout(a[i]) == layout) order.push_back(i);
        if (order.empty()) continue;
        cudaError_t e = cudaErrorInvalidValue;
        if (layout == kLayoutSingle) {
            e = rhs_group_chunks<T, P, SEG, kLayoutSingle>(a, order, s);
        } else if constexpr (SEG != kSegLong) {
            if constexpr (sizeof(T) == 4) {
                if (layout == kLayoutPair) e = rhs_group_chunks<T, P, SEG, kLayoutPair>(a, order, s);
            } else {
                if (layout == kLayoutWide) e = rhs_group_chunks<T, P, SEG, kLayoutWide>(a, order, s);
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// one elastic K1 launch: single-CTA layout (wide for FP64 lines of more than
// 8 segments); never a cluster pair (measured slower at 96^3), never direct mode
template <typename T, int P, int SEG, int LAYOUT>
cudaError_t rhs_el_p(const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s)
{
    constexpr bool PAIR = LAYOUT == kLayoutPair;
    if (!rhs_entry_ok(a, SEG) || (a.pair != 0) != PAIR || a.direct || el.n < 0 || el.n > kMaxExtra)
        return cudaErrorInvalidValue;
    if (std::max(a.lx.S, (PAIR || a.ty == a.d.my) ? a.ly.S : 0) > RhsThreads<T, LAYOUT>::value / 32)
        return cudaErrorInvalidValue;   // a segment without a warp
    for (int t = 0; t < el.n; ++t)
        if (!el.ex[t].in || !el.ex[t].by || !el.ex[t].bz || (el.ex[t].slot != 2 && el.ex[t].slot != 3) ||
            (el.ex[t].slot == 3 && !el.s3))
            return cudaErrorInvalidValue;
    RhsElGroup<T> g;
    std::memset(&g, 0, sizeof(g));
    g.a = a;
    g.el = el;
    // planes, carry buffers and the table image as the kernel carves them
    const RhsPlan q = rhs_plan(a.d.mx, a.d.my, a.ty, PAIR ? 1 : 0, a.lx.S, a.ly.S);
    const size_t n = (size_t)(el.s3 ? 3 : 2) * q.rows * q.RS + 2 * (size_t)q.Smax * P * q.cld;
    const size_t smem = n * sizeof(T) + 32 + (((size_t)a.img_bytes + 15) & ~(size_t)15);
    static std::atomic<size_t> smem_set{48 * 1024};
    if (cudaError_t e = raise_dyn_smem(k_rhs_el<T, P, SEG, LAYOUT>, smem_set, smem); e != cudaSuccess) return e;
    ++g_launches;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)rhs_blocks(a), 1, 1);
    cfg.blockDim = dim3(RhsThreads<T, LAYOUT>::value, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    std::memset(attr, 0, sizeof(attr));
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;   // pairs: the two halves of one z-plane
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_rhs_el<T, P, SEG, LAYOUT>, g);
}

template <typename T, int P, int SEG>
cudaError_t rhs_el_layout(const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s)
{
    const int layout = rhs_layout(a);
    if (layout == kLayoutSingle) return rhs_el_p<T, P, SEG, kLayoutSingle>(a, el, s);
    if constexpr (SEG != kSegLong) {
        if constexpr (sizeof(T) == 8) {
            if (layout == kLayoutWide) return rhs_el_p<T, P, SEG, kLayoutWide>(a, el, s);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
bool col_entry_ok(const ColArgs<T> &a, int seg)
{
    const int len = a.axis == 1 ? a.d.my : a.d.mz;
    return (a.axis == 1 || a.axis == 2) && a.d.mx > 0 && len > 0 && a.ln.seg == seg && a.ln.S * seg >= len &&
           a.ln.S <= 16 &&
           a.ln.base && !(a.ln.bytes & 15) && !((uintptr_t)a.ln.base & 15) && (a.mode == 0 || a.mode == 1);
}

template <typename T, int P, int NB, int SEG>
cudaError_t col_group_p(const ColArgs<T> *a, const ColMaps *maps, const int *order, int n, cudaStream_t s)
{
    ColGroup<T, NB> g;
    std::memset(&g, 0, sizeof(g));
    size_t smem = 0;
    long long blocks = 0;
    int smax = 1;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const ColArgs<T> &e = a[i];
        if (!col_entry_ok(e, SEG)) return cudaErrorInvalidValue;
        const int len = e.axis == 1 ? e.d.my : e.d.mz;
        const int outer = e.axis == 1 ? e.d.mz : e.d.my;
        const int box = col_box(len);
        size_t tiles = 0;
        g.tma[k] = 0;
        if (e.mode == 1) {
            tiles = 2 * (size_t)((len + box - 1) / box) * box * 32 * sizeof(T);
            if (128 + tiles + col_smem_bytes(P, sizeof(T), len, e.ln.S, SEG) <= 200 * 1024) {
                if (maps) g.maps[k] = maps[i];
                else if (!make_update_maps(&g.maps[k], e.P, e.Q, sizeof(T), e.d, e.axis)) return cudaErrorInvalidValue;
                g.tma[k] = 1;
            } else {
                tiles = 0;   // update from global memory
            }
        }
        g.a[k] = e;
        g.box[k] = box;
        g.off[k] = (int)blocks;
        blocks += (long long)((e.d.mx + 31) / 32) * outer;
        smem = std::max(smem, 128 + tiles + col_smem_bytes(P, sizeof(T), len, e.ln.S, SEG));
        smax = std::max(smax, e.ln.S);
    }
    if (blocks <= 0 || blocks > (1ll << 30)) return cudaErrorInvalidValue;
    g.off[n] = (int)blocks;
    g.n = n;
    static std::atomic<size_t> smem_set{48 * 1024};
    if (cudaError_t e = raise_dyn_smem(k_col<T, P, NB, SEG>, smem_set, smem); e != cudaSuccess) return e;
    // programmatic dependent launch (the kernel waits for the previous one before reading its data)
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(32 * smax, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    std::memset(attr, 0, sizeof(attr));
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++g_launches;
    return cudaLaunchKernelEx(&cfg, k_col<T, P, NB, SEG>, g);
}

template <typename T, int P>
cudaError_t col_group_dispatch(const ColArgs<T> *a, const ColMaps *maps, int n, cudaStream_t s)
{
    auto len = [&](int i) { return a[i].axis == 1 ? a[i].d.my : a[i].d.mz; };
    for (int i = 0; i < n; ++i)
        if (!seg_supported(a[i].ln.seg)) return cudaErrorInvalidValue;
    for (int seg : {kSeg, kSegAlt, kSegLong}) {
        std::vector<int> order;
        for (int i = 0; i < n; ++i)
            if (a[i].ln.seg == seg) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return len(i) > len(j); });
        const int m = (int)order.size();
        for (int k0 = 0; k0 < m; k0 += kBatch) {
            const int nk = std::min(kBatch, m - k0);
            cudaError_t e = seg == kSeg      ? col_group_p<T, P, kBatch, kSeg>(a, maps, order.data() + k0, nk, s)
                            : seg == kSegAlt ? col_group_p<T, P, kBatch, kSegAlt>(a, maps, order.data() + k0, nk, s)
                                             : col_group_p<T, P, kBatch, kSegLong>(a, maps, order.data() + k0, nk, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

#define ADS_DISPATCH_P(p, CALL)                      \
    switch (p) {                                     \
    case 1: return CALL(1);                          \
    case 2: return CALL(2);                          \
    case 3: return CALL(3);                          \
    case 4: return CALL(4);                          \
    default: return cudaErrorInvalidValue;           \
    }

}  // namespace

template <typename T, int SEG>
cudaError_t launch_rhs_seg(int p, const RhsArgs<T> *a, int n, cudaStream_t s)
{
    if (!a || n <= 0) return cudaErrorInvalidValue;
#define C(P) rhs_seg_p<T, P, SEG>(a, n, s)
    ADS_DISPATCH_P(p, C)
#undef C
}

template <typename T>
cudaError_t launch_col_group(int p, const ColArgs<T> *a, const ColMaps *maps, int n, cudaStream_t s)
{
    if (!a || n <= 0) return cudaErrorInvalidValue;
#define C(P) col_group_dispatch<T, P>(a, maps, n, s)
    ADS_DISPATCH_P(p, C)
#undef C
}

// the elastic K1 of segment length SEG (one translation unit per precision and length)
template <typename T, int SEG>
cudaError_t launch_rhs_el_seg(int p, const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s)
{
    if (a.lx.seg != SEG || a.ly.seg != SEG) return cudaErrorInvalidValue;
#define C(P) rhs_el_layout<T, P, SEG>(a, el, s)
    ADS_DISPATCH_P(p, C)
#undef C
}

}  // namespace ads
