// kernels.cuh -- launch interface of the device kernels (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

namespace ads {

// device error codes written to a simulation's error word by bounded waits
enum { kDevErrTimeout = 1, kDevErrAlign = 2, kDevErrConfig = 3 };

constexpr int kSeg = 32;      // rows per register segment of the line solves ...
constexpr int kSegAlt = 33;   // ... or 33, when that saves segments (m = 32 s + 1 -> s segments) ...
constexpr int kSegLong = 44;  // ... or 44, when 3 segments let every line group of a plane run at once (m <= 132)
inline bool seg_supported(int seg) { return seg == kSeg || seg == kSegAlt || seg == kSegLong; }
constexpr int kBatch = 32;   // simulations per grouped launch

// Interior field layout on the device: [z][y][x], x fastest, row pitch sx
// elements (sx >= mx, padding kept at zero), plane pitch sx*my.
struct Dims {
    int mx, my, mz, sx;
    int off;   // boundary functions dropped per side: 1 Dirichlet, 0 natural (full = unknowns)
    int offz;  // the same along z (0 for a 2D problem: one constant function along z)
    __host__ __device__ long long plane() const { return (long long)sx * my; }
    __host__ __device__ long long count() const { return plane() * mz; }
};

// Device tables of one directional factor set for the partitioned line
// solve (layouts in setup1d.h): factor rows [m][2p+1], fundamental
// solutions [m][p], transfer matrices [S][p][p], segment bounds [S+1].
// One contiguous buffer, in this order (T elements, no gaps):
//   fac [m_pad][2p+1] | phi [m_pad][p] | psi [m_pad][p] | Phi [S][p][p] | Psi [S][p][p]
// with m_pad = S * seg; segment s = rows [s*seg, (s+1)*seg).  It is copied
// to shared memory verbatim (one bulk copy) by the sweep kernels.
template <typename T>
struct LineDev {
    const T *base;
    int S;
    int bytes;            // padded to 16
    int seg;              // rows per segment (kSeg, kSegAlt or kSegLong)
};

// Operator band of one axis with its Toeplitz interior rows [lo, hi).
template <typename T>
struct BandDev {
    const T *v;           // [m][2p+1]
    int lo, hi;
};

// Source term of the scalar wave: F(t) = r(t) fx(x) fy(y) fz(z) (separable
// Gaussian times a Ricker wavelet).  fx == nullptr means no source.
template <typename T>
struct SrcDev {
    const T *fx, *fy, *fz;
    double amp, freq, t0;
};

// Fused RHS + directional sweeps (kernel K1), one z-plane tile per CTA:
//   out = Ax^{-1} [ F(t) - c2 (Kx.My.Mz + Mx.My.Kz + Mx.Ky.Mz) in ]   (along x)
// and, when the tile spans all of y (ty == my), also Ay^{-1} along y.
// Direct mode: out = Ax^{-1} [Ay^{-1}] in (the RHS is given).
// t = (step[0] + toff) * tau.
template <typename T>
struct RhsArgs {
    const T *in;
    T *out;
    Dims d;
    BandDev<T> bandM[3], bandK[3];
    LineDev<T> lx, ly;
    // shared-memory image of all 1D tables of this launch (see rhs_image_layout):
    //   bMx bKx [mxp][W] | bMy bKy [myp][W] | fx [mxp] | fy [myp] | lx tables | ly tables
    const T *img;
    int img_bytes;
    T c2;
    SrcDev<T> src;
    const long long *step;
    int toff;
    double tau;
    int ty;               // rows per tile (y); fused y sweep iff ty == my
    int *err;             // device error word (bounded waits)
    const T *srcfield;    // non-null: F(t) = r(t) srcfield (general load vector, interior layout)
    int direct;           // 1: `in` is the RHS itself (no quadrature): out = Ax^{-1} [Ay^{-1}] in
    int pair;             // 1 (FP32): a 2-CTA cluster per z-plane (fused y sweep across the pair)
};

// Extra Kronecker terms of the elastic right-hand side (the off-diagonal
// blocks of Sec. 5): coef (Ay (x) Az) in, contracted along z and y in K1's
// phase 1 and accumulated into plane `slot` (2: contracted along x with the
// image's second x band, M; 3: with the third, B), so that K1 forms
//   R = F - c2 (X1 s1 + Mx s2 + Bx s3)
// with s1, s2 from the stream of `in` (the diagonal block) and the extra
// terms inside s2, s3.
template <typename T>
struct ExtraTerm {
    const T *in;
    const T *by, *bz;   // bands [m_pad][2p+1] along y and z
    T coef;
    int slot;           // 2 or 3
    int init;           // 1: the first term of plane 3 writes it
};
constexpr int kMaxExtra = 4;
template <typename T>
struct RhsElas {
    ExtraTerm<T> ex[kMaxExtra];
    int n;
    int s3;             // 1: plane 3 exists (some term has slot 3); the image then ends with Bx [mxp][2p+1]
    // coefficients of the stream of `in`, applied after each contraction so
    // that the bands keep their exact row sums:
    //   s2 = cy (Ky Mz in) + cz (My Kz in),  R = F - c2 (cx X1 s1 + Mx s2 + Bx s3)
    T cx, cy, cz;
};
// one elastic K1 launch (a single simulation)
template <typename T>
struct RhsElGroup {
    RhsArgs<T> a;
    RhsElas<T> el;
};

// Column sweep along y (axis 1) or z (axis 2): 32 x-columns per CTA, one
// warp per line segment.
//   mode 0: out = A^{-1} in along the axis (in == out allowed)
//   mode 1 (Newmark epilogue, scalar wave state p,q,a):
//        a = A^{-1} in;  q += tau^2 a;  p += q;  a_out = a (if write_a)
//        and step[0] += 1 (one thread)
template <typename T>
struct ColArgs {
    const T *in;
    T *out;
    Dims d;
    int axis;
    LineDev<T> ln;
    int mode;
    T *P, *Q, *A;
    T tau2;
    int write_a;
    long long *step;
    int *err;             // device error word (bounded waits)
};

// TMA maps of the (p, q) state arrays for the K3 epilogue: 3D maps over
// [z][y][x] with a box of 32 columns x col_box(len) rows along the axis.
struct ColMaps {
    CUtensorMap P, Q;
};

// rows per TMA box along a line of length len (at most 256, equal chunks)
inline int col_box(int len)
{
    const int nch = (len + 255) / 256;
    return (len + nch - 1) / nch;
}
bool make_update_maps(ColMaps *m, const void *P, const void *Q, int elem, const Dims &d, int axis);

// Kernel parameter blocks of a grouped launch: NB simulations, block b of
// the flat grid belongs to simulation i with off[i] <= b < off[i+1].
template <typename T, int NB>
struct RhsGroup {
    RhsArgs<T> a[NB];
    int off[NB + 1];
    int n;
};

template <typename T, int NB>
struct ColGroup {
    ColMaps maps[NB];
    ColArgs<T> a[NB];
    int box[NB];
    int tma[NB];          // mode 1: p, q tiles staged by TMA (else updated in global memory)
    int off[NB + 1];
    int n;
};

// seg: register segment width of the partitioned solves (32); planes: the
// s-planes of the tile (2, or 3 for the elastic K1 with a B plane, whose
// image also holds Bx)
size_t rhs_smem_bytes(int p, int elem, const Dims &d, int ty, int Sx, int Sy, int seg, int pair = 0, int planes = 2);
int rhs_threads(int elem);
// element offsets of the K1 table image: returns total elements
size_t rhs_image_elems(int p, const Dims &d, int Sx, int Sy, int seg);
size_t line_image_elems(int p, int S, int seg);
size_t col_smem_bytes(int p, int elem, int len, int S, int seg);
// segment length for a space with interior sizes m[3] and elements of
// elem bytes: kSegAlt when it needs fewer segments in all than kSeg;
// kSegLong when it needs fewer rounds of line groups in K1 (measured in
// rows of dependent recurrence: rounds x segment length)
int choose_seg(const int *m, int elem);

template <typename T>
cudaError_t launch_rhs(int p, int seg, const RhsArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_col(int p, int seg, const ColArgs<T> &a, cudaStream_t s);
// Grouped launches: n independent simulations of degree p (any grids) in
// ceil(n / kBatch) launches; maps (nullable) holds precomputed update maps
// per entry (mode 1), else they are encoded here.
template <typename T>
cudaError_t launch_rhs_group(int p, const RhsArgs<T> *a, int n, cudaStream_t s);
// the entries of a[0..n) whose segment length is SEG (one translation unit each)
template <typename T, int SEG>
cudaError_t launch_rhs_seg(int p, const RhsArgs<T> *a, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_col_group(int p, const ColArgs<T> *a, const ColMaps *maps, int n, cudaStream_t s);
// Elastic K1 (one simulation): the diagonal block's right-hand side by sum
// factorisation plus el's extra terms, then the x [and y] sweeps
template <typename T>
cudaError_t launch_rhs_el(int p, const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s);
// the same for segment length SEG (one translation unit each)
template <typename T, int SEG>
cudaError_t launch_rhs_el_seg(int p, const RhsArgs<T> &a, const RhsElas<T> &el, cudaStream_t s);

// Sum of Kronecker products in one pass:
//   out = beta*out + sum_t alpha_t (Ax_t (x) Ay_t (x) Az_t) in_t
// (plain terms: alpha_t in_t, no contraction); row padding written as zero.
constexpr int kMaxKronTerms = 8;
template <typename T>
struct KronTerm {
    const T *bx, *by, *bz;   // bands [m_pad][2p+1] per axis
    const T *in;
    T alpha;
    int plain;
};
template <typename T>
struct KronSum {
    KronTerm<T> t[kMaxKronTerms];
    int nt;
    T beta;
};
template <typename T>
cudaError_t launch_kron_sum(int p, const KronSum<T> &ks, T *out, Dims d, cudaStream_t s);
// out = band applied along axis (0,1,2) to in; out = beta*out + alpha*(A in)
template <typename T>
cudaError_t launch_axis_apply(int p, const T *band, int axis, const T *in, T *out, Dims d, T alpha, T beta,
                              int transpose, cudaStream_t s);
// in-place line solve along x with a factor table [m][2p+1] (thread per line)
template <typename T>
cudaError_t launch_solve_x(int p, const T *fac, T *data, Dims d, cudaStream_t s);

// full FP64 [nz][ny][nx] <-> interior T
template <typename T>
cudaError_t launch_pack(const double *full, T *in, Dims d, double scale, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack(const T *in, double *full, Dims d, cudaStream_t s);
// convert between (u, v, a) FP64 interior and (p, q, a) T:
//   p = u + tau v + tau^2/4 a,  q = tau v + tau^2/2 a
template <typename T>
cudaError_t launch_uva_to_pq(const double *u, const double *v, const double *a, T *P, T *Q, T *A, Dims d,
                             double tau, cudaStream_t s);
//   u = p - q + tau^2/4 a,  v = (q - tau^2/2 a) / tau
template <typename T>
cudaError_t launch_pq_to_uva(const T *P, const T *Q, const T *A, double *u, double *v, double *a, Dims d,
                             double tau, cudaStream_t s);
// out = amp * gz[z] gy[y] gx[x]
cudaError_t launch_outer(const double *gx, const double *gy, const double *gz, double amp, double *out, Dims d,
                         cudaStream_t s);
// y = a*x + b*y (FP64, interior incl. padding)
cudaError_t launch_axpby(double a, const double *x, double b, double *y, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_convert(const T *x, double *y, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_convert_from(const double *x, T *y, long long n, cudaStream_t s);
// partial[block] = compensated sum of x*y; then a 1-block pass -> result[0]
cudaError_t launch_dot(const double *x, const double *y, long long n, double *partial, int nblocks,
                       double *result, cudaStream_t s);

// out = a*x + b*y over n elements (y may be null)
template <typename T>
cudaError_t launch_lincomb(T *out, T a, const T *x, T b, const T *y, long long n, cudaStream_t s);
// Newmark update of the (p, q) state from a solved acceleration x:
//   q += tau2 x;  p += q;  a = x (if write_a);  step[0] += 1
template <typename T>
cudaError_t launch_pq_update(T *P, T *Q, T *A, const T *x, long long n, T tau2, int write_a, long long *step,
                             cudaStream_t s);
// y += (double) x  over n elements
template <typename T>
cudaError_t launch_add_converted(const T *x, double *y, long long n, cudaStream_t s);
// three-level update (elasticity): t = U; U = 2U - Up + d; Up = t; step[0] += 1
template <typename T>
cudaError_t launch_atm_update(T *U, T *Up, const T *d, long long n, long long *step, cudaStream_t s);
// out[z][y][x] += scale * ricker(t) * fz[z] fy[y] fx[x],  t = (step[0] + toff) * tau
template <typename T>
cudaError_t launch_add_source(T *out, Dims d, const T *fx, const T *fy, const T *fz, double scale, double freq,
                              double t0, const long long *step, int toff, double tau, cudaStream_t s);
// out += scale * ricker(t) * field,  t = (step[0] + toff) * tau  (general load vector)
template <typename T>
cudaError_t launch_add_field(T *out, const T *field, long long n, double scale, double freq, double t0,
                             const long long *step, int toff, double tau, cudaStream_t s);
// FP64 views of the elastic state: u = U, v = (U - Up)/tau
template <typename T>
cudaError_t launch_el_to_uv(const T *U, const T *Up, double *u, double *v, long long n, double tau, cudaStream_t s);

// one thread sleeps for `ns` nanoseconds of the global timer (keeps the
// stream busy while the host queues the launches that follow)
cudaError_t launch_delay(unsigned long long ns, cudaStream_t s);
// bounded-wait self-test: err[0] = timeout code if the wait ran out, err[1] = 1 if it completed
cudaError_t launch_wait_selftest(long long cycles, int *err, cudaStream_t s);

// kernel launches issued by the library (all host threads)
extern std::atomic<unsigned long long> g_launches;

// Opt-in dynamic shared memory of one kernel, raised to at least `smem`
// bytes.  `cur` (one per kernel instantiation) only grows, under one lock,
// and only after the attribute holds it, so host threads that launch the
// same kernel with different sizes never lower it under one another.
std::mutex &attr_mutex();
template <typename K>
cudaError_t raise_dyn_smem(K *kernel, std::atomic<size_t> &cur, size_t smem)
{
    if (smem <= cur.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(attr_mutex());
    if (smem <= cur.load(std::memory_order_relaxed)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur.store(smem, std::memory_order_release);
    return e;
}

}  // namespace ads
