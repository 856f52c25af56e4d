// api.cpp -- the C ABI of include/ads.h: simulation objects, device tables,
// the per-step launch sequence (captured into CUDA graphs), boundary
// conversions, operators, energies and checkpoints.
#include "ads.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "setup1d.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define ADS_CK(expr)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError(); /* a failed launch or attribute call leaves no pending error */    \
            return fail(ADS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));        \
        }                                                                                         \
    } while (0)

}  // namespace

// Device tables of one directional factor set (banded LU factors plus the
// segment tables of the partitioned solve) in one contiguous buffer laid out
// as the kernels' shared-memory image (see LineDev), precision T.
struct LineTables {
    void *base = nullptr;
    int S = 0;
    int bytes = 0;
    int seg = 32;
};

enum { SET_SPLIT = 0, SET_MASS = 1, SET_IDENT = 2, SET_ELAS0 = 3, SET_ELAS1 = 4, NSETS = 5 };
// K1 table images: one per factor set (x and y tables of that set), plus the
// three mixed images of the elastic diagonal blocks (component i: set ELAS0
// on axis i, ELAS1 on the others)
enum { IMG_EL = NSETS, NIMG = NSETS + 3 };

// Device copy of a set of FP64 host tables in precision T.
struct TableSet {
    void *M[3] = {}, *K[3] = {}, *B[3] = {};   // operator bands [m_pad][2p+1]
    void *Bt[3] = {};                          // B^T bands (natural boundary)
    LineTables line[NSETS][3];                 // per factor set and axis
    void *img[NIMG] = {};                      // K1 images (x and y tables of a set)
    int img_bytes[NIMG] = {};
    void *gband[3] = {};                       // bands of M + eta c2 K (energies)
    void *src[3] = {};                         // separable source load vectors
    void *srcfield = nullptr;                  // general source load vector (interior layout)
    // fused elastic step (Dirichlet): the elastic K1 images [lower/upper][i]
    void *elimg[2][3] = {};
    int elimg_bytes[2][3] = {};
};

struct ads_sim {
    int kind = ADS_SCALAR_WAVE, prec = ADS_FP64, p = 2, device = 0;
    ads::Axis1D ax[3];
    double tau = 0, c2 = 1, lam = 1, mu = 1, rho = 1;
    ads::Dims d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ads_alloc_fn alloc = nullptr;
    ads_free_fn dfree = nullptr;
    void *actx = nullptr;
    std::map<void *, size_t> live;
    size_t bytes = 0;
    TableSet t64, t32;
    // host FP64 copies used to assemble the kernels' table images
    std::vector<double> hM[3], hK[3], hsrc[3];
    std::vector<double> hline[NSETS][3];
    int lineS[3] = {0, 0, 0};
    // scalar-wave state (precision prec): p = u + tau v + eta a, q = tau v + tau^2/2 a
    void *P = nullptr, *Q = nullptr, *A = nullptr, *X = nullptr;
    // elasticity state: U^n, U^{n-1} (3 components, component-major) and work
    void *U = nullptr, *Up = nullptr, *R = nullptr, *Y = nullptr;
    void *ebandFP64[3][2] = {};   // bands of M + d K (d = tau^2 c / (4 rho)), FP64, for the invariant
    long long *d_step = nullptr;
    long long h_step = 0;
    int *d_err = nullptr;   // device error word written by bounded waits
    bool has_src = false;
    ads_source_t src{};
    // kernel tiling of K1 per precision
    int ty[2] = {0, 0}, tz[2] = {0, 0}, fuse[2] = {0, 0};
    int pair[2] = {0, 0};   // FP32: K1 as a 2-CTA cluster per z-plane
    int ty_el[2] = {0, 0};  // rows per tile of the elastic K1 (three planes), per precision
    bool fused_el = false;  // elasticity: the fused alternating-triangular step
    int seg = 32;           // register segment width of the line solves
    // graphs: chunk size -> executable graph, and the kernels it launches
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, unsigned long long> graph_launches;
    bool warmed = false;
    // identity for cached batch graphs: uid is unique per process, version
    // changes whenever the launch arguments change (tables, tiles)
    unsigned long long uid = 0, version = 0;
    ads::ColMaps upd_maps{};   // TMA maps of P, Q for the z epilogue (scalar wave)
    bool has_maps = false;
    // FP64 residual correction of the FP32 scalar-wave step (option)
    bool refine = false;
    void *R64 = nullptr, *P64 = nullptr, *A64 = nullptr, *T64 = nullptr;
};

namespace {

size_t elem(const ads_sim *s) { return s->prec == ADS_FP64 ? 8 : 4; }

void *dalloc(ads_sim *s, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (s->alloc) {
        p = s->alloc(bytes, s->actx);
    } else {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) {
        s->live[p] = bytes;
        s->bytes += bytes;
    }
    return p;
}

void dfree(ads_sim *s, void *p)
{
    if (!p) return;
    auto it = s->live.find(p);
    if (it != s->live.end()) {
        s->bytes -= it->second;
        s->live.erase(it);
    }
    if (s->dfree) s->dfree(p, s->actx);
    else cudaFree(p);
}

// RAII scratch for one API call
struct Scratch {
    ads_sim *s;
    std::vector<void *> ptrs;
    explicit Scratch(ads_sim *s_) : s(s_) {}
    void *get(size_t bytes)
    {
        void *p = dalloc(s, bytes);
        if (p) ptrs.push_back(p);
        return p;
    }
    ~Scratch()
    {
        if (!ptrs.empty()) cudaStreamSynchronize(s->stream);
        for (void *p : ptrs) dfree(s, p);
    }
};

template <typename T>
int upload(ads_sim *s, const std::vector<double> &h, void **dst)
{
    std::vector<T> tmp(h.begin(), h.end());
    void *p = dalloc(s, tmp.size() * sizeof(T));
    if (!p) return fail(ADS_ERR_OOM, "device allocation failed (tables)");
    ADS_CK(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = p;
    return ADS_OK;
}

ads::Factor identity_factor(int m, int p)
{
    ads::Factor f;
    f.m = m;
    f.p = p;
    f.v.assign((size_t)m * (2 * p + 1), 0.0);
    for (int i = 0; i < m; ++i) f.v[(size_t)i * (2 * p + 1) + p] = 1.0;
    return f;
}

// Rows padded to a whole number of segments: m_pad = S * seg.
int padded(const ads_sim *s, int m) { return (m + s->seg - 1) / s->seg * s->seg; }

// band rows [m][2p+1] -> [m_pad][2p+1], zero rows appended
std::vector<double> pad_rows(const std::vector<double> &v, int m, int width, int m_pad, bool identity_factor)
{
    std::vector<double> out((size_t)m_pad * width, 0.0);
    std::copy(v.begin(), v.begin() + (size_t)m * width, out.begin());
    if (identity_factor)
        for (int i = m; i < m_pad; ++i) out[(size_t)i * width + width / 2] = 1.0;   // 1/u_0 = 1
    return out;
}

// host image of one factor set: fac | phi | psi | Phi | Psi (padded rows)
std::vector<double> line_image(const ads_sim *s, const ads::Factor &f, int *S)
{
    ads::Partition P = ads::partition_fixed(f, s->seg);
    const int mp = padded(s, f.m), W = 2 * f.p + 1;
    std::vector<double> img = pad_rows(f.v, f.m, W, mp, true);
    auto add = [&](const std::vector<double> &v) { img.insert(img.end(), v.begin(), v.end()); };
    add(pad_rows(P.phi, f.m, f.p, mp, false));
    add(pad_rows(P.psi, f.m, f.p, mp, false));
    add(P.Phi);
    add(P.Psi);
    *S = P.S;
    return img;
}

template <typename T>
int upload_padded(ads_sim *s, const std::vector<double> &h, void **dst, int *bytes)
{
    std::vector<T> tmp(h.begin(), h.end());
    while ((tmp.size() * sizeof(T)) % 16) tmp.push_back(T(0));
    void *p = dalloc(s, tmp.size() * sizeof(T));
    if (!p) return fail(ADS_ERR_OOM, "device allocation failed (tables)");
    ADS_CK(cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = p;
    if (bytes) *bytes = (int)(tmp.size() * sizeof(T));
    return ADS_OK;
}

// K1 image in slot `slot`: bMx bKx | bMy bKy | fx | fy | x tables of xset | y tables of yset
template <typename T>
int upload_rhs_image(ads_sim *s, TableSet &ts, int slot, int xset, int yset)
{
    if (s->hline[xset][0].empty() || s->hline[yset][1].empty()) return ADS_OK;
    std::vector<double> img;
    auto add = [&](const std::vector<double> &v) { img.insert(img.end(), v.begin(), v.end()); };
    add(s->hM[0]);
    add(s->hK[0]);
    add(s->hM[1]);
    add(s->hK[1]);
    for (int a = 0; a < 2; ++a) {
        const size_t mp = (size_t)padded(s, s->ax[a].m);
        if (s->hsrc[a].size() == mp) add(s->hsrc[a]);
        else img.insert(img.end(), mp, 0.0);
    }
    add(s->hline[xset][0]);
    add(s->hline[yset][1]);
    if (ts.img[slot]) {
        dfree(s, ts.img[slot]);
        ts.img[slot] = nullptr;
    }
    return upload_padded<T>(s, img, &ts.img[slot], &ts.img_bytes[slot]);
}

// c_{i,a} of the diagonal block Ups_ii = sum_a c_ia [K on axis a, M elsewhere]
double el_coef(const ads_sim *s, int i, int a) { return s->mu + (a == i ? s->lam + s->mu : 0.0); }

// Elastic K1 image of component i, kind 0 (lower sweep) or 1 (upper):
//   bMx | X1 | bMy | bKy | fx | fy | x tables | y tables | Bx
// X1 = Kx (lower: the diagonal block of Ups U; the kernel scales the
// contraction by -tau^2/rho c_i0) or Mx (upper: rho M y / rho); factor sets
// ELAS0 on axis i, ELAS1 elsewhere.
template <typename T>
int upload_el_image(ads_sim *s, TableSet &ts, int kind, int i)
{
    const int xset = i == 0 ? SET_ELAS0 : SET_ELAS1, yset = i == 1 ? SET_ELAS0 : SET_ELAS1;
    if (s->hline[xset][0].empty() || s->hline[yset][1].empty()) return ADS_OK;
    std::vector<double> img;
    auto add = [&](const std::vector<double> &v) { img.insert(img.end(), v.begin(), v.end()); };
    add(s->hM[0]);
    add(kind == 0 ? s->hK[0] : s->hM[0]);
    add(s->hM[1]);
    add(s->hK[1]);
    for (int a = 0; a < 2; ++a) {
        const size_t mp = (size_t)padded(s, s->ax[a].m);
        if (s->hsrc[a].size() == mp) add(s->hsrc[a]);
        else img.insert(img.end(), mp, 0.0);
    }
    add(s->hline[xset][0]);
    add(s->hline[yset][1]);
    const ads::Axis1D &ax = s->ax[0];
    add(pad_rows(ax.B.v, ax.m, 2 * ax.p + 1, padded(s, ax.m), false));
    if (ts.elimg[kind][i]) {
        dfree(s, ts.elimg[kind][i]);
        ts.elimg[kind][i] = nullptr;
    }
    return upload_padded<T>(s, img, &ts.elimg[kind][i], &ts.elimg_bytes[kind][i]);
}

// every K1 image of a table set
template <typename T>
int upload_rhs_images(ads_sim *s, TableSet &ts)
{
    for (int set = 0; set < NSETS; ++set) {
        int rc = upload_rhs_image<T>(s, ts, set, set, set);
        if (rc) return rc;
    }
    if (s->kind == ADS_ELASTIC)
        for (int i = 0; i < 3; ++i) {
            int rc = upload_rhs_image<T>(s, ts, IMG_EL + i, i == 0 ? SET_ELAS0 : SET_ELAS1,
                                         i == 1 ? SET_ELAS0 : SET_ELAS1);
            if (rc) return rc;
        }
    if (s->fused_el)
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 2; ++k) {
                int rc = upload_el_image<T>(s, ts, k, i);
                if (rc) return rc;
            }
    return ADS_OK;
}

template <typename T>
int upload_line(ads_sim *s, int set, int axis, LineTables *lt)
{
    int rc = upload_padded<T>(s, s->hline[set][axis], &lt->base, &lt->bytes);
    lt->S = s->lineS[axis];
    lt->seg = s->seg;
    return rc;
}

template <typename T>
int build_tables(ads_sim *s, TableSet &ts)
{
    const double eta = 0.25 * s->tau * s->tau;
    // host images (FP64), once
    if (s->hM[0].empty()) {
        for (int a = 0; a < 3; ++a) {
            const ads::Axis1D &ax = s->ax[a];
            const int mp = padded(s, ax.m), W = 2 * ax.p + 1;
            s->hM[a] = pad_rows(ax.M.v, ax.m, W, mp, false);
            s->hK[a] = pad_rows(ax.K.v, ax.m, W, mp, false);
            int S = 0;
            try {
                s->hline[SET_IDENT][a] = line_image(s, identity_factor(ax.m, ax.p), &S);
                s->hline[SET_MASS][a] = line_image(s, ads::factor_axis(ax, 0.0), &S);
                if (s->kind == ADS_SCALAR_WAVE) {
                    s->hline[SET_SPLIT][a] = line_image(s, ads::factor_axis(ax, eta * s->c2), &S);
                } else {
                    const double c[2] = {2 * s->mu + s->lam, s->mu};
                    for (int k = 0; k < 2; ++k)
                        s->hline[SET_ELAS0 + k][a] =
                            line_image(s, ads::factor_axis(ax, s->tau * s->tau * c[k] / (4 * s->rho)), &S);
                }
            } catch (const std::exception &e) {
                return fail(ADS_ERR_INVALID_ARG, e.what());
            }
            s->lineS[a] = S;
        }
    }
    for (int a = 0; a < 3; ++a) {
        const ads::Axis1D &ax = s->ax[a];
        const int mp = padded(s, ax.m), W = 2 * ax.p + 1;
        int rc;
        if ((rc = upload<T>(s, s->hM[a], &ts.M[a]))) return rc;
        if ((rc = upload<T>(s, s->hK[a], &ts.K[a]))) return rc;
        if ((rc = upload<T>(s, pad_rows(ax.B.v, ax.m, W, mp, false), &ts.B[a]))) return rc;
        if ((s->d.off == 0 || ax.ne == 0) && (rc = upload<T>(s, pad_rows(ax.Bt.v, ax.m, W, mp, false), &ts.Bt[a])))
            return rc;
        for (int set = 0; set < NSETS; ++set)
            if (!s->hline[set][a].empty() && (rc = upload_line<T>(s, set, a, &ts.line[set][a]))) return rc;
        if (s->kind == ADS_SCALAR_WAVE) {
            std::vector<double> g(ax.M.v.size());
            for (size_t i = 0; i < g.size(); ++i) g[i] = ax.M.v[i] + eta * s->c2 * ax.K.v[i];
            if ((rc = upload<T>(s, g, &ts.gband[a]))) return rc;
        }
    }
    return upload_rhs_images<T>(s, ts);
}

template <typename T>
ads::LineDev<T> line_dev(const LineTables &lt)
{
    ads::LineDev<T> l;
    l.base = (const T *)lt.base;
    l.S = lt.S;
    l.bytes = lt.bytes;
    l.seg = lt.seg;
    return l;
}

int segs(const ads_sim *s, int m) { return (m + s->seg - 1) / s->seg; }

void choose_tiles(ads_sim *s)
{
    const int Sx = segs(s, s->d.mx), Sy = segs(s, s->d.my);
    for (int pi = 0; pi < 2; ++pi) {
        const int el = pi == 0 ? 8 : 4;
        const int my = s->d.my;
        const size_t budget_fused = 220 * 1024, budget = 110 * 1024;
        const char *env = std::getenv("ADS_RHS_TILE");   // rows per tile, for experiments
        int ty = 0;
        auto fits = [&](int t, size_t b) { return ads::rhs_smem_bytes(s->p, el, s->d, t, Sx, Sy, s->seg) <= b; };
        if (env && std::sscanf(env, "%d", &ty) == 1 && ty > 0) {
            ty = std::min(ty, my);
            if (!fits(ty, budget_fused)) ty = 0;
        }
        if (ty == 0) {
            if (fits(my, budget_fused)) {
                ty = my;
            } else {
                ty = std::min(my, 32);
                while (ty > 1 && !fits(ty, budget)) ty /= 2;
            }
        }
        s->ty[pi] = ty;
        s->tz[pi] = 1;
        s->fuse[pi] = (ty == my) ? 1 : 0;
        // the elastic K1 holds a third plane (and Bx): the whole plane when it
        // fits, else row tiles followed by a y sweep
        auto fits3 = [&](int t, size_t b) {
            return ads::rhs_smem_bytes(s->p, el, s->d, t, Sx, Sy, s->seg, 0, 3) <= b;
        };
        int te = my;
        if (!fits3(te, budget_fused)) {
            te = std::min(my, 32);
            while (te > 1 && !fits3(te, budget)) te /= 2;
        }
        s->ty_el[pi] = te;
    }
}

template <typename T>
const TableSet &tables_for(const ads_sim *s)
{
    return sizeof(T) == 8 ? s->t64 : s->t32;
}

template <typename T>
ads::RhsArgs<T> rhs_args(const ads_sim *s, const T *in, T *out, int set, int toff, bool with_src)
{
    const TableSet &ts = tables_for<T>(s);
    const int pi = sizeof(T) == 8 ? 0 : 1;
    ads::RhsArgs<T> a{};
    a.in = in;
    a.out = out;
    a.d = s->d;
    for (int k = 0; k < 3; ++k) {
        a.bandM[k].v = (const T *)ts.M[k];
        a.bandK[k].v = (const T *)ts.K[k];
        a.bandM[k].lo = a.bandK[k].lo = s->ax[k].lo;
        a.bandM[k].hi = a.bandK[k].hi = s->ax[k].hi;
    }
    a.lx = line_dev<T>(ts.line[set][0]);
    a.ly = line_dev<T>(ts.line[set][1]);
    a.img = (const T *)ts.img[set];
    a.img_bytes = ts.img_bytes[set];
    a.c2 = (T)s->c2;
    if (with_src && s->has_src) {
        if (ts.srcfield) {
            a.srcfield = (const T *)ts.srcfield;
        } else {
            a.src.fx = (const T *)ts.src[0];
            a.src.fy = (const T *)ts.src[1];
            a.src.fz = (const T *)ts.src[2];
        }
        a.src.amp = 1.0;   // amplitude folded into the load vectors
        a.src.freq = s->src.freq;
        a.src.t0 = s->src.t0;
    }
    a.step = s->d_step;
    a.toff = toff;
    a.tau = s->tau;
    a.ty = s->ty[pi];
    a.pair = sizeof(T) == 4 ? s->pair[pi] : 0;
    a.err = s->d_err;
    return a;
}

// out = A^{-1} R along y then z (mode 0) after K1 has done x (and maybe y)
template <typename T>
int sweeps_yz(ads_sim *s, T *data, int set, bool y_done)
{
    ads::ColArgs<T> c{};
    c.d = s->d;
    c.mode = 0;
    c.in = data;
    c.out = data;
    c.err = s->d_err;
    if (!y_done) {
        c.axis = 1;
        c.ln = line_dev<T>(tables_for<T>(s).line[set][1]);
        ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    }
    c.axis = 2;
    c.ln = line_dev<T>(tables_for<T>(s).line[set][2]);
    ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    return ADS_OK;
}

// Generic Kronecker solve of an arbitrary FP64 interior field (in place).
int kron_solve64(ads_sim *s, double *data, int set)
{
    // the factor rows open the line buffer
    ADS_CK(ads::launch_solve_x<double>(s->p, (const double *)s->t64.line[set][0].base, data, s->d, s->stream));
    return sweeps_yz<double>(s, data, set, false);
}

// out = c2 K in (FP64), through the fused RHS kernel with identity factors:
// K1 computes fac_x^{-1}(F - c2 K in) = -c2 K in.
int apply_stiff64(ads_sim *s, const double *in, double *out)
{
    ads::RhsArgs<double> a = rhs_args<double>(s, in, out, SET_IDENT, 0, false);
    ADS_CK(ads::launch_rhs<double>(s->p, s->seg, a, s->stream));
    ADS_CK(ads::launch_axpby(0.0, out, -1.0, out, s->d.count(), s->stream));
    return ADS_OK;
}

// out = (A_x.A_y.A_z) in with bands (FP64), scratch tmp
int apply_kron64(ads_sim *s, void *const *band, const double *in, double *out, double *tmp)
{
    ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)band[0], 0, in, out, s->d, 1.0, 0.0, 0, s->stream));
    ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)band[1], 1, out, tmp, s->d, 1.0, 0.0, 0, s->stream));
    ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)band[2], 2, tmp, out, s->d, 1.0, 0.0, 0, s->stream));
    return ADS_OK;
}

int dot64_n(ads_sim *s, const double *x, const double *y, long long n, double *result_host)
{
    Scratch sc(s);
    const int nb = 304;
    double *part = (double *)sc.get(sizeof(double) * 2 * nb + sizeof(double));
    if (!part) return fail(ADS_ERR_OOM, "scratch allocation failed");
    double *res = part + 2 * nb;
    ADS_CK(ads::launch_dot(x, y, n, part, nb, res, s->stream));
    ADS_CK(cudaMemcpyAsync(result_host, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    ADS_CK(cudaStreamSynchronize(s->stream));
    return ADS_OK;
}

int dot64(ads_sim *s, const double *x, const double *y, double *result_host)
{
    return dot64_n(s, x, y, s->d.count(), result_host);
}

// stage a full FP64 field (host or device) into an interior FP64 array
int stage_in(ads_sim *s, Scratch &sc, const double *src, int mem, size_t count, double *dst_interior, double scale)
{
    const double *full = src;
    if (mem == ADS_HOST) {
        double *tmp = (double *)sc.get(count * sizeof(double));
        if (!tmp) return fail(ADS_ERR_OOM, "scratch allocation failed");
        ADS_CK(cudaMemcpyAsync(tmp, src, count * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        full = tmp;
    }
    ADS_CK(ads::launch_pack<double>(full, dst_interior, s->d, scale, s->stream));
    return ADS_OK;
}

int stage_out(ads_sim *s, Scratch &sc, const double *interior, double *dst, int mem, size_t count)
{
    double *full = dst;
    if (mem == ADS_HOST) {
        full = (double *)sc.get(count * sizeof(double));
        if (!full) return fail(ADS_ERR_OOM, "scratch allocation failed");
    }
    ADS_CK(ads::launch_unpack<double>(interior, full, s->d, s->stream));
    if (mem == ADS_HOST) {
        ADS_CK(cudaMemcpyAsync(dst, full, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    return ADS_OK;   // the caller waits for the stream once, after its last field
}

// A bounded wait that gave up records a nonzero word; report it once.
int check_device_error(ads_sim *s)
{
    int e = 0;
    ADS_CK(cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        cudaMemset(s->d_err, 0, sizeof(int));
        if (e == 2) return fail(ADS_ERR_CUDA, "a kernel found a misaligned TMA shared-memory address and skipped it");
        if (e == 3) return fail(ADS_ERR_UNSUPPORTED, "a sweep kernel was launched with fewer warps than line segments");
        return fail(ADS_ERR_TIMEOUT, "a device-side wait timed out (TMA transfer did not complete)");
    }
    return ADS_OK;
}

size_t full_count(const ads_sim *s)
{
    const int o = 2 * s->d.off, oz = 2 * s->d.offz;
    return (size_t)(s->d.mx + o) * (s->d.my + o) * (s->d.mz + oz) * (s->kind == ADS_ELASTIC ? 3 : 1);
}

// a = M^{-1}(F(t_n) - K u) for an FP64 interior u
int consistent_accel64(ads_sim *s, const double *u, double *a)
{
    ads::RhsArgs<double> r = rhs_args<double>(s, u, a, SET_MASS, 0, true);
    ADS_CK(ads::launch_rhs<double>(s->p, s->seg, r, s->stream));
    return sweeps_yz<double>(s, a, SET_MASS, r.ty == s->d.my);
}

template <typename T>
int set_pq(ads_sim *s, const double *u, const double *v, const double *a)
{
    ADS_CK(ads::launch_uva_to_pq<T>(u, v, a, (T *)s->P, (T *)s->Q, (T *)s->A, s->d, s->tau, s->stream));
    return ADS_OK;
}

template <typename T>
int get_uva(ads_sim *s, double *u, double *v, double *a)
{
    ADS_CK(ads::launch_pq_to_uva<T>((const T *)s->P, (const T *)s->Q, (const T *)s->A, u, v, a, s->d, s->tau,
                                    s->stream));
    return ADS_OK;
}

// Optional per-kernel event recording (measurement entry point only).
struct KernelTimer {
    std::vector<cudaEvent_t> ev;
    std::vector<const char *> names;
    int mark(cudaStream_t st, const char *name)
    {
        cudaEvent_t e;
        ADS_CK(cudaEventCreate(&e));
        ADS_CK(cudaEventRecord(e, st));
        ev.push_back(e);
        names.push_back(name);
        return ADS_OK;
    }
    ~KernelTimer()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Launch arguments of one scalar-wave step: K1 (RHS + x [+ y]), K2 (y
// sweep, only when K1's tile does not span y), K3 (z sweep + update).
template <typename T>
struct PwaveLaunch {
    ads::RhsArgs<T> rhs;
    ads::ColArgs<T> ycol, zcol;
    bool fused;
};

template <typename T>
PwaveLaunch<T> pwave_launch(const ads_sim *s, bool write_a)
{
    const TableSet &ts = tables_for<T>(s);
    PwaveLaunch<T> L;
    L.rhs = rhs_args<T>(s, (const T *)s->P, (T *)s->X, SET_SPLIT, 1, true);
    L.fused = L.rhs.ty == s->d.my;
    ads::ColArgs<T> c{};
    c.d = s->d;
    c.in = (const T *)s->X;
    c.out = (T *)s->X;
    c.err = s->d_err;
    c.axis = 1;
    c.mode = 0;
    c.ln = line_dev<T>(ts.line[SET_SPLIT][1]);
    L.ycol = c;
    c.axis = 2;
    c.mode = 1;
    c.ln = line_dev<T>(ts.line[SET_SPLIT][2]);
    c.P = (T *)s->P;
    c.Q = (T *)s->Q;
    c.A = (T *)s->A;
    c.tau2 = (T)(s->tau * s->tau);
    c.write_a = write_a ? 1 : 0;
    c.step = s->d_step;
    L.zcol = c;
    return L;
}

// FP32 step with one FP64 residual correction (iterative refinement):
//   a  = G~^{-1} R          FP32 sweeps (K1, K2, z sweep without update)
//   r  = F - c2 K p - G~ a  in FP64 from the FP32 state p
//   a += G~^{-1} r          FP32 sweeps of the residual
// then the Newmark update of (p, q) with the corrected a.
int pwave_refine_step(ads_sim *s, bool write_a, KernelTimer *kt)
{
    const PwaveLaunch<float> L = pwave_launch<float>(s, write_a);
    const long long n = s->d.count();
    float *X = (float *)s->X;
    double *R = (double *)s->R64, *P64 = (double *)s->P64, *A64 = (double *)s->A64, *T = (double *)s->T64;
    int rc;
    if (kt && (rc = kt->mark(s->stream, L.fused ? "rhs_xy_sweep" : "rhs_x_sweep"))) return rc;
    ADS_CK(ads::launch_rhs_group<float>(s->p, &L.rhs, 1, s->stream));
    if (kt && (rc = kt->mark(s->stream, "yz_sweeps"))) return rc;
    if ((rc = sweeps_yz<float>(s, X, SET_SPLIT, L.fused))) return rc;
    if (kt && (rc = kt->mark(s->stream, "residual_fp64"))) return rc;
    ADS_CK(ads::launch_convert<float>((const float *)s->P, P64, n, s->stream));
    ADS_CK(ads::launch_convert<float>(X, A64, n, s->stream));
    // R = F(t_{n+1}) - c2 K p: K1 in FP64 with identity factors
    ads::RhsArgs<double> r = rhs_args<double>(s, P64, R, SET_IDENT, 1, true);
    ADS_CK(ads::launch_rhs_group<double>(s->p, &r, 1, s->stream));
    if ((rc = apply_kron64(s, s->t64.gband, A64, T, P64))) return rc;
    ADS_CK(ads::launch_axpby(-1.0, T, 1.0, R, n, s->stream));
    if (kt && (rc = kt->mark(s->stream, "correction_sweeps"))) return rc;
    ADS_CK(ads::launch_convert_from<float>(R, X, n, s->stream));
    ads::RhsArgs<float> rd = rhs_args<float>(s, X, X, SET_SPLIT, 0, false);   // given RHS: x (and y) sweeps
    rd.direct = 1;
    ADS_CK(ads::launch_rhs_group<float>(s->p, &rd, 1, s->stream));
    if ((rc = sweeps_yz<float>(s, X, SET_SPLIT, rd.ty == s->d.my || rd.pair))) return rc;
    ADS_CK(ads::launch_add_converted<float>(X, A64, n, s->stream));
    ADS_CK(ads::launch_convert_from<float>(A64, X, n, s->stream));
    if (kt && (rc = kt->mark(s->stream, "update"))) return rc;
    ADS_CK(ads::launch_pq_update<float>((float *)s->P, (float *)s->Q, (float *)s->A, X, n,
                                        (float)(s->tau * s->tau), write_a ? 1 : 0, s->d_step, s->stream));
    if (kt && (rc = kt->mark(s->stream, ""))) return rc;
    return ADS_OK;
}

// One scalar-wave step of one simulation (a group of one).
template <typename T>
int pwave_step(ads_sim *s, bool write_a, KernelTimer *kt = nullptr)
{
    if (sizeof(T) == 4 && s->refine) return pwave_refine_step(s, write_a, kt);
    const PwaveLaunch<T> L = pwave_launch<T>(s, write_a);
    int rc;
    if (kt && (rc = kt->mark(s->stream, L.fused ? "rhs_xy_sweep" : "rhs_x_sweep"))) return rc;
    ADS_CK(ads::launch_rhs_group<T>(s->p, &L.rhs, 1, s->stream));
    if (!L.fused) {
        if (kt && (rc = kt->mark(s->stream, "y_sweep"))) return rc;
        ADS_CK(ads::launch_col_group<T>(s->p, &L.ycol, nullptr, 1, s->stream));
    }
    if (kt && (rc = kt->mark(s->stream, "z_sweep_update"))) return rc;
    ADS_CK(ads::launch_col_group<T>(s->p, &L.zcol, s->has_maps ? &s->upd_maps : nullptr, 1, s->stream));
    if (kt && (rc = kt->mark(s->stream, ""))) return rc;
    return ADS_OK;
}

// One scalar-wave step of a group of simulations of one degree and
// precision, in three grouped launches on stream st (Sec. 2 step for every
// member; the members are independent, so each result is the one its
// simulation gets alone).
template <typename T>
int pwave_group_step(const std::vector<ads_sim *> &g, cudaStream_t st, bool write_a)
{
    if (g.empty()) return ADS_OK;
    std::vector<ads::RhsArgs<T>> r;
    std::vector<ads::ColArgs<T>> ya, za;
    std::vector<ads::ColMaps> zm;
    bool all_maps = true;
    for (ads_sim *s : g) {
        const PwaveLaunch<T> L = pwave_launch<T>(s, write_a);
        r.push_back(L.rhs);
        if (!L.fused) ya.push_back(L.ycol);
        za.push_back(L.zcol);
        zm.push_back(s->upd_maps);
        all_maps = all_maps && s->has_maps;
    }
    const int p = g[0]->p;
    ADS_CK(ads::launch_rhs_group<T>(p, r.data(), (int)r.size(), st));
    if (!ya.empty()) ADS_CK(ads::launch_col_group<T>(p, ya.data(), nullptr, (int)ya.size(), st));
    ADS_CK(ads::launch_col_group<T>(p, za.data(), all_maps ? zm.data() : nullptr, (int)za.size(), st));
    return ADS_OK;
}

// ------------------------------------------------------------------ elasticity
// Blocks of Upsilon with the Dirichlet restriction (B^T = -B on the interior):
//   Ups_ii = mu (Kx My Mz + Mx Ky Mz + Mx My Kz) + (mu + lam) [K on axis i]
//   Ups_ij = -(mu + lam) [B on axis i, B on axis j, M on the third],  i != j
// (bilinear form 2 mu e(w):e(u) + lam div w div u, Sec. 5).

// Kronecker term coef * (A0 (x) A1 (x) A2) in; which[a]: 0 = M, 1 = K, 2 = B
template <typename T>
ads::KronTerm<T> kterm(const ads_sim *s, const int *which, const T *in, T coef)
{
    const TableSet &ts = tables_for<T>(s);
    const void *band[3];
    for (int a = 0; a < 3; ++a)
        band[a] = which[a] == 0 ? ts.M[a] : (which[a] == 1 ? ts.K[a] : (which[a] == 2 ? ts.B[a] : ts.Bt[a]));
    ads::KronTerm<T> t{};
    t.bx = (const T *)band[0];
    t.by = (const T *)band[1];
    t.bz = (const T *)band[2];
    t.in = in;
    t.alpha = coef;
    return t;
}

template <typename T>
ads::KronTerm<T> plain_term(const T *in, T coef)
{
    ads::KronTerm<T> t{};
    t.in = in;
    t.alpha = coef;
    t.plain = 1;
    return t;
}

// a full term list marks the sum invalid (nt = -1): the launch then fails
template <typename T>
void add_term(ads::KronSum<T> &ks, const ads::KronTerm<T> &t)
{
    if (ks.nt < 0 || ks.nt >= ads::kMaxKronTerms) {
        ks.nt = -1;
        return;
    }
    ks.t[ks.nt++] = t;
}

// Off-diagonal block Ups_ij (i != j) as Kronecker terms scaled by coef:
//   mu [B^T on axis i, B on axis j] + lam [B on axis i, B^T on axis j]  (M on the third);
// with the Dirichlet restriction B^T = -B, so this is -(mu + lam) [B_i B_j]
// (one term).
template <typename T>
void add_offdiag(const ads_sim *s, ads::KronSum<T> &ks, int i, int j, const T *in, double coef)
{
    int b[3] = {0, 0, 0};
    if (s->d.off == 1) {
        b[i] = 2;
        b[j] = 2;
        add_term(ks, kterm<T>(s, b, in, (T)(-coef * (s->lam + s->mu))));
        return;
    }
    b[i] = 3;
    b[j] = 2;
    add_term(ks, kterm<T>(s, b, in, (T)(coef * s->mu)));
    b[i] = 2;
    b[j] = 3;
    add_term(ks, kterm<T>(s, b, in, (T)(coef * s->lam)));
}

// out_i = coef (Ups U)_i, i = 0..2 (component stride cnt), one launch per
// component:  (Ups U)_i = sum_a c_ia (K on axis a, M elsewhere) U_i
//                         + sum_{j != i} Ups_ij U_j,   c_ia = mu + (mu + lam) [a == i]
template <typename T>
int apply_upsilon(ads_sim *s, const T *U, T *out, T *ta, T *tb, T coef = T(1))
{
    (void)ta;
    (void)tb;
    const long long cnt = s->d.count();
    const double lm = s->lam + s->mu;
    for (int i = 0; i < 3; ++i) {
        ads::KronSum<T> ks{};
        for (int a = 0; a < 3; ++a) {
            int w[3] = {0, 0, 0};
            w[a] = 1;
            add_term(ks, kterm<T>(s, w, U + i * cnt, (T)(coef * (s->mu + (a == i ? lm : 0.0)))));
        }
        for (int j = 0; j < 3; ++j)
            if (j != i) add_offdiag<T>(s, ks, i, j, U + j * cnt, (double)coef);
        ADS_CK(ads::launch_kron_sum<T>(s->p, ks, out + i * cnt, s->d, s->stream));
    }
    return ADS_OK;
}

// data <- (x)_xi (M_xi + d_i,xi K_xi)^{-1} data, d = tau^2 c_i,xi / (4 rho),
// c_i,xi = 2 mu + lam on axis i, mu otherwise (eq. spill): K1 in direct
// mode (x, and y when the plane fits), then the y sweep if needed and the z
// sweep
template <typename T>
int elastic_diag_solve(ads_sim *s, int i, T *data)
{
    const TableSet &ts = tables_for<T>(s);
    auto set = [&](int a) { return a == i ? SET_ELAS0 : SET_ELAS1; };
    ads::RhsArgs<T> r = rhs_args<T>(s, data, data, set(0), 0, false);
    r.direct = 1;
    r.ly = line_dev<T>(ts.line[set(1)][1]);
    r.img = (const T *)ts.img[IMG_EL + i];
    r.img_bytes = ts.img_bytes[IMG_EL + i];
    ADS_CK(ads::launch_rhs_group<T>(s->p, &r, 1, s->stream));
    ads::ColArgs<T> c{};
    c.d = s->d;
    c.mode = 0;
    c.in = data;
    c.out = data;
    c.err = s->d_err;
    if (r.ty != s->d.my) {
        c.axis = 1;
        c.ln = line_dev<T>(ts.line[set(1)][1]);
        ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    }
    c.axis = 2;
    c.ln = line_dev<T>(ts.line[set(2)][2]);
    ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    return ADS_OK;
}

// r_i += tau^2 dir_i r(t_{n+toff}) F  (body force at level n)
template <typename T>
int add_body_force(ads_sim *s, T *r, double scale, int toff)
{
    if (!s->has_src) return ADS_OK;
    const TableSet &ts = tables_for<T>(s);
    const long long cnt = s->d.count();
    for (int i = 0; i < 3; ++i) {
        const double di = s->src.shape.dir[i];
        if (di == 0.0) continue;
        if (ts.srcfield)
            ADS_CK(ads::launch_add_field<T>(r + i * cnt, (const T *)ts.srcfield, cnt, scale * di, s->src.freq,
                                            s->src.t0, s->d_step, toff, s->tau, s->stream));
        else
            ADS_CK(ads::launch_add_source<T>(r + i * cnt, s->d, (const T *)ts.src[0], (const T *)ts.src[1],
                                             (const T *)ts.src[2], scale * di, s->src.freq, s->src.t0, s->d_step,
                                             toff, s->tau, s->stream));
    }
    return ADS_OK;
}

// One alternating-triangular step (eqs. decom, pre, corr, spill, gen with
// sigma = 1/2):  D delta = tau^2 (f^n - Ups U^n),
//   D = (rho M + tau^2/2 Ups1~) (rho M)^{-1} (rho M + tau^2/2 Ups2~),
// block-lower solve, rho M, block-upper solve, U^{n+1} = 2U^n - U^{n-1} + delta.
template <typename T>
int elastic_step_fused(ads_sim *s, KernelTimer *kt);

template <typename T>
int elastic_step(ads_sim *s, KernelTimer *kt = nullptr)
{
    if (s->fused_el) return elastic_step_fused<T>(s, kt);
    const long long cnt = s->d.count();
    T *U = (T *)s->U, *Up = (T *)s->Up, *R = (T *)s->R, *Y = (T *)s->Y;
    const T tau2 = (T)(s->tau * s->tau), rho = (T)s->rho;
    int rc;
    if (kt && (rc = kt->mark(s->stream, "elastic_rhs"))) return rc;
    // R = tau^2 (f^n - Ups U^n)
    if ((rc = apply_upsilon<T>(s, U, R, nullptr, nullptr, -tau2))) return rc;
    if ((rc = add_body_force<T>(s, R, s->tau * s->tau, 0))) return rc;
    if (kt && (rc = kt->mark(s->stream, "elastic_lower"))) return rc;
    // lower: y_i = L~_i^{-1} (R_i / rho - tau^2/(2 rho) sum_{j<i} Ups_ij y_j)
    const double hr = 0.5 * s->tau * s->tau / s->rho;
    for (int i = 0; i < 3; ++i) {
        ads::KronSum<T> ks{};
        add_term(ks, plain_term<T>(R + i * cnt, T(1) / rho));
        for (int j = 0; j < i; ++j) add_offdiag<T>(s, ks, i, j, Y + j * cnt, -hr);
        ADS_CK(ads::launch_kron_sum<T>(s->p, ks, Y + i * cnt, s->d, s->stream));
        if ((rc = elastic_diag_solve<T>(s, i, Y + i * cnt))) return rc;
    }
    if (kt && (rc = kt->mark(s->stream, "elastic_upper"))) return rc;
    // rho M y, then upper: delta_i = L~_i^{-1} (M y_i - tau^2/(2 rho) sum_{j>i} Ups_ij delta_j),
    // delta stored in R
    for (int i = 2; i >= 0; --i) {
        ads::KronSum<T> ks{};
        const int m3[3] = {0, 0, 0};
        add_term(ks, kterm<T>(s, m3, Y + i * cnt, T(1)));
        for (int j = i + 1; j < 3; ++j) add_offdiag<T>(s, ks, i, j, R + j * cnt, -hr);
        ADS_CK(ads::launch_kron_sum<T>(s->p, ks, R + i * cnt, s->d, s->stream));
        if ((rc = elastic_diag_solve<T>(s, i, R + i * cnt))) return rc;
    }
    if (kt && (rc = kt->mark(s->stream, "elastic_update"))) return rc;
    ADS_CK(ads::launch_atm_update<T>(U, Up, R, 3 * cnt, s->d_step, s->stream));
    if (kt && (rc = kt->mark(s->stream, ""))) return rc;
    return ADS_OK;
}

// Fused alternating-triangular step (Dirichlet): every diagonal-block solve
// is one elastic K1 (the block's right-hand side by sum factorisation, with
// the off-diagonal blocks Ups_ij of the other components as extra Kronecker
// terms, then the x [and y] sweeps) and one z sweep:
//   lower, i = 0, 1, 2:  rhs_i = tau^2/rho (f_i - sum_j Ups_ij U^n_j)
//                                - tau^2/(2 rho) sum_{j<i} Ups_ij y_j,
//                        y_i = L~_i^{-1} rhs_i
//   upper, i = 2, 1, 0:  rhs_i = M y_i - tau^2/(2 rho) sum_{j>i} Ups_ij delta_j,
//                        delta_i = L~_i^{-1} rhs_i
//   U^{n+1} = 2U^n - U^{n-1} + delta
// (eqs. decom, pre, corr, spill, gen with sigma = 1/2; L~_i has the factored
// blocks of eq. spill scaled by 1/rho).  Ups_ij (i != j) = -(mu + lam)
// [B on axes i and j, M on the third].  13 launches per step.
template <typename T>
int elastic_block_solve(ads_sim *s, int kind, int i, const T *main_in, T *out, const ads::RhsElas<T> &el)
{
    const TableSet &ts = tables_for<T>(s);
    const int pi = sizeof(T) == 8 ? 0 : 1;
    auto set = [&](int a) { return a == i ? SET_ELAS0 : SET_ELAS1; };
    ads::RhsArgs<T> r = rhs_args<T>(s, main_in, out, set(0), 0, kind == 0);
    r.ly = line_dev<T>(ts.line[set(1)][1]);
    r.img = (const T *)ts.elimg[kind][i];
    r.img_bytes = ts.elimg_bytes[kind][i];
    r.c2 = T(-1);
    r.pair = 0;
    r.ty = s->ty_el[pi];
    r.direct = 0;
    // body force of component i at level n: tau^2/rho r(t_n) dir_i g
    r.src.amp = s->tau * s->tau / s->rho * s->src.shape.dir[i];
    ADS_CK(ads::launch_rhs_el<T>(s->p, r, el, s->stream));
    ads::ColArgs<T> c{};
    c.d = s->d;
    c.mode = 0;
    c.in = out;
    c.out = out;
    c.err = s->d_err;
    if (r.ty != s->d.my) {
        c.axis = 1;
        c.ln = line_dev<T>(ts.line[set(1)][1]);
        ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    }
    c.axis = 2;
    c.ln = line_dev<T>(ts.line[set(2)][2]);
    ADS_CK(ads::launch_col<T>(s->p, s->seg, c, s->stream));
    return ADS_OK;
}

// the off-diagonal block Ups_ij applied to `in`, coef times, as an extra term
// of component i's elastic K1: B on axes i and j, M on the third
template <typename T>
void add_extra(const ads_sim *s, ads::RhsElas<T> &el, int i, int j, const T *in, double coef)
{
    const TableSet &ts = tables_for<T>(s);
    auto band = [&](int a) { return (const T *)((a == i || a == j) ? ts.B[a] : ts.M[a]); };
    ads::ExtraTerm<T> &e = el.ex[el.n++];
    e.in = in;
    e.by = band(1);
    e.bz = band(2);
    e.coef = (T)(coef * -(s->lam + s->mu));
    e.slot = (i == 0 || j == 0) ? 3 : 2;
    e.init = 0;
    if (e.slot == 3 && !el.s3) {
        el.s3 = 1;
        e.init = 1;
    }
}

template <typename T>
int elastic_step_fused(ads_sim *s, KernelTimer *kt)
{
    const long long cnt = s->d.count();
    T *U = (T *)s->U, *Up = (T *)s->Up, *R = (T *)s->R, *Y = (T *)s->Y;
    const double g = s->tau * s->tau / s->rho, h = 0.5 * g;
    int rc;
    if (kt && (rc = kt->mark(s->stream, "elastic_lower"))) return rc;
    for (int i = 0; i < 3; ++i) {
        ads::RhsElas<T> el{};
        // the diagonal block -tau^2/rho Ups_ii U_i, Ups_ii = sum_a c_ia [K on axis a]
        el.cx = (T)(-g * el_coef(s, i, 0));
        el.cy = (T)(-g * el_coef(s, i, 1));
        el.cz = (T)(-g * el_coef(s, i, 2));
        for (int j = 0; j < 3; ++j)
            if (j != i) add_extra<T>(s, el, i, j, U + j * cnt, -g);   // -tau^2/rho Ups_ij U_j
        for (int j = 0; j < i; ++j) add_extra<T>(s, el, i, j, Y + j * cnt, -h);
        if ((rc = elastic_block_solve<T>(s, 0, i, U + i * cnt, Y + i * cnt, el))) return rc;
    }
    if (kt && (rc = kt->mark(s->stream, "elastic_upper"))) return rc;
    for (int i = 2; i >= 0; --i) {
        ads::RhsElas<T> el{};
        el.cx = T(1);   // M y_i: X1 = Mx, no K part
        el.cy = T(0);
        el.cz = T(0);
        for (int j = i + 1; j < 3; ++j) add_extra<T>(s, el, i, j, R + j * cnt, -h);
        if ((rc = elastic_block_solve<T>(s, 1, i, Y + i * cnt, R + i * cnt, el))) return rc;
    }
    if (kt && (rc = kt->mark(s->stream, "elastic_update"))) return rc;
    ADS_CK(ads::launch_atm_update<T>(U, Up, R, 3 * cnt, s->d_step, s->stream));
    if (kt && (rc = kt->mark(s->stream, ""))) return rc;
    return ADS_OK;
}

// U^{-1} = U0 - tau V0 + tau^2/2 A0,  A0 = (rho M)^{-1}(f(t_n) - Ups U0)   (FP64)
int elastic_set64(ads_sim *s, Scratch &sc, const double *U0, const double *V0)
{
    const long long cnt = s->d.count();
    const size_t bytes = (size_t)cnt * sizeof(double);
    double *A = (double *)sc.get(3 * bytes), *t1 = (double *)sc.get(bytes), *t2 = (double *)sc.get(bytes);
    double *Upv = (double *)sc.get(3 * bytes);
    if (!A || !t1 || !t2 || !Upv) return fail(ADS_ERR_OOM, "scratch allocation failed");
    int rc;
    if ((rc = apply_upsilon<double>(s, U0, A, t1, t2))) return rc;
    ADS_CK(ads::launch_lincomb<double>(A, -1.0, A, 0.0, nullptr, 3 * cnt, s->stream));
    if ((rc = add_body_force<double>(s, A, 1.0, 0))) return rc;
    for (int i = 0; i < 3; ++i)
        if ((rc = kron_solve64(s, A + i * cnt, SET_MASS))) return rc;
    // Up = U0 - tau V0 + tau^2/(2 rho) A
    ADS_CK(ads::launch_lincomb<double>(Upv, 1.0, U0, -s->tau, V0, 3 * cnt, s->stream));
    ADS_CK(ads::launch_lincomb<double>(Upv, 1.0, Upv, 0.5 * s->tau * s->tau / s->rho, A, 3 * cnt, s->stream));
    if (s->prec == ADS_FP64) {
        ADS_CK(cudaMemcpyAsync(s->U, U0, 3 * bytes, cudaMemcpyDeviceToDevice, s->stream));
        ADS_CK(cudaMemcpyAsync(s->Up, Upv, 3 * bytes, cudaMemcpyDeviceToDevice, s->stream));
    } else {
        ADS_CK(ads::launch_convert_from<float>(U0, (float *)s->U, 3 * cnt, s->stream));
        ADS_CK(ads::launch_convert_from<float>(Upv, (float *)s->Up, 3 * cnt, s->stream));
    }
    return ADS_OK;
}

int step_once(ads_sim *s, bool write_a)
{
    if (s->kind == ADS_ELASTIC) return s->prec == ADS_FP64 ? elastic_step<double>(s) : elastic_step<float>(s);
    return s->prec == ADS_FP64 ? pwave_step<double>(s, write_a) : pwave_step<float>(s, write_a);
}

int get_graph(ads_sim *s, int chunk, cudaGraphExec_t *out)
{
    auto it = s->graphs.find(chunk);
    if (it != s->graphs.end()) {
        *out = it->second;
        return ADS_OK;
    }
    cudaGraph_t g = nullptr;
    const unsigned long long before = ads::g_launches;
    ADS_CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    int rc = ADS_OK;
    for (int i = 0; i < chunk && rc == ADS_OK; ++i) rc = step_once(s, i == chunk - 1);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    s->graph_launches[chunk] = ads::g_launches - before;   // kernels recorded in the graph
    ads::g_launches = before;
    if (rc != ADS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ADS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ADS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    s->graphs[chunk] = ge;
    *out = ge;
    return ADS_OK;
}

// Captured graphs hold launch arguments: drop them whenever those change.
void drop_graphs(ads_sim *s)
{
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    s->graph_launches.clear();
    ++s->version;
}

// K1 images carry the source vectors: rebuild after a source change, and
// drop captured graphs (they hold the old image pointers)
int rebuild_images(ads_sim *s)
{
    int rc = upload_rhs_images<double>(s, s->t64);
    if (rc) return rc;
    if (s->prec == ADS_FP32 && (rc = upload_rhs_images<float>(s, s->t32))) return rc;
    drop_graphs(s);
    return ADS_OK;
}


// ------------------------------------------------------------------ batching

// Process-wide resources of grouped launches on one device: one stream per
// (precision, degree) group so that groups overlap, and a small cache of
// captured batch graphs keyed by the members' identities.
struct BatchKey {
    int prec, p, chunk;
    std::vector<std::pair<unsigned long long, unsigned long long>> ids;   // (uid, version) per member
    bool operator<(const BatchKey &o) const
    {
        if (prec != o.prec) return prec < o.prec;
        if (p != o.p) return p < o.p;
        if (chunk != o.chunk) return chunk < o.chunk;
        return ids < o.ids;
    }
};

struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;
    unsigned long long last_use = 0;
};

struct BatchRes {
    std::map<std::pair<int, int>, cudaStream_t> streams;
    std::map<BatchKey, BatchGraph> graphs;
    unsigned long long clock = 0;
};

constexpr int kBatchChunk = 16;        // steps per captured batch graph
constexpr size_t kBatchGraphs = 16;    // cached batch graphs per device

// Batch streams, graphs and the tuning cache are process-wide: one mutex
// serialises the host-side work of ads_batch_step, ads_autotune and the
// graph clean-up of ads_destroy across host threads.
std::mutex &batch_mutex()
{
    static std::mutex m;
    return m;
}

BatchRes &batch_res(int device)
{
    static std::map<int, BatchRes> res;
    return res[device];
}

// drop cached batch graphs that hold a simulation about to be destroyed
void forget_batch_graphs(const ads_sim *s)
{
    std::lock_guard<std::mutex> lock(batch_mutex());
    BatchRes &br = batch_res(s->device);
    for (auto it = br.graphs.begin(); it != br.graphs.end();) {
        bool holds = false;
        for (const auto &id : it->first.ids) holds = holds || id.first == s->uid;
        if (holds) {
            cudaGraphExecDestroy(it->second.exec);
            it = br.graphs.erase(it);
        } else {
            ++it;
        }
    }
}

int group_stream(BatchRes &br, int prec, int p, cudaStream_t *out)
{
    auto it = br.streams.find({prec, p});
    if (it == br.streams.end()) {
        cudaStream_t st;
        ADS_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        it = br.streams.emplace(std::make_pair(prec, p), st).first;
    }
    *out = it->second;
    return ADS_OK;
}

int group_steps(const std::vector<ads_sim *> &g, cudaStream_t st, int n, bool write_last)
{
    for (int i = 0; i < n; ++i) {
        const bool wa = write_last && i == n - 1;
        int rc = g[0]->prec == ADS_FP64 ? pwave_group_step<double>(g, st, wa) : pwave_group_step<float>(g, st, wa);
        if (rc) return rc;
    }
    return ADS_OK;
}

// captured graph of kBatchChunk grouped steps for the members of g
int batch_graph(BatchRes &br, const std::vector<ads_sim *> &g, cudaStream_t st, BatchGraph **out)
{
    BatchKey key{g[0]->prec, g[0]->p, kBatchChunk, {}};
    for (ads_sim *s : g) key.ids.push_back({s->uid, s->version});
    auto it = br.graphs.find(key);
    if (it == br.graphs.end()) {
        if (br.graphs.size() >= kBatchGraphs) {   // evict the least recently used
            auto lru = br.graphs.begin();
            for (auto jt = br.graphs.begin(); jt != br.graphs.end(); ++jt)
                if (jt->second.last_use < lru->second.last_use) lru = jt;
            cudaGraphExecDestroy(lru->second.exec);
            br.graphs.erase(lru);
        }
        cudaGraph_t graph = nullptr;
        const unsigned long long before = ads::g_launches;
        ADS_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = group_steps(g, st, kBatchChunk, true);
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        const unsigned long long launches = ads::g_launches - before;
        ads::g_launches = before;
        if (rc != ADS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(ADS_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(ADS_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
        BatchGraph bg;
        bg.exec = ge;
        bg.launches = launches;
        it = br.graphs.emplace(key, bg).first;
    }
    it->second.last_use = ++br.clock;
    *out = &it->second;
    return ADS_OK;
}

// Advance every group by nsteps, and the other simulations (elasticity, the
// residual-corrected FP32 step) by ads_step on their own streams.  Each group
// runs on its own stream after the members' streams (pending work on any
// member) and the members' streams wait for it again, so stream order per
// simulation is kept.  Every group joins the members' streams before any
// group's completion is queued on them: members that share one stream
// (the usual case) would otherwise make each group wait for the one before,
// and the groups would run one after another instead of side by side.
int batch_groups(std::map<std::pair<int, int>, std::vector<ads_sim *>> &groups, const std::vector<ads_sim *> &others,
                 int nsteps)
{
    std::unique_lock<std::mutex> lock(batch_mutex());
    std::vector<cudaEvent_t> evs;
    auto new_event = [&](cudaEvent_t *e) -> int {
        ADS_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        evs.push_back(*e);
        return ADS_OK;
    };
    struct Cleanup {
        std::vector<cudaEvent_t> &e;
        ~Cleanup()
        {
            for (cudaEvent_t x : e) cudaEventDestroy(x);
        }
    } cleanup{evs};
    int rc;
    struct Run {
        std::vector<ads_sim *> *g;
        cudaStream_t st;
        std::vector<cudaStream_t> member_streams;
    };
    std::vector<Run> runs;
    // 1. every group's stream joins its members' streams
    for (auto &kv : groups) {
        Run r{&kv.second, nullptr, {}};
        BatchRes &br = batch_res(kv.second[0]->device);
        if ((rc = group_stream(br, kv.first.first, kv.first.second, &r.st))) return rc;
        for (ads_sim *s : kv.second)
            if (std::find(r.member_streams.begin(), r.member_streams.end(), s->stream) == r.member_streams.end())
                r.member_streams.push_back(s->stream);
        for (cudaStream_t ms : r.member_streams) {
            cudaEvent_t e;
            if ((rc = new_event(&e))) return rc;
            ADS_CK(cudaEventRecord(e, ms));
            ADS_CK(cudaStreamWaitEvent(r.st, e, 0));
        }
        runs.push_back(std::move(r));
    }
    // 2. the groups' steps
    for (Run &r : runs) {
        std::vector<ads_sim *> &g = *r.g;
        BatchRes &br = batch_res(g[0]->device);
        int left = nsteps;
        bool warmed = true;
        for (ads_sim *s : g) warmed = warmed && s->warmed;
        if (!warmed) {   // first grouped step outside capture (kernel attributes)
            if ((rc = group_steps(g, r.st, 1, left == 1))) return rc;
            for (ads_sim *s : g) s->warmed = true;
            --left;
        }
        if (left >= kBatchChunk) {
            BatchGraph *bg;
            if ((rc = batch_graph(br, g, r.st, &bg))) return rc;
            const int full = left / kBatchChunk;
            for (int i = 0; i < full; ++i) ADS_CK(cudaGraphLaunch(bg->exec, r.st));
            ads::g_launches += (unsigned long long)full * bg->launches;
            left -= full * kBatchChunk;
        }
        if (left > 0 && (rc = group_steps(g, r.st, left, true))) return rc;
        for (ads_sim *s : g) s->h_step += nsteps;
    }
    // 3. each group's completion, recorded before the lock is released (a
    // group stream is shared by every caller of the same precision and degree)
    std::vector<cudaEvent_t> done(runs.size());
    for (size_t i = 0; i < runs.size(); ++i) {
        if ((rc = new_event(&done[i]))) return rc;
        ADS_CK(cudaEventRecord(done[i], runs[i].st));
    }
    lock.unlock();
    // 4. the other simulations, queued on their own streams after the joins
    // above, so they run beside the groups (ads_step takes no batch lock)
    for (ads_sim *s : others)
        if ((rc = ads_step(s, nsteps))) return rc;
    // 5. the members' streams wait for their groups
    for (size_t i = 0; i < runs.size(); ++i)
        for (cudaStream_t ms : runs[i].member_streams) ADS_CK(cudaStreamWaitEvent(ms, done[i], 0));
    return ADS_OK;
}

// ------------------------------------------------------------------ autotuner

// K1 layouts this simulation can take: the whole plane (fused y sweep) in
// one CTA when it fits the shared-memory budget, the plane split over a
// 2-CTA cluster (FP32, when two such CTAs fit an SM), and row tiles of
// 8..64 rows with a separate y sweep.  (rows, pair)
std::vector<std::pair<int, int>> tile_candidates(const ads_sim *s)
{
    const int el = (int)elem(s);
    const int Sx = segs(s, s->d.mx), Sy = segs(s, s->d.my), my = s->d.my;
    std::vector<std::pair<int, int>> c;
    if (ads::rhs_smem_bytes(s->p, el, s->d, my, Sx, Sy, s->seg) <= 220 * 1024) c.push_back({my, 0});
    if (el == 4 && my >= 2 && Sx <= 8 && Sy <= 8 && s->seg != ads::kSegLong && ads::rhs_smem_bytes(s->p, el, s->d, my, Sx, Sy, s->seg, 1) <= 110 * 1024)
        c.push_back({my, 1});
    for (int t : {8, 16, 32, 64})
        if (t < my && ads::rhs_smem_bytes(s->p, el, s->d, t, Sx, Sy, s->seg) <= 220 * 1024) c.push_back({t, 0});
    return c;
}

struct TuneKey {
    int mx, my, mz, p, prec, kind;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(mx, my, mz, p, prec, kind) < std::tie(o.mx, o.my, o.mz, o.p, o.prec, o.kind);
    }
};

std::map<TuneKey, std::pair<int, int>> &tune_cache()
{
    static std::map<TuneKey, std::pair<int, int>> c;
    return c;
}

void set_tile(ads_sim *s, std::pair<int, int> t)
{
    const int pi = s->prec == ADS_FP64 ? 0 : 1;
    if (s->ty[pi] == t.first && s->pair[pi] == t.second) return;
    s->ty[pi] = t.first;
    s->pair[pi] = t.second;
    s->fuse[pi] = t.first == s->d.my;
    drop_graphs(s);
}

// Time each candidate tile on the simulation itself for trial_steps steps
// (after one untimed step), restoring state and step counter after every
// trial; keep the fastest.  Results are cached per (grid, p, precision,
// kind) for the process.
int autotune(ads_sim *s, int trial_steps)
{
    std::lock_guard<std::mutex> lock(batch_mutex());
    const TuneKey key{s->d.mx, s->d.my, s->d.mz, s->p, s->prec, s->kind};
    auto hit = tune_cache().find(key);
    if (hit != tune_cache().end()) {
        set_tile(s, hit->second);
        return ADS_OK;
    }
    const std::vector<std::pair<int, int>> cand = tile_candidates(s);
    if (cand.empty()) return fail(ADS_ERR_UNSUPPORTED, "ads_autotune: no tile fits shared memory");
    if (cand.size() == 1 || trial_steps == 0) {
        set_tile(s, cand[0]);
        tune_cache()[key] = cand[0];
        return ADS_OK;
    }
    // snapshot of everything a step writes
    const size_t n = (size_t)s->d.count() * elem(s);
    std::vector<std::pair<void *, size_t>> state;
    if (s->kind == ADS_SCALAR_WAVE) state = {{s->P, n}, {s->Q, n}, {s->A, n}};
    else state = {{s->U, 3 * n}, {s->Up, 3 * n}};
    state.push_back({s->d_step, sizeof(long long)});
    Scratch sc(s);
    std::vector<void *> saved;
    for (auto &st : state) {
        void *b = sc.get(st.second);
        if (!b) return fail(ADS_ERR_OOM, "ads_autotune: scratch allocation failed");
        ADS_CK(cudaMemcpyAsync(b, st.first, st.second, cudaMemcpyDeviceToDevice, s->stream));
        saved.push_back(b);
    }
    auto restore = [&]() -> int {
        for (size_t i = 0; i < state.size(); ++i)
            ADS_CK(cudaMemcpyAsync(state[i].first, saved[i], state[i].second, cudaMemcpyDeviceToDevice, s->stream));
        return ADS_OK;
    };
    cudaEvent_t e0, e1;
    ADS_CK(cudaEventCreate(&e0));
    ADS_CK(cudaEventCreate(&e1));
    const int pi = s->prec == ADS_FP64 ? 0 : 1;
    const std::pair<int, int> orig{s->ty[pi], s->pair[pi]};
    std::pair<int, int> best = cand[0];
    int rc = ADS_OK;
    float best_ms = 1e30f;
    const unsigned long long launches = ads::g_launches;
    for (const std::pair<int, int> &t : cand) {
        set_tile(s, t);
        if ((rc = step_once(s, false))) break;
        cudaEventRecord(e0, s->stream);
        for (int i = 0; i < trial_steps && rc == ADS_OK; ++i) rc = step_once(s, false);
        cudaEventRecord(e1, s->stream);
        if (rc || (rc = restore())) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(ADS_ERR_CUDA, "ads_autotune: timing failed");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    ads::g_launches = launches;   // trial launches are not part of any step
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        set_tile(s, orig);
        return rc;
    }
    if ((rc = check_device_error(s))) return rc;
    set_tile(s, best);
    tune_cache()[key] = best;
    return ADS_OK;
}

}  // namespace

// Energies of the elastic state (FP64): kinetic 1/2 rho V^T M V with
// V = (U^n - U^{n-1})/tau, potential 1/2 U^T Ups U, and the discrete
// invariant of the three-level scheme at n-1/2 (f = 0):
//   E = |V|^2_{D - tau^2 Ups/4} + |(U^n + U^{n-1})/2|^2_Ups,
//   |x|^2_D = (L^T x)^T (rho M)^{-1} (L^T x), L^T the block-upper factor.
int elastic_energy(ads_sim *s, double *kinetic, double *potential, double *kin_mod)
{
    Scratch sc(s);
    const long long cnt = s->d.count();
    const size_t b1 = (size_t)cnt * sizeof(double), b3 = 3 * b1;
    double *u = (double *)sc.get(b3), *v = (double *)sc.get(b3), *w = (double *)sc.get(b3), *z = (double *)sc.get(b3);
    double *t1 = (double *)sc.get(b1), *t2 = (double *)sc.get(b1);
    if (!u || !v || !w || !z || !t1 || !t2) return fail(ADS_ERR_OOM, "ads_energy: scratch allocation failed");
    if (s->prec == ADS_FP64)
        ADS_CK(ads::launch_el_to_uv<double>((const double *)s->U, (const double *)s->Up, u, v, 3 * cnt, s->tau,
                                            s->stream));
    else
        ADS_CK(ads::launch_el_to_uv<float>((const float *)s->U, (const float *)s->Up, u, v, 3 * cnt, s->tau,
                                           s->stream));
    auto dot3 = [&](const double *x, const double *y, double *out) { return dot64_n(s, x, y, 3 * cnt, out); };
    int rc;
    double vmv = 0, uuu = 0;
    for (int i = 0; i < 3; ++i)
        if ((rc = apply_kron64(s, s->t64.M, v + i * cnt, w + i * cnt, t1))) return rc;
    if ((rc = dot3(v, w, &vmv))) return rc;
    if ((rc = apply_upsilon<double>(s, u, w, t1, t2)) || (rc = dot3(u, w, &uuu))) return rc;
    if (kinetic) *kinetic = 0.5 * s->rho * vmv;
    if (potential) *potential = 0.5 * uuu;
    if (!kin_mod) return ADS_OK;
    // w = L^T v: rho (x)(M + d K) v_i + tau^2/2 sum_{j>i} Ups_ij v_j
    for (int i = 0; i < 3; ++i) {
        void *eb[3];
        for (int a = 0; a < 3; ++a) eb[a] = s->ebandFP64[a][a == i ? 0 : 1];
        if ((rc = apply_kron64(s, eb, v + i * cnt, w + i * cnt, t1))) return rc;
        ads::KronSum<double> ks{};
        ks.beta = s->rho;
        for (int j = i + 1; j < 3; ++j) add_offdiag<double>(s, ks, i, j, v + j * cnt, 0.5 * s->tau * s->tau);
        ADS_CK(ads::launch_kron_sum<double>(s->p, ks, w + i * cnt, s->d, s->stream));
    }
    // z = (rho M)^{-1} w
    ADS_CK(cudaMemcpyAsync(z, w, b3, cudaMemcpyDeviceToDevice, s->stream));
    for (int i = 0; i < 3; ++i)
        if ((rc = kron_solve64(s, z + i * cnt, SET_MASS))) return rc;
    double wz = 0, vuv = 0, aua = 0;
    if ((rc = dot3(w, z, &wz))) return rc;
    wz /= s->rho;
    if ((rc = apply_upsilon<double>(s, v, z, t1, t2)) || (rc = dot3(v, z, &vuv))) return rc;
    // average (U^n + U^{n-1})/2 = u - tau/2 v
    ADS_CK(ads::launch_lincomb<double>(w, 1.0, u, -0.5 * s->tau, v, 3 * cnt, s->stream));
    if ((rc = apply_upsilon<double>(s, w, z, t1, t2)) || (rc = dot3(w, z, &aua))) return rc;
    *kin_mod = wz - 0.25 * s->tau * s->tau * vuv + aua;
    return ADS_OK;
}

// ====================================================================== ABI

extern "C" {

const char *ads_last_error(void) { return g_err.c_str(); }

long long ads_launch_count(void) { return (long long)ads::g_launches; }

int ads_create(const ads_grid_t *grid, int p, double tau, const ads_material_t *mat, const ads_options_t *opts,
               ads_sim_t **out)
{
    if (!grid || !mat || !out) return fail(ADS_ERR_INVALID_ARG, "ads_create: null argument");
    *out = nullptr;
    if (p < 1 || p > 4) return fail(ADS_ERR_UNSUPPORTED, "ads_create: p must be in 1..4");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(ADS_ERR_INVALID_ARG, "ads_create: tau must be > 0");
    if (mat->kind != ADS_SCALAR_WAVE && mat->kind != ADS_ELASTIC)
        return fail(ADS_ERR_INVALID_ARG, "ads_create: unknown material kind");
    if (mat->kind == ADS_SCALAR_WAVE && !(mat->c2 > 0.0)) return fail(ADS_ERR_INVALID_ARG, "ads_create: c2 must be > 0");
    if (mat->kind == ADS_ELASTIC && !(mat->mu > 0.0 && mat->rho > 0.0 && mat->lambda >= 0.0))
        return fail(ADS_ERR_INVALID_ARG, "ads_create: elasticity needs mu > 0, rho > 0, lambda >= 0");
    if (grid->boundary != ADS_DIRICHLET && grid->boundary != ADS_NATURAL)
        return fail(ADS_ERR_INVALID_ARG, "ads_create: boundary must be ADS_DIRICHLET or ADS_NATURAL");
    const int drop = grid->boundary == ADS_NATURAL ? 0 : 2;
    const bool plane2d = grid->n_elem[2] == 0;   // a 2D problem on [0,Lx] x [0,Ly]
    for (int a = 0; a < (plane2d ? 2 : 3); ++a) {
        if (grid->n_elem[a] < 1) return fail(ADS_ERR_INVALID_ARG, "ads_create: n_elem must be >= 1");
        if (!(grid->length[a] > 0.0)) return fail(ADS_ERR_INVALID_ARG, "ads_create: length must be > 0");
        if (grid->n_elem[a] + p - drop < 1) return fail(ADS_ERR_INVALID_ARG, "ads_create: no interior basis function");
        if (grid->n_elem[a] + p - drop > 512)
            return fail(ADS_ERR_UNSUPPORTED, "ads_create: more than 512 unknowns per axis");
    }
    ads_options_t o{};
    o.precision = ADS_FP64;
    o.device = -1;
    if (opts) o = *opts;
    if (o.precision != ADS_FP64 && o.precision != ADS_FP32) return fail(ADS_ERR_INVALID_ARG, "ads_create: precision");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(ADS_ERR_INVALID_ARG, "ads_create: alloc and free go together");

    ads_sim *s = new (std::nothrow) ads_sim();
    if (!s) return fail(ADS_ERR_OOM, "ads_create: host allocation failed");
    s->kind = mat->kind;
    s->prec = o.precision;
    s->p = p;
    s->tau = tau;
    s->c2 = mat->kind == ADS_ELASTIC ? 1.0 : mat->c2;
    s->lam = mat->lambda;
    s->mu = mat->mu;
    s->rho = mat->rho;
    s->alloc = o.alloc;
    s->dfree = o.free;
    s->actx = o.alloc_ctx;
    s->refine = o.residual_correction != 0 && mat->kind == ADS_SCALAR_WAVE && o.precision == ADS_FP32;
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) {
            delete s;
            return fail(ADS_ERR_CUDA, "ads_create: no CUDA device");
        }
    }
    s->device = dev;
    if (cudaSetDevice(dev) != cudaSuccess) {
        delete s;
        return fail(ADS_ERR_CUDA, "ads_create: cudaSetDevice failed");
    }
    if (o.stream) {
        s->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return fail(ADS_ERR_CUDA, "ads_create: stream creation failed");
        }
        s->own_stream = true;
    }
    try {
        for (int a = 0; a < 3; ++a)
            s->ax[a] = (a == 2 && plane2d) ? ads::trivial_axis(p)
                                           : ads::build_axis(grid->n_elem[a], p, grid->length[a],
                                                             grid->boundary == ADS_NATURAL);
    } catch (const std::exception &e) {
        ads_destroy(s);
        return fail(ADS_ERR_INVALID_ARG, e.what());
    }
    s->d.mx = s->ax[0].m;
    s->d.my = s->ax[1].m;
    s->d.mz = s->ax[2].m;
    s->d.sx = (s->d.mx + 7) / 8 * 8;
    s->d.off = grid->boundary == ADS_NATURAL ? 0 : 1;
    s->d.offz = plane2d ? 0 : s->d.off;
    // elasticity with the Dirichlet restriction takes the fused step (its
    // off-diagonal blocks are single Kronecker terms); the natural boundary
    // keeps the step through the Kronecker-sum kernel
    s->fused_el = s->kind == ADS_ELASTIC && s->d.off == 1;
    if (const char *env = std::getenv("ADS_ELASTIC_STEP"))   // "kron": the unfused step, for comparisons
        if (std::strcmp(env, "kron") == 0) s->fused_el = false;
    {
        const int m3[3] = {s->d.mx, s->d.my, s->d.mz};
        // 33-row segments when they save segments (m = 32 s + 1), 44 when they save K1 rounds
        s->seg = ads::choose_seg(m3, s->prec == ADS_FP64 ? 8 : 4);
    }
    choose_tiles(s);
    if (o.tile_lines > 0) {
        // user override of the tile height (rows of one z-plane per CTA)
        const int pi = s->prec == ADS_FP64 ? 0 : 1;
        s->ty[pi] = std::min(s->d.my, o.tile_lines);
        s->fuse[pi] = s->ty[pi] == s->d.my;
    }
    int rc = build_tables<double>(s, s->t64);
    if (rc == ADS_OK && s->prec == ADS_FP32) rc = build_tables<float>(s, s->t32);
    if (rc != ADS_OK) {
        std::string msg = g_err;
        ads_destroy(s);
        return fail(rc, msg);
    }
    const size_t n = (size_t)s->d.count() * elem(s);
    s->d_step = (long long *)dalloc(s, sizeof(long long));
    s->d_err = (int *)dalloc(s, sizeof(int));
    bool ok = s->d_step && s->d_err;
    if (s->kind == ADS_SCALAR_WAVE) {
        s->P = dalloc(s, n);
        s->Q = dalloc(s, n);
        s->A = dalloc(s, n);
        s->X = dalloc(s, n);
        ok = ok && s->P && s->Q && s->A && s->X;
        if (ok && s->refine) {
            const size_t n64 = (size_t)s->d.count() * sizeof(double);
            s->R64 = dalloc(s, n64);
            s->P64 = dalloc(s, n64);
            s->A64 = dalloc(s, n64);
            s->T64 = dalloc(s, n64);
            ok = s->R64 && s->P64 && s->A64 && s->T64;
        }
    } else {
        s->U = dalloc(s, 3 * n);
        s->Up = dalloc(s, 3 * n);
        s->R = dalloc(s, 3 * n);
        s->Y = dalloc(s, 3 * n);
        ok = ok && s->U && s->Up && s->R && s->Y;
        // bands of M + d K for the discrete invariant (FP64)
        for (int a = 0; a < 3 && ok; ++a)
            for (int k = 0; k < 2 && ok; ++k) {
                const ads::Axis1D &ax = s->ax[a];
                const double c = k == 0 ? 2 * s->mu + s->lam : s->mu;
                const double dd = s->tau * s->tau * c / (4 * s->rho);
                std::vector<double> g(ax.M.v.size());
                for (size_t i = 0; i < g.size(); ++i) g[i] = ax.M.v[i] + dd * ax.K.v[i];
                ok = upload<double>(s, pad_rows(g, ax.m, 2 * ax.p + 1, padded(s, ax.m), false), &s->ebandFP64[a][k]) ==
                     ADS_OK;
            }
    }
    if (!ok) {
        ads_destroy(s);
        return fail(ADS_ERR_OOM, "ads_create: device allocation of the state failed");
    }
    for (void *q : {s->P, s->Q, s->A, s->X, s->U, s->Up, s->R, s->Y})
        if (q) cudaMemsetAsync(q, 0, q == s->U || q == s->Up || q == s->R || q == s->Y ? 3 * n : n, s->stream);
    cudaMemsetAsync(s->d_step, 0, sizeof(long long), s->stream);
    cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    static std::atomic<unsigned long long> next_uid{0};
    s->uid = ++next_uid;
    if (s->kind == ADS_SCALAR_WAVE)
        s->has_maps = ads::make_update_maps(&s->upd_maps, s->P, s->Q, (int)elem(s), s->d, 2);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        ads_destroy(s);
        return fail(ADS_ERR_CUDA, "ads_create: initialisation failed");
    }
    *out = s;
    return ADS_OK;
}

void ads_destroy(ads_sim_t *s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->uid) forget_batch_graphs(s);
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    std::vector<void *> ptrs;
    for (auto &kv : s->live) ptrs.push_back(kv.first);
    for (void *p : ptrs) dfree(s, p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int ads_dims(const ads_sim_t *s, int *n, int *comps)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_dims: null sim");
    if (n) {
        n[0] = s->d.mx + 2 * s->d.off;
        n[1] = s->d.my + 2 * s->d.off;
        n[2] = s->d.mz + 2 * s->d.offz;
    }
    if (comps) *comps = s->kind == ADS_ELASTIC ? 3 : 1;
    return ADS_OK;
}

int ads_set_source(ads_sim_t *s, const ads_source_t *src)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_set_source: null sim");
    cudaSetDevice(s->device);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(ADS_ERR_CUDA, "ads_set_source: stream error");
    for (TableSet *ts : {&s->t64, &s->t32}) {
        for (int a = 0; a < 3; ++a) {
            dfree(s, ts->src[a]);
            ts->src[a] = nullptr;
        }
        dfree(s, ts->srcfield);
        ts->srcfield = nullptr;
    }
    s->has_src = false;
    for (int a = 0; a < 3; ++a) s->hsrc[a].clear();
    if (!src) return rebuild_images(s);
    if (!(src->shape.den > 0.0)) return fail(ADS_ERR_INVALID_ARG, "ads_set_source: den must be > 0");
    s->src = *src;
    for (int a = 0; a < 3; ++a) {
        std::vector<double> g = ads::gaussian_load(s->ax[a], src->shape.center[a], src->shape.den);
        if (a == 0)
            for (double &v : g) v *= src->shape.amp;
        g.resize(padded(s, s->ax[a].m), 0.0);   // padded like every 1D table
        s->hsrc[a] = g;
        int rc = upload<double>(s, g, &s->t64.src[a]);
        if (rc) return rc;
        if (s->prec == ADS_FP32 && (rc = upload<float>(s, g, &s->t32.src[a]))) return rc;
    }
    s->has_src = true;
    return rebuild_images(s);
}

int ads_set_source_field(ads_sim_t *s, const double *g, size_t count, int mem, const double *dir, double freq,
                         double t0)
{
    if (!s || !g) return fail(ADS_ERR_INVALID_ARG, "ads_set_source_field: null argument");
    if (mem != ADS_HOST && mem != ADS_DEVICE) return fail(ADS_ERR_INVALID_ARG, "ads_set_source_field: mem");
    const size_t nf = full_count(s) / (s->kind == ADS_ELASTIC ? 3 : 1);
    if (count != nf) return fail(ADS_ERR_INVALID_ARG, "ads_set_source_field: count must be n0*n1*n2");
    if (!std::isfinite(freq) || !std::isfinite(t0)) return fail(ADS_ERR_INVALID_ARG, "ads_set_source_field: freq, t0");
    int rc = ads_set_source(s, nullptr);   // drop any previous source
    if (rc) return rc;
    Scratch sc(s);
    const size_t ni = (size_t)s->d.count() * sizeof(double);
    void *f64 = dalloc(s, ni);
    if (!f64) return fail(ADS_ERR_OOM, "ads_set_source_field: device allocation failed");
    s->t64.srcfield = f64;
    if ((rc = stage_in(s, sc, g, mem, count, (double *)f64, 1.0))) return rc;
    if (s->prec == ADS_FP32) {
        void *f32 = dalloc(s, (size_t)s->d.count() * sizeof(float));
        if (!f32) return fail(ADS_ERR_OOM, "ads_set_source_field: device allocation failed");
        s->t32.srcfield = f32;
        ADS_CK(ads::launch_convert_from<float>((const double *)f64, (float *)f32, s->d.count(), s->stream));
    }
    ADS_CK(cudaStreamSynchronize(s->stream));
    std::memset(&s->src, 0, sizeof(s->src));
    s->src.shape.amp = 1.0;
    if (dir)
        for (int i = 0; i < 3; ++i) s->src.shape.dir[i] = dir[i];
    s->src.freq = freq;
    s->src.t0 = t0;
    s->has_src = true;
    return rebuild_images(s);
}

int ads_set_state(ads_sim_t *s, const double *u, const double *v, const double *a, size_t count, int mem)
{
    if (!s || !u || !v) return fail(ADS_ERR_INVALID_ARG, "ads_set_state: null argument");
    if (count != full_count(s)) return fail(ADS_ERR_INVALID_ARG, "ads_set_state: count does not match the space");
    if (mem != ADS_HOST && mem != ADS_DEVICE) return fail(ADS_ERR_INVALID_ARG, "ads_set_state: mem");
    if (s->kind == ADS_ELASTIC && a) return fail(ADS_ERR_INVALID_ARG, "ads_set_state: elasticity takes u and v only");
    cudaSetDevice(s->device);
    Scratch sc(s);
    const int comps = s->kind == ADS_ELASTIC ? 3 : 1;
    const size_t ncomp = count / comps;
    const size_t ni = (size_t)s->d.count() * sizeof(double);
    double *tu = (double *)sc.get(comps * ni), *tv = (double *)sc.get(comps * ni), *ta = (double *)sc.get(ni);
    if (!tu || !tv || !ta) return fail(ADS_ERR_OOM, "ads_set_state: scratch allocation failed");
    int rc;
    for (int c = 0; c < comps; ++c) {
        const size_t io = (size_t)c * s->d.count();
        if ((rc = stage_in(s, sc, u + c * ncomp, mem, ncomp, tu + io, 1.0))) return rc;
        if ((rc = stage_in(s, sc, v + c * ncomp, mem, ncomp, tv + io, 1.0))) return rc;
    }
    ADS_CK(cudaMemcpyAsync(s->d_step, &s->h_step, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    if (s->kind == ADS_ELASTIC) {
        if ((rc = elastic_set64(s, sc, tu, tv))) return rc;
        ADS_CK(cudaStreamSynchronize(s->stream));
        return ADS_OK;
    }
    if (a) {
        if ((rc = stage_in(s, sc, a, mem, count, ta, 1.0))) return rc;
    } else {
        if ((rc = consistent_accel64(s, tu, ta))) return rc;
    }
    rc = s->prec == ADS_FP64 ? set_pq<double>(s, tu, tv, ta) : set_pq<float>(s, tu, tv, ta);
    if (rc) return rc;
    ADS_CK(cudaStreamSynchronize(s->stream));
    return ADS_OK;
}

int ads_set_gaussian_state(ads_sim_t *s, const ads_gaussian_t *u0, const ads_gaussian_t *v0)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_set_gaussian_state: null sim");
    cudaSetDevice(s->device);
    Scratch sc(s);
    const int comps = s->kind == ADS_ELASTIC ? 3 : 1;
    const long long cnt = s->d.count();
    const size_t ni = (size_t)cnt * sizeof(double);
    double *tu = (double *)sc.get(comps * ni), *tv = (double *)sc.get(comps * ni), *ta = (double *)sc.get(ni);
    if (!tu || !tv || !ta) return fail(ADS_ERR_OOM, "ads_set_gaussian_state: scratch allocation failed");
    const ads_gaussian_t *gs[2] = {u0, v0};
    double *dst[2] = {tu, tv};
    for (int f = 0; f < 2; ++f) {
        ADS_CK(cudaMemsetAsync(dst[f], 0, comps * ni, s->stream));
        if (!gs[f]) continue;
        if (!(gs[f]->den > 0.0)) return fail(ADS_ERR_INVALID_ARG, "ads_set_gaussian_state: den must be > 0");
        // separable: projection = (Mx^-1 gx) (x) (My^-1 gy) (x) (Mz^-1 gz), done
        // on the device as the outer product of the loads and a mass solve
        void *g[3];
        for (int a = 0; a < 3; ++a) {
            std::vector<double> h = ads::gaussian_load(s->ax[a], gs[f]->center[a], gs[f]->den);
            g[a] = sc.get(h.size() * sizeof(double));
            if (!g[a]) return fail(ADS_ERR_OOM, "scratch allocation failed");
            ADS_CK(cudaMemcpyAsync(g[a], h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream));
            ADS_CK(cudaStreamSynchronize(s->stream));
        }
        for (int c = 0; c < comps; ++c) {
            const double amp = gs[f]->amp * (comps == 3 ? gs[f]->dir[c] : 1.0);
            if (amp == 0.0) continue;
            double *dc = dst[f] + (size_t)c * cnt;
            ADS_CK(ads::launch_outer((const double *)g[0], (const double *)g[1], (const double *)g[2], amp, dc, s->d,
                                     s->stream));
            int rc = kron_solve64(s, dc, SET_MASS);
            if (rc) return rc;
        }
    }
    s->h_step = 0;
    ADS_CK(cudaMemsetAsync(s->d_step, 0, sizeof(long long), s->stream));
    int rc;
    if (s->kind == ADS_ELASTIC) {
        if ((rc = elastic_set64(s, sc, tu, tv))) return rc;
        ADS_CK(cudaStreamSynchronize(s->stream));
        return ADS_OK;
    }
    if ((rc = consistent_accel64(s, tu, ta))) return rc;
    rc = s->prec == ADS_FP64 ? set_pq<double>(s, tu, tv, ta) : set_pq<float>(s, tu, tv, ta);
    if (rc) return rc;
    ADS_CK(cudaStreamSynchronize(s->stream));
    return ADS_OK;
}

int ads_get_state(ads_sim_t *s, double *u, double *v, double *a, size_t count, int mem)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_get_state: null sim");
    if (count != full_count(s)) return fail(ADS_ERR_INVALID_ARG, "ads_get_state: count does not match the space");
    if (mem != ADS_HOST && mem != ADS_DEVICE) return fail(ADS_ERR_INVALID_ARG, "ads_get_state: mem");
    if (s->kind == ADS_ELASTIC && a) return fail(ADS_ERR_INVALID_ARG, "ads_get_state: elasticity returns u and v only");
    cudaSetDevice(s->device);
    Scratch sc(s);
    const int comps = s->kind == ADS_ELASTIC ? 3 : 1;
    const long long cnt = s->d.count();
    const size_t ni = (size_t)cnt * sizeof(double);
    double *tu = (double *)sc.get(comps * ni), *tv = (double *)sc.get(comps * ni), *ta = (double *)sc.get(ni);
    if (!tu || !tv || !ta) return fail(ADS_ERR_OOM, "ads_get_state: scratch allocation failed");
    int rc;
    if (s->kind == ADS_ELASTIC) {
        if (s->prec == ADS_FP64)
            ADS_CK(ads::launch_el_to_uv<double>((const double *)s->U, (const double *)s->Up, tu, tv, 3 * cnt, s->tau,
                                                s->stream));
        else
            ADS_CK(ads::launch_el_to_uv<float>((const float *)s->U, (const float *)s->Up, tu, tv, 3 * cnt, s->tau,
                                               s->stream));
    } else {
        rc = s->prec == ADS_FP64 ? get_uva<double>(s, tu, tv, ta) : get_uva<float>(s, tu, tv, ta);
        if (rc) return rc;
    }
    const size_t ncomp = count / comps;
    double *outs[3] = {u, v, a};
    double *ins[3] = {tu, tv, ta};
    for (int f = 0; f < 3; ++f) {
        if (!outs[f]) continue;
        for (int c = 0; c < comps; ++c)
            if ((rc = stage_out(s, sc, ins[f] + (size_t)c * cnt, outs[f] + c * ncomp, mem, ncomp))) return rc;
    }
    ADS_CK(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

int ads_step(ads_sim_t *s, int nsteps)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_step: null sim");
    if (nsteps < 0) return fail(ADS_ERR_INVALID_ARG, "ads_step: nsteps < 0");
    if (nsteps == 0) return ADS_OK;
    cudaSetDevice(s->device);
    int rc;
    if (!s->warmed) {
        // first launch outside capture (sets kernel attributes)
        if ((rc = step_once(s, nsteps == 1))) return rc;
        s->warmed = true;
        s->h_step += 1;
        --nsteps;
        if (nsteps == 0) return ADS_OK;
    }
    const int chunk = 16;
    if (nsteps >= chunk) {
        cudaGraphExec_t ge;
        if ((rc = get_graph(s, chunk, &ge))) return rc;
        const int full = nsteps / chunk;
        for (int i = 0; i < full; ++i) ADS_CK(cudaGraphLaunch(ge, s->stream));
        ads::g_launches += (unsigned long long)full * s->graph_launches[chunk];
        nsteps -= full * chunk;
        s->h_step += (long long)full * chunk;
    }
    if (nsteps > 0) {
        cudaGraphExec_t ge;
        if ((rc = get_graph(s, nsteps, &ge))) return rc;
        ADS_CK(cudaGraphLaunch(ge, s->stream));
        ads::g_launches += s->graph_launches[nsteps];
        s->h_step += nsteps;
    }
    return ADS_OK;
}

int ads_batch_step(ads_sim_t *const *sims, int count, int nsteps)
{
    if (!sims || count < 0 || nsteps < 0) return fail(ADS_ERR_INVALID_ARG, "ads_batch_step: bad arguments");
    if (count == 0 || nsteps == 0) return ADS_OK;
    for (int i = 0; i < count; ++i) {
        if (!sims[i]) return fail(ADS_ERR_INVALID_ARG, "ads_batch_step: null simulation");
        if (sims[i]->device != sims[0]->device) return fail(ADS_ERR_INVALID_ARG, "ads_batch_step: mixed devices");
        for (int j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return fail(ADS_ERR_INVALID_ARG, "ads_batch_step: a simulation appears twice");
    }
    cudaSetDevice(sims[0]->device);
    // scalar-wave simulations share grouped launches per (precision, degree);
    // elasticity (and the residual-corrected FP32 step) advances on each
    // simulation's own stream meanwhile
    std::map<std::pair<int, int>, std::vector<ads_sim *>> groups;
    std::vector<ads_sim *> others;
    for (int i = 0; i < count; ++i) {
        ads_sim *s = sims[i];
        if (s->kind == ADS_SCALAR_WAVE && !s->refine) groups[{s->prec, s->p}].push_back(s);
        else others.push_back(s);
    }
    return batch_groups(groups, others, nsteps);
}

int ads_selftest_timeout(int device, long long cycles)
{
    if (cycles < 1 || cycles > 4000000000LL) return fail(ADS_ERR_INVALID_ARG, "ads_selftest_timeout: cycles");
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) return fail(ADS_ERR_CUDA, "no CUDA device");
    ADS_CK(cudaSetDevice(device));
    int *err = nullptr;
    ADS_CK(cudaMalloc(&err, 2 * sizeof(int)));
    int h[2] = {0, 0};
    cudaError_t e = cudaMemset(err, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = ads::launch_wait_selftest(cycles, err, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, err, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return fail(ADS_ERR_CUDA, std::string("ads_selftest_timeout: ") + cudaGetErrorString(e));
    if (h[0] == ads::kDevErrTimeout) return fail(ADS_ERR_TIMEOUT, "self-test: the bounded device wait ran out");
    return ADS_OK;
}

int ads_autotune(ads_sim_t *s, int trial_steps, int *tile_rows)
{
    if (!s || trial_steps < 0) return fail(ADS_ERR_INVALID_ARG, "ads_autotune: bad arguments");
    cudaSetDevice(s->device);
    int rc = autotune(s, trial_steps);
    if (rc) return rc;
    const int pi = s->prec == ADS_FP64 ? 0 : 1;
    // a pair reports the rows of its larger CTA (the split is a multiple of 32)
    int cut = ((s->d.my / 2) + 31) & ~31;
    if (cut > s->d.my) cut = s->d.my;
    if (tile_rows) *tile_rows = s->pair[pi] ? std::max(cut, s->d.my - cut) : s->ty[pi];
    return ADS_OK;
}

int ads_sync(ads_sim_t *s)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_sync: null sim");
    cudaSetDevice(s->device);
    ADS_CK(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

int ads_get_step(const ads_sim_t *s, long long *n)
{
    if (!s || !n) return fail(ADS_ERR_INVALID_ARG, "ads_get_step: null argument");
    *n = s->h_step;
    return ADS_OK;
}

int ads_energy(ads_sim_t *s, double *kinetic, double *potential, double *kin_mod)
{
    if (!s) return fail(ADS_ERR_INVALID_ARG, "ads_energy: null sim");
    cudaSetDevice(s->device);
    if (s->kind == ADS_ELASTIC) return elastic_energy(s, kinetic, potential, kin_mod);
    Scratch sc(s);
    const size_t ni = (size_t)s->d.count() * sizeof(double);
    double *u = (double *)sc.get(ni), *v = (double *)sc.get(ni), *w = (double *)sc.get(ni), *t = (double *)sc.get(ni);
    if (!u || !v || !w || !t) return fail(ADS_ERR_OOM, "ads_energy: scratch allocation failed");
    int rc = s->prec == ADS_FP64 ? get_uva<double>(s, u, v, nullptr) : get_uva<float>(s, u, v, nullptr);
    if (rc) return rc;
    double vmv = 0, uku = 0, vgv = 0, vkv = 0;
    if ((rc = apply_kron64(s, s->t64.M, v, w, t)) || (rc = dot64(s, v, w, &vmv))) return rc;
    if ((rc = apply_stiff64(s, u, w)) || (rc = dot64(s, u, w, &uku))) return rc;
    if (kin_mod) {
        if ((rc = apply_kron64(s, s->t64.gband, v, w, t)) || (rc = dot64(s, v, w, &vgv))) return rc;
        if ((rc = apply_stiff64(s, v, w)) || (rc = dot64(s, v, w, &vkv))) return rc;
        *kin_mod = 0.5 * (vgv - 0.25 * s->tau * s->tau * vkv);
    }
    if (kinetic) *kinetic = 0.5 * vmv;
    if (potential) *potential = 0.5 * uku;
    return ADS_OK;
}

int ads_apply(ads_sim_t *s, int op, const double *in, double *out, size_t count, int mem)
{
    if (!s || !in || !out) return fail(ADS_ERR_INVALID_ARG, "ads_apply: null argument");
    const size_t nf = full_count(s) / (s->kind == ADS_ELASTIC ? 3 : 1);
    if (count != nf) return fail(ADS_ERR_INVALID_ARG, "ads_apply: count must be n0*n1*n2");
    if (mem != ADS_HOST && mem != ADS_DEVICE) return fail(ADS_ERR_INVALID_ARG, "ads_apply: mem");
    if (op == ADS_OP_SPLIT_SOLVE && s->kind != ADS_SCALAR_WAVE)
        return fail(ADS_ERR_INVALID_ARG, "ads_apply: split solve is defined for the scalar wave");
    cudaSetDevice(s->device);
    Scratch sc(s);
    const size_t ni = (size_t)s->d.count() * sizeof(double);
    double *x = (double *)sc.get(ni), *y = (double *)sc.get(ni), *t = (double *)sc.get(ni);
    if (!x || !y || !t) return fail(ADS_ERR_OOM, "ads_apply: scratch allocation failed");
    int rc = stage_in(s, sc, in, mem, count, x, 1.0);
    if (rc) return rc;
    switch (op) {
    case ADS_OP_MASS: rc = apply_kron64(s, s->t64.M, x, y, t); break;
    case ADS_OP_STIFF: rc = apply_stiff64(s, x, y); break;
    case ADS_OP_MASS_SOLVE: rc = kron_solve64(s, x, SET_MASS); y = x; break;
    case ADS_OP_SPLIT_SOLVE: rc = kron_solve64(s, x, SET_SPLIT); y = x; break;
    default: return fail(ADS_ERR_INVALID_ARG, "ads_apply: unknown op");
    }
    if (rc) return rc;
    if ((rc = stage_out(s, sc, y, out, mem, count))) return rc;
    ADS_CK(cudaStreamSynchronize(s->stream));
    return ADS_OK;
}

// raw state arrays of the simulation: scalar wave p, q, a; elasticity U^n, U^{n-1}
static int state_arrays(ads_sim_t *s, void **arr, size_t *bytes)
{
    const size_t n = (size_t)s->d.count() * elem(s);
    if (s->kind == ADS_ELASTIC) {
        arr[0] = s->U;
        arr[1] = s->Up;
        bytes[0] = bytes[1] = 3 * n;
        return 2;
    }
    arr[0] = s->P;
    arr[1] = s->Q;
    arr[2] = s->A;
    bytes[0] = bytes[1] = bytes[2] = n;
    return 3;
}

size_t ads_checkpoint_bytes(const ads_sim_t *s)
{
    if (!s) return 0;
    void *arr[3];
    size_t b[3], tot = sizeof(long long);
    const int k = state_arrays(const_cast<ads_sim_t *>(s), arr, b);
    for (int i = 0; i < k; ++i) tot += b[i];
    return tot;
}

int ads_checkpoint_save(ads_sim_t *s, void *host, size_t bytes)
{
    if (!s || !host || bytes != ads_checkpoint_bytes(s)) return fail(ADS_ERR_INVALID_ARG, "ads_checkpoint_save: bad arguments");
    cudaSetDevice(s->device);
    void *arr[3];
    size_t b[3];
    const int k = state_arrays(s, arr, b);
    char *h = (char *)host;
    for (int i = 0; i < k; ++i) {
        ADS_CK(cudaMemcpyAsync(h, arr[i], b[i], cudaMemcpyDeviceToHost, s->stream));
        h += b[i];
    }
    ADS_CK(cudaStreamSynchronize(s->stream));
    std::memcpy(h, &s->h_step, sizeof(long long));
    return ADS_OK;
}

int ads_checkpoint_load(ads_sim_t *s, const void *host, size_t bytes)
{
    if (!s || !host || bytes != ads_checkpoint_bytes(s)) return fail(ADS_ERR_INVALID_ARG, "ads_checkpoint_load: bad arguments");
    cudaSetDevice(s->device);
    void *arr[3];
    size_t b[3];
    const int k = state_arrays(s, arr, b);
    const char *h = (const char *)host;
    for (int i = 0; i < k; ++i) {
        ADS_CK(cudaMemcpyAsync(arr[i], h, b[i], cudaMemcpyHostToDevice, s->stream));
        h += b[i];
    }
    std::memcpy(&s->h_step, h, sizeof(long long));
    ADS_CK(cudaMemcpyAsync(s->d_step, &s->h_step, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    ADS_CK(cudaStreamSynchronize(s->stream));
    return ADS_OK;
}

size_t ads_device_bytes(const ads_sim_t *s) { return s ? s->bytes : 0; }

size_t ads_estimate_bytes(const ads_grid_t *grid, int p, int kind, int precision)
{
    if (!grid || p < 1 || p > 4 || (kind != ADS_SCALAR_WAVE && kind != ADS_ELASTIC) ||
        (precision != ADS_FP64 && precision != ADS_FP32))
        return 0;
    size_t m[3], mp[3], S[3];
    int mi[3];
    for (int a = 0; a < 3; ++a) {
        long long me = (long long)grid->n_elem[a] + p - (grid->boundary == ADS_NATURAL ? 0 : 2);
        if (a == 2 && grid->n_elem[2] == 0) me = 1;   // 2D
        else if (grid->n_elem[a] < 1 || me < 1 || me > (1 << 20)) return 0;
        m[a] = (size_t)me;
        mi[a] = (int)me;
    }
    const int seg = ads::choose_seg(mi, precision == ADS_FP64 ? 8 : 4);
    for (int a = 0; a < 3; ++a) {
        S[a] = (m[a] + seg - 1) / seg;
        mp[a] = S[a] * seg;
    }
    const size_t W = 2 * (size_t)p + 1, el = precision == ADS_FP64 ? 8 : 4;
    const size_t cnt = (m[0] + 7) / 8 * 8 * m[1] * m[2];
    size_t b = 0;
    // every allocation rounded up as a caching allocator would (512 B, 2 MiB above 1 MiB)
    auto add = [&](size_t x) { b += x > (1u << 20) ? (x + (2u << 20) - 1) / (2u << 20) * (2u << 20) : (x + 511) / 512 * 512; };
    add(sizeof(long long));
    add(sizeof(int));
    if (kind == ADS_SCALAR_WAVE) {
        for (int i = 0; i < 4; ++i) add(cnt * el);
    } else {
        for (int i = 0; i < 4; ++i) add(3 * cnt * el);
        for (int a = 0; a < 3; ++a) add(2 * mp[a] * W * 8);
    }
    const int nsets = kind == ADS_SCALAR_WAVE ? 3 : 4;
    for (int t = 0; t < (precision == ADS_FP32 ? 2 : 1); ++t) {
        const size_t e = t == 0 ? 8 : 4;
        for (int a = 0; a < 3; ++a) {
            add(3 * mp[a] * W * e + 64);                                    // M, K, B
            if (grid->boundary == ADS_NATURAL) add(mp[a] * W * e);          // B^T
            for (int k = 0; k < nsets; ++k) add(ads::line_image_elems(p, (int)S[a], seg) * e + 64);
            add(mp[a] * W * e);                                             // bands of M + eta K
            add(mp[a] * e);                                                 // source load vector
        }
        const int nimg = nsets + (kind == ADS_ELASTIC ? 3 : 0);   // per-set images + mixed elastic images
        for (int k = 0; k < nimg; ++k)
            add(2 * (mp[0] + mp[1]) * W * e + (mp[0] + mp[1]) * e +
                (ads::line_image_elems(p, (int)S[0], seg) + ads::line_image_elems(p, (int)S[1], seg)) * e + 64);
        if (kind == ADS_ELASTIC && grid->boundary != ADS_NATURAL) {
            // fused step: six elastic K1 images (with Bx)
            for (int k = 0; k < 6; ++k)
                add((3 * mp[0] + 2 * mp[1]) * W * e + (mp[0] + mp[1]) * e +
                    (ads::line_image_elems(p, (int)S[0], seg) + ads::line_image_elems(p, (int)S[1], seg)) * e + 64);
        }
    }
    return b;
}

}  // extern "C"

size_t ads_internal_interior_count(const ads_sim_t *s) { return s ? (size_t)s->d.count() : 0; }

int ads_internal_sim_device(const ads_sim_t *s) { return s ? s->device : 0; }

int ads_internal_fail(int code, const char *msg) { return fail(code, msg); }

int ads_internal_apply_scratch(ads_sim_t *s, int op, const double *in, double *out, size_t count, double *s0,
                               double *s1)
{
    if (!s || !in || !out || !s0 || !s1) return fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: null argument");
    const size_t nf = full_count(s) / (s->kind == ADS_ELASTIC ? 3 : 1);
    if (count != nf) return fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: count must be n0*n1*n2");
    if (op == ADS_OP_SPLIT_SOLVE && s->kind != ADS_SCALAR_WAVE)
        return fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: split solve is defined for the scalar wave");
    // (the caller has made the simulation's device current)
    // interior scratch starts from zero (padding columns are read as zeros)
    ADS_CK(cudaMemsetAsync(s0, 0, (size_t)s->d.count() * sizeof(double), s->stream));
    ADS_CK(cudaMemsetAsync(s1, 0, (size_t)s->d.count() * sizeof(double), s->stream));
    ADS_CK(ads::launch_pack<double>(in, s0, s->d, 1.0, s->stream));
    int rc;
    double *res = s1;
    switch (op) {
    case ADS_OP_MASS:
        // s0 -> s1 -> s0 -> s1 along x, y, z
        ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)s->t64.M[0], 0, s0, s1, s->d, 1.0, 0.0, 0, s->stream));
        ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)s->t64.M[1], 1, s1, s0, s->d, 1.0, 0.0, 0, s->stream));
        ADS_CK(ads::launch_axis_apply<double>(s->p, (const double *)s->t64.M[2], 2, s0, s1, s->d, 1.0, 0.0, 0, s->stream));
        rc = ADS_OK;
        break;
    case ADS_OP_STIFF: rc = apply_stiff64(s, s0, s1); break;
    case ADS_OP_MASS_SOLVE: rc = kron_solve64(s, s0, SET_MASS); res = s0; break;
    case ADS_OP_SPLIT_SOLVE: rc = kron_solve64(s, s0, SET_SPLIT); res = s0; break;
    default: return fail(ADS_ERR_INVALID_ARG, "ads_apply_noalloc: unknown op");
    }
    if (rc) return rc;
    ADS_CK(ads::launch_unpack<double>(res, out, s->d, s->stream));
    ADS_CK(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

extern "C" {

int ads_profile_step(ads_sim_t *s, const char **names, float *ms, int cap, int *count)
{
    if (!s || !count || cap < 0) return fail(ADS_ERR_INVALID_ARG, "ads_profile_step: bad arguments");
    cudaSetDevice(s->device);
    KernelTimer kt;
    int rc;
    // the stream sleeps while the step and its events are queued, so every
    // interval measures device time only, not the host's launch latency
    ADS_CK(ads::launch_delay(2000000ull, s->stream));
    if (s->kind == ADS_ELASTIC)
        rc = s->prec == ADS_FP64 ? elastic_step<double>(s, &kt) : elastic_step<float>(s, &kt);
    else
        rc = s->prec == ADS_FP64 ? pwave_step<double>(s, true, &kt) : pwave_step<float>(s, true, &kt);
    if (rc) return rc;
    s->h_step += 1;
    s->warmed = true;
    ADS_CK(cudaStreamSynchronize(s->stream));
    const int nk = (int)kt.ev.size() - 1;
    for (int i = 0; i < nk && i < cap; ++i) {
        float t = 0.f;
        ADS_CK(cudaEventElapsedTime(&t, kt.ev[i], kt.ev[i + 1]));
        if (ms) ms[i] = t;
        if (names) names[i] = kt.names[i];
    }
    *count = nk;
    return ADS_OK;
}

int ads_profile_rhs(ads_sim_t *s, int reps, float *ms_per_launch)
{
    if (!s || !ms_per_launch || reps < 1 || reps > 10000)
        return fail(ADS_ERR_INVALID_ARG, "ads_profile_rhs: bad arguments");
    if (s->kind != ADS_SCALAR_WAVE) return fail(ADS_ERR_UNSUPPORTED, "ads_profile_rhs: scalar-wave simulations only");
    cudaSetDevice(s->device);
    cudaEvent_t e[2];
    ADS_CK(cudaEventCreate(&e[0]));
    if (cudaEventCreate(&e[1]) != cudaSuccess) {
        cudaEventDestroy(e[0]);
        return fail(ADS_ERR_CUDA, "ads_profile_rhs: cudaEventCreate failed");
    }
    // the K1 launch of a step, repeated: it reads p and overwrites the work field only
    auto run = [&]() -> int {
        ADS_CK(ads::launch_delay(2000000ull, s->stream));
        ADS_CK(cudaEventRecord(e[0], s->stream));
        for (int i = 0; i < reps; ++i) {
            if (s->prec == ADS_FP64)
                ADS_CK(ads::launch_rhs<double>(s->p, s->seg, pwave_launch<double>(s, false).rhs, s->stream));
            else
                ADS_CK(ads::launch_rhs<float>(s->p, s->seg, pwave_launch<float>(s, false).rhs, s->stream));
        }
        ADS_CK(cudaEventRecord(e[1], s->stream));
        ADS_CK(cudaEventSynchronize(e[1]));
        float t = 0.f;
        ADS_CK(cudaEventElapsedTime(&t, e[0], e[1]));
        *ms_per_launch = t / reps;
        return ADS_OK;
    };
    const int rc = run();
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
    return rc;
}

}  // extern "C"
