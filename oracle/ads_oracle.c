/*
 * ads_oracle.c -- plain FP64 CPU oracle of the alternating-direction
 * isogeometric wave solver of Los, Behnoudfar, Paszynski and Calo,
 * "Fast isogeometric solvers for hyperbolic wave propagation problems".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may build, load or call this file.  It shares no code,
 * header, table or helper with the CUDA library: everything below is written
 * out again from the paper, deliberately plain (dense 1D matrices, textbook
 * Cox-de Boor recursion, Newton-iterated Gauss-Legendre rule, Doolittle LU
 * restricted to the band, unfused 1D operator sweeps).
 *
 * Arrays of the 3D space hold the interior coefficients only (the first and
 * last B-spline per axis carry the homogeneous Dirichlet condition and are
 * dropped), laid out [z][y][x] with x fastest: index = (k*my + j)*mx + i.
 *
 * Readings of the paper taken here (the paper is garbled or silent there):
 *  - time scheme: Newmark average acceleration (beta=1/4, gamma=1/2) with the
 *    split operator of eq. (pwave2); the literal eq. (scheme) does not
 *    converge, so the acceleration of step n enters the predictor;
 *  - 3D operator: Laplacian Kronecker sum Kx.My.Mz + Mx.Ky.Mz + Mx.My.Kz
 *    (Sec. 2 derives the 2D case);
 *  - elasticity blocks from the bilinear form 2mu(e(w),e(u)) + lam(div w,div u)
 *    (Sec. 5, eq. lin is garbled);
 *  - alternating-triangular scheme with sigma = 1/2 (eliminating the predictor
 *    from eqs. pre/corr), diagonal blocks factored as eq. spill;
 *  - start-up U^{-1} = U^0 - tau V^0 + tau^2/2 A^0.
 *
 * Parity pins: every function here is checked against closed forms,
 * brute-force dense assembly or SciPy by the CPU test suite.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* 1D spline space (Sec. 2; Appendix: local support over p+1 elements)       */
/* ------------------------------------------------------------------------ */

/* Open uniform knot vector on [0, L]: p+1 copies of each end point and the
 * uniform interior break points.  Length ne + 2p + 1; ne + p basis functions. */
void ora_knots(int ne, int p, double L, double *t)
{
    int k = 0;
    for (int i = 0; i < p; i++) t[k++] = 0.0;
    for (int i = 0; i <= ne; i++) t[k++] = L * (double)i / (double)ne;
    for (int i = 0; i < p; i++) t[k++] = L;
}

/* Gauss-Legendre rule with q points on [-1, 1]: roots of the Legendre
 * polynomial P_q found by Newton's method from the three-term recurrence,
 * weights 2 / ((1 - x^2) P_q'(x)^2). */
void ora_gauss(int q, double *x, double *w)
{
    for (int i = 0; i < q; i++) {
        double r = cos(ORA_PI * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= q; k++) {
                double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = r; p0 = 1.0; }
            dp = q * (r * p1 - p0) / (r * r - 1.0);
            double dr = p1 / dp;
            r -= dr;
            if (fabs(dr) < 1e-16) break;
        }
        /* recompute the derivative at the converged root */
        {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= q; k++) {
                double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (r * p1 - p0) / (r * r - 1.0);
        }
        x[q - 1 - i] = r;
        w[q - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
}

/* All n basis functions of degree p and their first derivatives at x, by the
 * Cox-de Boor recursion.  The degree-0 indicator is taken from `span` (the
 * knot interval [t_span, t_span+1) that contains x) rather than from floating
 * comparisons, so points on element boundaries are attributed to the element
 * being integrated.  0/0 terms of the recursion are taken as 0. */
void ora_basis(const double *t, int n, int p, int span, double x, double *N, double *dN)
{
    int nk = n + p + 1;              /* number of knots */
    double *B = (double *)calloc((size_t)nk, sizeof(double));
    double *Bprev = (double *)calloc((size_t)nk, sizeof(double));
    /* degree 0: nk-1 functions */
    for (int i = 0; i < nk - 1; i++) B[i] = (i == span) ? 1.0 : 0.0;
    for (int k = 1; k <= p; k++) {
        memcpy(Bprev, B, sizeof(double) * (size_t)nk);
        for (int i = 0; i < nk - 1 - k; i++) {
            double a = 0.0, b = 0.0;
            double d1 = t[i + k] - t[i];
            double d2 = t[i + k + 1] - t[i + 1];
            if (d1 > 0.0) a = (x - t[i]) / d1 * Bprev[i];
            if (d2 > 0.0) b = (t[i + k + 1] - x) / d2 * Bprev[i + 1];
            B[i] = a + b;
        }
        if (k == p) {
            /* derivative of degree-p functions from degree p-1 ones */
            for (int i = 0; i < n; i++) {
                double a = 0.0, b = 0.0;
                double d1 = t[i + p] - t[i];
                double d2 = t[i + p + 1] - t[i + 1];
                if (d1 > 0.0) a = p / d1 * Bprev[i];
                if (d2 > 0.0) b = p / d2 * Bprev[i + 1];
                dN[i] = a - b;
            }
        }
        for (int i = nk - 1 - k; i < nk; i++) B[i] = 0.0;
    }
    if (p == 0) for (int i = 0; i < n; i++) dN[i] = 0.0;
    for (int i = 0; i < n; i++) N[i] = B[i];
    free(B);
    free(Bprev);
}

/* Full (unrestricted) n x n 1D matrices by (p+1)-point Gauss quadrature per
 * element, Sec. 2 definitions:  M[a][c] = (N_a, N_c),  K[a][c] = (N'_a, N'_c),
 * and the mixed matrix of Sec. 5,  B[a][c] = (N'_a, N_c).  Any output may be
 * NULL.  Row-major, n = ne + p. */
void ora_mats1d(int ne, int p, double L, double *M, double *K, double *B)
{
    int n = ne + p;
    double *t = (double *)malloc(sizeof(double) * (size_t)(ne + 2 * p + 1));
    double *gx = (double *)malloc(sizeof(double) * (size_t)(p + 1));
    double *gw = (double *)malloc(sizeof(double) * (size_t)(p + 1));
    double *N = (double *)malloc(sizeof(double) * (size_t)n);
    double *dN = (double *)malloc(sizeof(double) * (size_t)n);
    ora_knots(ne, p, L, t);
    ora_gauss(p + 1, gx, gw);
    if (M) memset(M, 0, sizeof(double) * (size_t)n * n);
    if (K) memset(K, 0, sizeof(double) * (size_t)n * n);
    if (B) memset(B, 0, sizeof(double) * (size_t)n * n);
    for (int e = 0; e < ne; e++) {
        double a = t[p + e], b = t[p + e + 1];
        for (int g = 0; g <= p; g++) {
            double x = 0.5 * (a + b) + 0.5 * (b - a) * gx[g];
            double w = 0.5 * (b - a) * gw[g];
            ora_basis(t, n, p, p + e, x, N, dN);
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    if (M) M[i * n + j] += w * N[i] * N[j];
                    if (K) K[i * n + j] += w * dN[i] * dN[j];
                    if (B) B[i * n + j] += w * dN[i] * N[j];
                }
        }
    }
    free(t); free(gx); free(gw); free(N); free(dN);
}

/* ------------------------------------------------------------------------ */
/* 3D tensor-product space with homogeneous Dirichlet restriction            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int ne[3], p, n[3], m[3];
    int off;                      /* 1: Dirichlet (first/last function dropped), 0: natural */
    double L[3];
    double *M[3], *K[3], *B[3];   /* restricted m x m, row-major */
    double *t[3];                 /* knot vectors */
} ora_space;

/* natural != 0 keeps every basis function (traction-free / natural boundary,
 * Sec. 5); otherwise the homogeneous Dirichlet restriction drops the first
 * and last function per axis.  ne[2] == 0 is a 2D problem (Sec. 2 derives
 * the method in 2D): the z axis carries one constant function, M = [1],
 * K = B = [0], so every 3D operator below reduces to its 2D form. */
ora_space *ora_space_new_bc(const int *ne, int p, const double *L, int natural)
{
    ora_space *s = (ora_space *)calloc(1, sizeof(ora_space));
    s->p = p;
    s->off = natural ? 0 : 1;
    for (int a = 0; a < 3; a++) {
        if (a == 2 && ne[2] == 0) {
            s->ne[2] = 0;
            s->n[2] = s->m[2] = 1;
            s->L[2] = 1.0;
            s->M[2] = (double *)calloc(1, sizeof(double));
            s->K[2] = (double *)calloc(1, sizeof(double));
            s->B[2] = (double *)calloc(1, sizeof(double));
            s->M[2][0] = 1.0;
            s->t[2] = NULL;
            continue;
        }
        int n = ne[a] + p, m = n - 2 * s->off;
        s->ne[a] = ne[a];
        s->n[a] = n;
        s->m[a] = m;
        s->L[a] = L[a];
        double *Mf = (double *)malloc(sizeof(double) * (size_t)n * n);
        double *Kf = (double *)malloc(sizeof(double) * (size_t)n * n);
        double *Bf = (double *)malloc(sizeof(double) * (size_t)n * n);
        ora_mats1d(ne[a], p, L[a], Mf, Kf, Bf);
        s->M[a] = (double *)malloc(sizeof(double) * (size_t)m * m);
        s->K[a] = (double *)malloc(sizeof(double) * (size_t)m * m);
        s->B[a] = (double *)malloc(sizeof(double) * (size_t)m * m);
        /* Dirichlet: drop basis functions 0 and n-1 */
        const int o = s->off;
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) {
                s->M[a][i * m + j] = Mf[(i + o) * n + (j + o)];
                s->K[a][i * m + j] = Kf[(i + o) * n + (j + o)];
                s->B[a][i * m + j] = Bf[(i + o) * n + (j + o)];
            }
        free(Mf); free(Kf); free(Bf);
        s->t[a] = (double *)malloc(sizeof(double) * (size_t)(ne[a] + 2 * p + 1));
        ora_knots(ne[a], p, L[a], s->t[a]);
    }
    return s;
}

ora_space *ora_space_new(const int *ne, int p, const double *L) { return ora_space_new_bc(ne, p, L, 0); }

void ora_space_free(ora_space *s)
{
    if (!s) return;
    for (int a = 0; a < 3; a++) { free(s->M[a]); free(s->K[a]); free(s->B[a]); free(s->t[a]); }
    free(s);
}

void ora_space_dims(const ora_space *s, int *m) { for (int a = 0; a < 3; a++) m[a] = s->m[a]; }

/* copy out a restricted 1D matrix: which = 0 (M), 1 (K), 2 (B) */
void ora_space_mat(const ora_space *s, int axis, int which, double *out)
{
    const double *src = which == 0 ? s->M[axis] : (which == 1 ? s->K[axis] : s->B[axis]);
    memcpy(out, src, sizeof(double) * (size_t)s->m[axis] * s->m[axis]);
}

static size_t ora_size(const ora_space *s) { return (size_t)s->m[0] * s->m[1] * s->m[2]; }

/* out = A applied along `axis` to in (A is m_axis x m_axis, row-major, only
 * its band |i-j| <= p is nonzero: Appendix, M_ij = 0 iff |i-j| > p).
 * transpose != 0 applies A^T.  out must not alias in. */
static void apply_axis(const ora_space *s, const double *A, int transpose, int axis,
                       const double *in, double *out)
{
    int mx = s->m[0], my = s->m[1], mz = s->m[2], p = s->p;
    int ma = s->m[axis];
    long stride = axis == 0 ? 1 : (axis == 1 ? mx : (long)mx * my);
    long nlines = (long)mx * my * mz / ma;
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nlines; l++) {
        long base;
        if (axis == 0) base = l * mx;
        else if (axis == 1) base = (l / mx) * (long)mx * my + (l % mx);
        else base = l;
        for (int i = 0; i < ma; i++) {
            double acc = 0.0;
            int j0 = i - p < 0 ? 0 : i - p, j1 = i + p > ma - 1 ? ma - 1 : i + p;
            for (int j = j0; j <= j1; j++) {
                double aij = transpose ? A[j * ma + i] : A[i * ma + j];
                acc += aij * in[base + j * stride];
            }
            out[base + i * stride] = acc;
        }
    }
}

/* out = (A_x (x) A_y (x) A_z) in, one 1D operator per axis (NULL = identity),
 * applied as three unfused axis sweeps.  tr[a] selects the transpose. */
static void apply_kron(const ora_space *s, const double *Ax, const double *Ay, const double *Az,
                       const int *tr, const double *in, double *out)
{
    size_t N = ora_size(s);
    double *t1 = (double *)malloc(sizeof(double) * N);
    double *t2 = (double *)malloc(sizeof(double) * N);
    const double *A[3] = {Ax, Ay, Az};
    memcpy(t1, in, sizeof(double) * N);
    for (int a = 0; a < 3; a++) {
        if (!A[a]) continue;
        apply_axis(s, A[a], tr ? tr[a] : 0, a, t1, t2);
        double *tmp = t1; t1 = t2; t2 = tmp;
    }
    memcpy(out, t1, sizeof(double) * N);
    free(t1);
    free(t2);
}

/* K u for the 3D Laplacian stiffness (reading of Sec. 2 in 3D):
 *   K = Kx.My.Mz + Mx.Ky.Mz + Mx.My.Kz, scaled by c2. */
void ora_apply_lap(const ora_space *s, double c2, const double *in, double *out)
{
    size_t N = ora_size(s);
    double *t = (double *)malloc(sizeof(double) * N);
    apply_kron(s, s->K[0], s->M[1], s->M[2], NULL, in, out);
    apply_kron(s, s->M[0], s->K[1], s->M[2], NULL, in, t);
    for (size_t i = 0; i < N; i++) out[i] += t[i];
    apply_kron(s, s->M[0], s->M[1], s->K[2], NULL, in, t);
    for (size_t i = 0; i < N; i++) out[i] = c2 * (out[i] + t[i]);
    free(t);
}

/* M u with the 3D mass matrix Mx.My.Mz */
void ora_apply_mass(const ora_space *s, const double *in, double *out)
{
    apply_kron(s, s->M[0], s->M[1], s->M[2], NULL, in, out);
}

/* ---- banded LU (Appendix: O(N) solve by 1D banded multi-RHS solves) ---- */

/* Pivot-free Doolittle LU of an m x m matrix whose nonzeros lie in the band
 * |i-j| <= p; the factors overwrite A (unit lower L below the diagonal).
 * Without pivoting no fill appears outside the band.  The 1D matrices used
 * here are SPD, so no pivot vanishes. */
static void lu_band(double *A, int m, int p)
{
    for (int k = 0; k < m; k++) {
        int iend = k + p < m - 1 ? k + p : m - 1;
        for (int i = k + 1; i <= iend; i++) {
            double l = A[i * m + k] / A[k * m + k];
            A[i * m + k] = l;
            for (int j = k + 1; j <= iend; j++) A[i * m + j] -= l * A[k * m + j];
        }
    }
}

/* solve (LU) x = b along `axis` for every line, in place on v */
static void solve_axis(const ora_space *s, const double *LU, int axis, double *v)
{
    int mx = s->m[0], my = s->m[1], mz = s->m[2], p = s->p;
    int ma = s->m[axis];
    long stride = axis == 0 ? 1 : (axis == 1 ? mx : (long)mx * my);
    long nlines = (long)mx * my * mz / ma;
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nlines; l++) {
        long base;
        if (axis == 0) base = l * mx;
        else if (axis == 1) base = (l / mx) * (long)mx * my + (l % mx);
        else base = l;
        /* forward: L y = b */
        for (int i = 0; i < ma; i++) {
            double acc = v[base + i * stride];
            int j0 = i - p < 0 ? 0 : i - p;
            for (int j = j0; j < i; j++) acc -= LU[i * ma + j] * v[base + j * stride];
            v[base + i * stride] = acc;
        }
        /* backward: U x = y */
        for (int i = ma - 1; i >= 0; i--) {
            double acc = v[base + i * stride];
            int j1 = i + p > ma - 1 ? ma - 1 : i + p;
            for (int j = i + 1; j <= j1; j++) acc -= LU[i * ma + j] * v[base + j * stride];
            v[base + i * stride] = acc / LU[i * ma + i];
        }
    }
}

/* out = (A_x (x) A_y (x) A_z)^{-1} in with A_a = M_a + d[a] K_a, via three
 * directional banded solves (Appendix).  d = {0,0,0} gives the exact mass
 * inverse. */
void ora_solve_kron(const ora_space *s, const double *d, const double *in, double *out)
{
    size_t N = ora_size(s);
    if (out != in) memcpy(out, in, sizeof(double) * N);
    for (int a = 0; a < 3; a++) {
        int m = s->m[a];
        double *A = (double *)malloc(sizeof(double) * (size_t)m * m);
        for (int i = 0; i < m * m; i++) A[i] = s->M[a][i] + d[a] * s->K[a][i];
        lu_band(A, m, s->p);
        solve_axis(s, A, a, out);
        free(A);
    }
}

void ora_solve_mass(const ora_space *s, const double *in, double *out)
{
    const double d[3] = {0.0, 0.0, 0.0};
    ora_solve_kron(s, d, in, out);
}

/* ---- load vectors ---- */

/* Interior load vector (g, N_ijk) of g(x) = amp * exp(-|x - c|^2 / den) by
 * plain 3D tensor Gauss quadrature, (p+1)^3 points per element. */
void ora_load_gauss(const ora_space *s, double amp, const double *c, double den, double *out)
{
    int p = s->p, q = p + 1;
    int mx = s->m[0], my = s->m[1];
    size_t N = ora_size(s);
    memset(out, 0, sizeof(double) * N);
    double *gx = (double *)malloc(sizeof(double) * (size_t)q);
    double *gw = (double *)malloc(sizeof(double) * (size_t)q);
    ora_gauss(q, gx, gw);
    /* basis values at every quadrature point of every element, per axis */
    double *V[3];
    double *X[3], *W[3];
    const int dim2 = s->ne[2] == 0;
    for (int a = 0; a < 3; a++) {
        if (a == 2 && dim2) {   /* one "element", one point of weight 1, value 1 */
            V[2] = (double *)calloc((size_t)q * (p + 1), sizeof(double));
            X[2] = (double *)calloc((size_t)q, sizeof(double));
            W[2] = (double *)calloc((size_t)q, sizeof(double));
            V[2][0] = 1.0;
            W[2][0] = 1.0;
            X[2][0] = c[2];
            continue;
        }
        int ne = s->ne[a], n = s->n[a];
        V[a] = (double *)malloc(sizeof(double) * (size_t)ne * q * (p + 1));
        X[a] = (double *)malloc(sizeof(double) * (size_t)ne * q);
        W[a] = (double *)malloc(sizeof(double) * (size_t)ne * q);
        double *Nb = (double *)malloc(sizeof(double) * (size_t)n);
        double *dNb = (double *)malloc(sizeof(double) * (size_t)n);
        for (int e = 0; e < ne; e++) {
            double lo = s->t[a][p + e], hi = s->t[a][p + e + 1];
            for (int g = 0; g < q; g++) {
                double x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[g];
                X[a][e * q + g] = x;
                W[a][e * q + g] = 0.5 * (hi - lo) * gw[g];
                ora_basis(s->t[a], n, p, p + e, x, Nb, dNb);
                /* nonzero functions on element e are e .. e+p */
                for (int b = 0; b <= p; b++) V[a][(e * q + g) * (p + 1) + b] = Nb[e + b];
            }
        }
        free(Nb);
        free(dNb);
    }
    const int nez = dim2 ? 1 : s->ne[2], qz = dim2 ? 1 : q, offz = dim2 ? 0 : s->off;
    for (int ez = 0; ez < nez; ez++)
        for (int ey = 0; ey < s->ne[1]; ey++)
            for (int ex = 0; ex < s->ne[0]; ex++)
                for (int gz = 0; gz < qz; gz++)
                    for (int gy = 0; gy < q; gy++)
                        for (int gxi = 0; gxi < q; gxi++) {
                            int iz = ez * q + gz, iy = ey * q + gy, ix = ex * q + gxi;
                            double dx = X[0][ix] - c[0], dy = X[1][iy] - c[1], dz = X[2][iz] - c[2];
                            double g = amp * exp(-(dx * dx + dy * dy + dz * dz) / den);
                            double w = W[0][ix] * W[1][iy] * W[2][iz] * g;
                            for (int bz = 0; bz <= (dim2 ? 0 : p); bz++) {
                                int k = ez + bz - offz;       /* unknown index */
                                if (k < 0 || k >= s->m[2]) continue;
                                double vz = V[2][iz * (p + 1) + bz];
                                for (int by = 0; by <= p; by++) {
                                    int j = ey + by - s->off;
                                    if (j < 0 || j >= my) continue;
                                    double vy = V[1][iy * (p + 1) + by];
                                    for (int bx = 0; bx <= p; bx++) {
                                        int i = ex + bx - s->off;
                                        if (i < 0 || i >= mx) continue;
                                        double vx = V[0][ix * (p + 1) + bx];
                                        out[((size_t)k * my + j) * mx + i] += w * vx * vy * vz;
                                    }
                                }
                            }
                        }
    for (int a = 0; a < 3; a++) { free(V[a]); free(X[a]); free(W[a]); }
    free(gx);
    free(gw);
}

/* L2 projection of amp*exp(-|x-c|^2/den): exact mass solve of the load
 * (the isogeometric L2 projection closing the Appendix). */
void ora_project_gauss(const ora_space *s, double amp, const double *c, double den, double *out)
{
    size_t N = ora_size(s);
    double *f = (double *)malloc(sizeof(double) * N);
    ora_load_gauss(s, amp, c, den, f);
    ora_solve_mass(s, f, out);
    free(f);
}

/* Ricker wavelet r(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2) */
double ora_ricker(double f, double t0, double t)
{
    double a = ORA_PI * ORA_PI * f * f * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}

/* ------------------------------------------------------------------------ */
/* Scalar P-wave: Newmark average acceleration with the split operator       */
/* (eq. pwave2, Sec. 2, read as beta = 1/4, gamma = 1/2)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double tau, c2;
    const double *G;      /* spatial load (g, w), NULL = no source */
    double rick_f, rick_t0;
} ora_pwave;

/* Consistent initial acceleration a0 = M^{-1}(F(t) - K u0) (exact mass). */
void ora_pwave_accel(const ora_space *s, double c2, const double *G, double rf, double rt0,
                     double t, const double *u, double *a)
{
    size_t N = ora_size(s);
    double *r = (double *)malloc(sizeof(double) * N);
    ora_apply_lap(s, c2, u, r);
    double rt = G ? ora_ricker(rf, rt0, t) : 0.0;
    for (size_t i = 0; i < N; i++) r[i] = (G ? rt * G[i] : 0.0) - r[i];
    ora_solve_mass(s, r, a);
    free(r);
}

/* Advance (u, v, a) by nsteps steps starting at step index step0 (time
 * step0*tau).  Per step:
 *   G~ a1 = F(t_{n+1}) - K (u + tau v + eta a),   G~ = (x)_xi (M_xi + eta K_xi)
 *   u1 = u + tau v + eta (a + a1),  v1 = v + tau/2 (a + a1),  eta = tau^2/4. */
void ora_pwave_run(const ora_space *s, double tau, double c2, const double *G, double rf, double rt0,
                   long step0, int nsteps, double *u, double *v, double *a)
{
    size_t N = ora_size(s);
    double eta = 0.25 * tau * tau;
    double d[3] = {eta * c2, eta * c2, eta * c2};
    double *pr = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *a1 = (double *)malloc(sizeof(double) * N);
    for (int n = 0; n < nsteps; n++) {
        double t1 = (double)(step0 + n + 1) * tau;
        for (size_t i = 0; i < N; i++) pr[i] = u[i] + tau * v[i] + eta * a[i];
        ora_apply_lap(s, c2, pr, r);
        double rt = G ? ora_ricker(rf, rt0, t1) : 0.0;
        for (size_t i = 0; i < N; i++) r[i] = (G ? rt * G[i] : 0.0) - r[i];
        ora_solve_kron(s, d, r, a1);
        for (size_t i = 0; i < N; i++) {
            u[i] = u[i] + tau * v[i] + eta * (a[i] + a1[i]);
            v[i] = v[i] + 0.5 * tau * (a[i] + a1[i]);
            a[i] = a1[i];
        }
    }
    free(pr);
    free(r);
    free(a1);
}

static double dot(const double *x, const double *y, size_t N)
{
    double s = 0.0;
    for (size_t i = 0; i < N; i++) s += x[i] * y[i];
    return s;
}

/* Energies of the P-wave state: kinetic 1/2 v^T M v, potential 1/2 u^T K u,
 * and the kinetic part 1/2 v^T (G~ - eta K) v of the discrete invariant of the
 * split Newmark scheme (conserved exactly when f = 0). */
void ora_pwave_energy(const ora_space *s, double tau, double c2, const double *u, const double *v,
                      double *kin, double *pot, double *kin_mod)
{
    size_t N = ora_size(s);
    double eta = 0.25 * tau * tau;
    double *t = (double *)malloc(sizeof(double) * N);
    double *t2 = (double *)malloc(sizeof(double) * N);
    ora_apply_mass(s, v, t);
    *kin = 0.5 * dot(v, t, N);
    ora_apply_lap(s, c2, u, t);
    *pot = 0.5 * dot(u, t, N);
    /* G~ v */
    double *A[3];
    for (int a = 0; a < 3; a++) {
        int m = s->m[a];
        A[a] = (double *)malloc(sizeof(double) * (size_t)m * m);
        for (int i = 0; i < m * m; i++) A[a][i] = s->M[a][i] + eta * c2 * s->K[a][i];
    }
    apply_kron(s, A[0], A[1], A[2], NULL, v, t);
    ora_apply_lap(s, c2, v, t2);
    for (size_t i = 0; i < N; i++) t[i] -= eta * t2[i];
    *kin_mod = 0.5 * dot(v, t, N);
    for (int a = 0; a < 3; a++) free(A[a]);
    free(t);
    free(t2);
}

/* ------------------------------------------------------------------------ */
/* Linear elasticity (Sec. 5), 3 components stored component-major          */
/* ------------------------------------------------------------------------ */

/* which 1D factor on each axis: 0 = M, 1 = K, 2 = B, 3 = B^T */
static const double *fac(const ora_space *s, int axis, int which, int *tr)
{
    *tr = 0;
    if (which == 0) return s->M[axis];
    if (which == 1) return s->K[axis];
    if (which == 3) *tr = 1;
    return s->B[axis];
}

static void kron_term(const ora_space *s, const int *which, double coef, const double *in, double *acc,
                      double *tmp)
{
    int tr[3];
    const double *A0 = fac(s, 0, which[0], &tr[0]);
    const double *A1 = fac(s, 1, which[1], &tr[1]);
    const double *A2 = fac(s, 2, which[2], &tr[2]);
    apply_kron(s, A0, A1, A2, tr, in, tmp);
    size_t N = ora_size(s);
    for (size_t i = 0; i < N; i++) acc[i] += coef * tmp[i];
}

/* out_i += Upsilon_ij in_j for one block (i, j), from the bilinear form
 * 2 mu (e(w), e(u)) + lam (div w, div u):
 *   i == j: mu (Kx My Mz + Mx Ky Mz + Mx My Kz) + (mu + lam) [K on axis i]
 *   i != j: mu [B^T on axis i, B on axis j] + lam [B on axis i, B^T on axis j]
 * with B[a][c] = (N'_a, N_c) (derivative on the test function). */
void ora_elastic_block(const ora_space *s, double lam, double mu, int i, int j, const double *in,
                       double *out)
{
    size_t N = ora_size(s);
    double *tmp = (double *)malloc(sizeof(double) * N);
    if (i == j) {
        for (int k = 0; k < 3; k++) {
            int w[3] = {0, 0, 0};
            w[k] = 1;
            kron_term(s, w, mu + (k == i ? mu + lam : 0.0), in, out, tmp);
        }
    } else {
        int w1[3] = {0, 0, 0}, w2[3] = {0, 0, 0};
        w1[i] = 3; w1[j] = 2;
        w2[i] = 2; w2[j] = 3;
        kron_term(s, w1, mu, in, out, tmp);
        kron_term(s, w2, lam, in, out, tmp);
    }
    free(tmp);
}

/* out = Upsilon U (all 3 components) */
void ora_elastic_apply(const ora_space *s, double lam, double mu, const double *U, double *out)
{
    size_t N = ora_size(s);
    memset(out, 0, sizeof(double) * 3 * N);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) ora_elastic_block(s, lam, mu, i, j, U + j * N, out + i * N);
}

/* diagonal-block solve of eq. (spill):
 *   L~_i = rho (x)_xi (M_xi + tau^2 c_{i,xi} / (4 rho) K_xi),
 *   c_{i,xi} = 2 mu + lam if xi == i else mu. */
static void elastic_diag_solve(const ora_space *s, double tau, double lam, double mu, double rho, int i,
                               const double *in, double *out)
{
    double d[3];
    for (int a = 0; a < 3; a++) d[a] = tau * tau * (a == i ? 2.0 * mu + lam : mu) / (4.0 * rho);
    ora_solve_kron(s, d, in, out);
    size_t N = ora_size(s);
    for (size_t k = 0; k < N; k++) out[k] /= rho;
}

/* One alternating-triangular step (eqs. pre, corr, gen with sigma = 1/2):
 *   D (U1 - 2U + U0) / tau^2 + Upsilon U = f,  f = 0 here,
 *   D = (rho M + tau^2/2 Ups1~) (rho M)^{-1} (rho M + tau^2/2 Ups2~).
 * Block-lower solve for y, y -> rho M y, block-upper solve for delta. */
void ora_elastic_run_src(const ora_space *s, double tau, double lam, double mu, double rho, int nsteps,
                         double *Ucur, double *Uprev, const double *G, const double *dir, double rf, double rt0,
                         long step0);

void ora_elastic_run(const ora_space *s, double tau, double lam, double mu, double rho, int nsteps,
                     double *Ucur, double *Uprev)
{
    ora_elastic_run_src(s, tau, lam, mu, rho, nsteps, Ucur, Uprev, NULL, NULL, 0.0, 0.0, 0);
}

/* As ora_elastic_run with a body force f^n = r(t_n) dir_i g (eq. gen: the
 * right-hand side at level n, t_n = n tau), G = (g, w) the scalar load;
 * G == NULL: no force.  step0 = index n of Ucur. */
void ora_elastic_run_src(const ora_space *s, double tau, double lam, double mu, double rho, int nsteps,
                         double *Ucur, double *Uprev, const double *G, const double *dir, double rf, double rt0,
                         long step0)
{
    size_t N = ora_size(s);
    double *r = (double *)malloc(sizeof(double) * 3 * N);
    double *y = (double *)malloc(sizeof(double) * 3 * N);
    double *sv = (double *)malloc(sizeof(double) * 3 * N);
    double *dl = (double *)malloc(sizeof(double) * 3 * N);
    double *rhs = (double *)malloc(sizeof(double) * N);
    double *tmp = (double *)malloc(sizeof(double) * N);
    double h = 0.5 * tau * tau;
    for (int n = 0; n < nsteps; n++) {
        ora_elastic_apply(s, lam, mu, Ucur, r);
        for (size_t k = 0; k < 3 * N; k++) r[k] = -tau * tau * r[k];
        if (G) {
            const double rt = ora_ricker(rf, rt0, (double)(step0 + n) * tau);
            for (int i = 0; i < 3; i++)
                for (size_t k = 0; k < N; k++) r[i * N + k] += tau * tau * rt * dir[i] * G[k];
        }
        /* block lower: for i = x, y, z */
        for (int i = 0; i < 3; i++) {
            memcpy(rhs, r + i * N, sizeof(double) * N);
            for (int j = 0; j < i; j++) {
                memset(tmp, 0, sizeof(double) * N);
                ora_elastic_block(s, lam, mu, i, j, y + j * N, tmp);
                for (size_t k = 0; k < N; k++) rhs[k] -= h * tmp[k];
            }
            elastic_diag_solve(s, tau, lam, mu, rho, i, rhs, y + i * N);
        }
        /* rho M y */
        for (int i = 0; i < 3; i++) {
            ora_apply_mass(s, y + i * N, sv + i * N);
            for (size_t k = 0; k < N; k++) sv[i * N + k] *= rho;
        }
        /* block upper: for i = z, y, x */
        for (int i = 2; i >= 0; i--) {
            memcpy(rhs, sv + i * N, sizeof(double) * N);
            for (int j = i + 1; j < 3; j++) {
                memset(tmp, 0, sizeof(double) * N);
                ora_elastic_block(s, lam, mu, i, j, dl + j * N, tmp);
                for (size_t k = 0; k < N; k++) rhs[k] -= h * tmp[k];
            }
            elastic_diag_solve(s, tau, lam, mu, rho, i, rhs, dl + i * N);
        }
        for (size_t k = 0; k < 3 * N; k++) {
            double u1 = 2.0 * Ucur[k] - Uprev[k] + dl[k];
            Uprev[k] = Ucur[k];
            Ucur[k] = u1;
        }
    }
    free(r); free(y); free(sv); free(dl); free(rhs); free(tmp);
}

/* Start-up of the three-level scheme: U^{-1} = U0 - tau V0 + tau^2/2 A0 with
 * A0 = (rho M)^{-1}(f - Upsilon U0), f = 0. */
void ora_elastic_start_src(const ora_space *s, double tau, double lam, double mu, double rho, const double *U0,
                           const double *V0, double *Uprev, const double *G, const double *dir, double rf, double rt0,
                           double t0);

void ora_elastic_start(const ora_space *s, double tau, double lam, double mu, double rho, const double *U0,
                       const double *V0, double *Uprev)
{
    ora_elastic_start_src(s, tau, lam, mu, rho, U0, V0, Uprev, NULL, NULL, 0.0, 0.0, 0.0);
}

/* start-up with a body force f(t0) = r(t0) dir_i g */
void ora_elastic_start_src(const ora_space *s, double tau, double lam, double mu, double rho, const double *U0,
                           const double *V0, double *Uprev, const double *G, const double *dir, double rf, double rt0,
                           double t0)
{
    size_t N = ora_size(s);
    double *r = (double *)malloc(sizeof(double) * 3 * N);
    double *A0 = (double *)malloc(sizeof(double) * 3 * N);
    ora_elastic_apply(s, lam, mu, U0, r);
    const double rt = G ? ora_ricker(rf, rt0, t0) : 0.0;
    for (int i = 0; i < 3; i++) {
        for (size_t k = 0; k < N; k++)
            r[i * N + k] = ((G ? rt * dir[i] * G[k] : 0.0) - r[i * N + k]) / rho;
        ora_solve_mass(s, r + i * N, A0 + i * N);
    }
    for (size_t k = 0; k < 3 * N; k++) Uprev[k] = U0[k] - tau * V0[k] + 0.5 * tau * tau * A0[k];
    free(r);
    free(A0);
}

/* Discrete invariant of the three-level scheme (f = 0):
 *   E = |(U1 - U)/tau|^2_{D - tau^2 Ups/4} + |(U1 + U)/2|^2_Ups,
 * with |x|^2_D = (L^T x)^T (rho M)^{-1} (L^T x) and L^T the block-upper factor. */
double ora_elastic_invariant(const ora_space *s, double tau, double lam, double mu, double rho,
                             const double *U1, const double *U)
{
    size_t N = ora_size(s);
    double h = 0.5 * tau * tau;
    double *vh = (double *)malloc(sizeof(double) * 3 * N);
    double *av = (double *)malloc(sizeof(double) * 3 * N);
    double *w = (double *)malloc(sizeof(double) * 3 * N);
    double *z = (double *)malloc(sizeof(double) * 3 * N);
    double *tmp = (double *)malloc(sizeof(double) * N);
    for (size_t k = 0; k < 3 * N; k++) {
        vh[k] = (U1[k] - U[k]) / tau;
        av[k] = 0.5 * (U1[k] + U[k]);
    }
    /* w = L^T vh: diagonal blocks L~_i (as operators), upper blocks h Ups_ij */
    memset(w, 0, sizeof(double) * 3 * N);
    for (int i = 0; i < 3; i++) {
        int m0 = s->m[0], m1 = s->m[1], m2 = s->m[2];
        double *A[3];
        int dims[3] = {m0, m1, m2};
        for (int a = 0; a < 3; a++) {
            int m = dims[a];
            double d = tau * tau * (a == i ? 2.0 * mu + lam : mu) / (4.0 * rho);
            A[a] = (double *)malloc(sizeof(double) * (size_t)m * m);
            for (int q = 0; q < m * m; q++) A[a][q] = s->M[a][q] + d * s->K[a][q];
        }
        apply_kron(s, A[0], A[1], A[2], NULL, vh + i * N, tmp);
        for (size_t k = 0; k < N; k++) w[i * N + k] += rho * tmp[k];
        for (int a = 0; a < 3; a++) free(A[a]);
        for (int j = i + 1; j < 3; j++) {
            memset(tmp, 0, sizeof(double) * N);
            ora_elastic_block(s, lam, mu, i, j, vh + j * N, tmp);
            for (size_t k = 0; k < N; k++) w[i * N + k] += h * tmp[k];
        }
    }
    for (int i = 0; i < 3; i++) {
        ora_solve_mass(s, w + i * N, z + i * N);
        for (size_t k = 0; k < N; k++) z[i * N + k] /= rho;
    }
    double e = dot(w, z, 3 * N);
    ora_elastic_apply(s, lam, mu, vh, z);
    e -= 0.25 * tau * tau * dot(vh, z, 3 * N);
    ora_elastic_apply(s, lam, mu, av, z);
    e += dot(av, z, 3 * N);
    free(vh); free(av); free(w); free(z); free(tmp);
    return e;
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the OpenMP loops from now on (n >= 1); timing only, the
 * arithmetic and its order do not depend on it */
void ora_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
