// setup1d.cpp -- see setup1d.h.  FP64, O(n p^2) per axis; runs once per
// simulation (never inside a time step).
#include "setup1d.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace ads {

// Gauss-Legendre nodes/weights on [-1,1]: Newton on P_q with the Bonnet
// recurrence, symmetric pairs computed once.
void gauss_legendre(int q, double *x, double *w)
{
    const double pi = 3.141592653589793238462643;
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5));
        double dpz = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm1 = 0.0, pc = 1.0;
            for (int k = 1; k <= q; ++k) {
                double pn = ((2 * k - 1) * z * pc - (k - 1) * pm1) / k;
                pm1 = pc;
                pc = pn;
            }
            dpz = q * (z * pc - pm1) / (z * z - 1.0);
            double dz = pc / dpz;
            z -= dz;
            if (std::fabs(dz) <= 1e-16 * std::fabs(z) + 1e-300) {
                // final derivative at the converged root
                pm1 = 0.0; pc = 1.0;
                for (int k = 1; k <= q; ++k) {
                    double pn = ((2 * k - 1) * z * pc - (k - 1) * pm1) / k;
                    pm1 = pc;
                    pc = pn;
                }
                dpz = q * (z * pc - pm1) / (z * z - 1.0);
                break;
            }
        }
        double wt = 2.0 / ((1.0 - z * z) * dpz * dpz);
        x[i] = -z;  w[i] = wt;
        x[q - 1 - i] = z;  w[q - 1 - i] = wt;
    }
    if (q % 2 == 1) x[q / 2] = 0.0;
}

namespace {

// The p+1 nonzero B-splines N_{s-p..s} and derivatives at x in knot span s,
// by the triangular table of left/right knot differences.
void local_basis(const std::vector<double> &t, int s, int p, double x, double *N, double *dN)
{
    double ndu[5][5];
    double left[5], right[5];
    ndu[0][0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = x - t[s + 1 - j];
        right[j] = t[s + j] - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            ndu[j][r] = right[r + 1] + left[j - r];         // knot difference (lower)
            double tmp = ndu[r][j - 1] / ndu[j][r];
            ndu[r][j] = saved + right[r + 1] * tmp;         // basis (upper)
            saved = left[j - r] * tmp;
        }
        ndu[j][j] = saved;
    }
    for (int r = 0; r <= p; ++r) N[r] = ndu[r][p];
    if (p == 0) { dN[0] = 0.0; return; }
    // first derivative: p * (N_{r,p-1}/(t_{r+p}-t_r) - N_{r+1,p-1}/(t_{r+p+1}-t_{r+1}))
    for (int r = 0; r <= p; ++r) {
        double d = 0.0;
        if (r >= 1) d += ndu[r - 1][p - 1] / ndu[p][r - 1];
        if (r <= p - 1) d -= ndu[r][p - 1] / ndu[p][r];
        dN[r] = p * d;
    }
}

}  // namespace

Axis1D build_axis(int ne, int p, double L, bool natural)
{
    if (ne < 1 || p < 1 || p > 4) throw std::invalid_argument("build_axis: ne >= 1, 1 <= p <= 4");
    Axis1D ax;
    ax.off = natural ? 0 : 1;
    ax.ne = ne; ax.p = p; ax.n = ne + p; ax.m = ne + p - 2 * ax.off; ax.L = L;
    if (ax.m < 1) throw std::invalid_argument("build_axis: no interior function");
    std::vector<double> t(ne + 2 * p + 1);
    for (int i = 0; i <= p; ++i) { t[i] = 0.0; t[ne + p + i] = L; }
    for (int i = 1; i < ne; ++i) t[p + i] = L * i / ne;
    for (Band *b : {&ax.M, &ax.K, &ax.B}) { b->m = ax.m; b->p = p; b->v.assign((size_t)ax.m * (2 * p + 1), 0.0); }
    double gx[8], gw[8], N[5], dN[5];
    gauss_legendre(p + 1, gx, gw);
    for (int e = 0; e < ne; ++e) {
        double a = t[p + e], b = t[p + e + 1], h = b - a;
        for (int g = 0; g <= p; ++g) {
            double x = a + 0.5 * h * (1.0 + gx[g]), w = 0.5 * h * gw[g];
            local_basis(t, p + e, p, x, N, dN);
            for (int r = 0; r <= p; ++r) {
                int i = e + r - ax.off;            // unknown index of function e+r
                if (i < 0 || i >= ax.m) continue;
                for (int c = 0; c <= p; ++c) {
                    int j = e + c - ax.off;
                    if (j < 0 || j >= ax.m) continue;
                    ax.M.at(i, j - i) += w * N[r] * N[c];
                    ax.K.at(i, j - i) += w * dN[r] * dN[c];
                    ax.B.at(i, j - i) += w * dN[r] * N[c];
                }
            }
        }
    }
    // one exact interior stencil row for all Toeplitz rows of M, K and B
    auto rm = canonicalize_interior(ax.M);
    auto rk = canonicalize_interior(ax.K);
    auto rb = canonicalize_interior(ax.B);
    ax.lo = std::max(rm.first, std::max(rk.first, rb.first));
    ax.hi = std::min(rm.second, std::min(rk.second, rb.second));
    if (ax.hi < ax.lo) ax.hi = ax.lo;
    // B^T in band storage: Bt[i][i+k] = B[i+k][i]
    ax.Bt.m = ax.m;
    ax.Bt.p = p;
    ax.Bt.v.assign((size_t)ax.m * (2 * p + 1), 0.0);
    for (int i = 0; i < ax.m; ++i)
        for (int k = -p; k <= p; ++k)
            if (i + k >= 0 && i + k < ax.m) ax.Bt.at(i, k) = ax.B.at(i + k, -k);
    return ax;
}

Axis1D trivial_axis(int p)
{
    Axis1D ax;
    ax.ne = 0; ax.p = p; ax.n = 1; ax.m = 1; ax.off = 0; ax.L = 1.0;
    for (Band *b : {&ax.M, &ax.K, &ax.B, &ax.Bt}) { b->m = 1; b->p = p; b->v.assign((size_t)(2 * p + 1), 0.0); }
    ax.M.at(0, 0) = 1.0;
    ax.lo = ax.hi = 0;
    return ax;
}

Factor factor_axis(const Axis1D &ax, double d)
{
    const int m = ax.m, p = ax.p, W = 2 * p + 1;
    Band A;
    A.m = m; A.p = p; A.v.resize((size_t)m * W);
    for (size_t i = 0; i < A.v.size(); ++i) A.v[i] = ax.M.v[i] + d * ax.K.v[i];
    // in-place band LU, no pivoting: A.at(i,k<0) <- l, A.at(i,k>=0) <- U
    for (int k = 0; k < m; ++k) {
        double piv = A.at(k, 0);
        if (!(piv > 0.0)) throw std::runtime_error("factor_axis: nonpositive pivot");
        for (int i = k + 1; i <= std::min(m - 1, k + p); ++i) {
            double l = A.at(i, k - i) / piv;
            A.at(i, k - i) = l;
            for (int j = k + 1; j <= std::min(m - 1, k + p); ++j) A.at(i, j - i) -= l * A.at(k, j - k);
        }
    }
    Factor f;
    f.m = m; f.p = p; f.v.assign((size_t)m * W, 0.0);
    for (int i = 0; i < m; ++i) {
        double *row = &f.v[(size_t)i * W];
        for (int k = 1; k <= p; ++k) {
            row[p - k] = (i - k >= 0) ? A.at(i, -k) : 0.0;
            row[p + k] = (i + k < m) ? A.at(i, k) : 0.0;
        }
        row[p] = 1.0 / A.at(i, 0);
    }
    return f;
}

std::vector<double> gaussian_load(const Axis1D &ax, double c, double den)
{
    if (ax.ne == 0) return std::vector<double>(1, 1.0);   // the missing axis of a 2D problem
    const int p = ax.p, ne = ax.ne;
    std::vector<double> t(ne + 2 * p + 1);
    for (int i = 0; i <= p; ++i) { t[i] = 0.0; t[ne + p + i] = ax.L; }
    for (int i = 1; i < ne; ++i) t[p + i] = ax.L * i / ne;
    std::vector<double> out(ax.m, 0.0);
    double gx[8], gw[8], N[5], dN[5];
    gauss_legendre(p + 1, gx, gw);
    for (int e = 0; e < ne; ++e) {
        double a = t[p + e], b = t[p + e + 1], h = b - a;
        for (int g = 0; g <= p; ++g) {
            double x = a + 0.5 * h * (1.0 + gx[g]), w = 0.5 * h * gw[g];
            local_basis(t, p + e, p, x, N, dN);
            double gv = w * std::exp(-(x - c) * (x - c) / den);
            for (int r = 0; r <= p; ++r) {
                int i = e + r - ax.off;
                if (i >= 0 && i < ax.m) out[i] += gv * N[r];
            }
        }
    }
    return out;
}

// fundamental solutions and transfer matrices for the boundaries in P.b
void fill_partition(const Factor &f, Partition &P)
{
    const int m = f.m, p = f.p, W = 2 * p + 1, S = P.S;
    P.phi.assign((size_t)m * p, 0.0);
    P.psi.assign((size_t)m * p, 0.0);
    P.Phi.assign((size_t)S * p * p, 0.0);
    P.Psi.assign((size_t)S * p * p, 0.0);
    auto L = [&](int i, int q) { return f.v[(size_t)i * W + (p - q)]; };   // l_q of row i
    auto U = [&](int i, int q) { return f.v[(size_t)i * W + (p + q)]; };   // u_q of row i
    auto D = [&](int i) { return f.v[(size_t)i * W + p]; };                // 1/u_0
    std::vector<double> w(m + 2 * p);
    for (int s = 0; s < S; ++s) {
        const int b0 = P.b[s], b1 = P.b[s + 1];
        for (int k = 0; k < p; ++k) {
            // forward fundamental solution with carry e_k (w_{b0-1-k} = 1)
            if (s > 0) {
                std::fill(w.begin(), w.end(), 0.0);
                auto W_ = [&](int i) -> double & { return w[i + p]; };   // index shift for i >= -p
                W_(b0 - 1 - k) = 1.0;
                for (int i = b0; i < b1; ++i) {
                    double acc = 0.0;
                    for (int q = 1; q <= p; ++q) acc -= L(i, q) * W_(i - q);
                    W_(i) = acc;
                    P.phi[(size_t)i * p + k] = acc;
                }
                for (int r = 0; r < p; ++r) P.Phi[((size_t)s * p + r) * p + k] = W_(b1 - 1 - r);
            }
            // backward fundamental solution with carry e_k (x_{b1+k} = 1)
            if (s < S - 1) {
                std::fill(w.begin(), w.end(), 0.0);
                auto X_ = [&](int i) -> double & { return w[i - b0 + p]; };
                std::vector<double> xs((size_t)(b1 - b0) + 2 * p, 0.0);
                auto XS = [&](int i) -> double & { return xs[(size_t)(i - b0)]; };
                XS(b1 + k) = 1.0;
                for (int i = b1 - 1; i >= b0; --i) {
                    double acc = 0.0;
                    for (int q = 1; q <= p; ++q) acc -= U(i, q) * XS(i + q);
                    XS(i) = acc * D(i);
                    P.psi[(size_t)i * p + k] = XS(i);
                }
                for (int r = 0; r < p; ++r) P.Psi[((size_t)s * p + r) * p + k] = XS(b0 + r);
                (void)X_;
            }
        }
    }
}

Partition partition_fixed(const Factor &f, int seg)
{
    const int S = (f.m + seg - 1) / seg;
    Partition Q;
    Q.m = f.m; Q.p = f.p; Q.S = S;
    Q.b.resize(S + 1);
    for (int s = 0; s < S; ++s) Q.b[s] = s * seg;
    Q.b[S] = f.m;
    fill_partition(f, Q);
    return Q;
}

std::pair<int, int> canonicalize_interior(Band &b)
{
    const int m = b.m, p = b.p, W = 2 * p + 1;
    if (m < 4 * p + 3) return {0, 0};
    const int mid = m / 2;
    double rmax = 0.0;
    for (int k = 0; k < W; ++k) rmax = std::max(rmax, std::fabs(b.v[(size_t)mid * W + k]));
    // quadrature of shifted elements reproduces the stencil only up to
    // rounding (~1e-14 of the row for 256 elements): compare at 1e-12
    auto close = [&](int i) {
        for (int k = 0; k < W; ++k) {
            const double a = b.v[(size_t)i * W + k], c = b.v[(size_t)mid * W + k];
            if (std::fabs(a - c) > 1e-12 * rmax) return false;
        }
        return true;
    };
    int lo = mid, hi = mid + 1;
    while (lo > 0 && close(lo - 1)) --lo;
    while (hi < m && close(hi)) ++hi;
    for (int i = lo; i < hi; ++i)
        for (int k = 0; k < W; ++k) b.v[(size_t)i * W + k] = b.v[(size_t)mid * W + k];
    return {lo, hi};
}

Partition partition(const Factor &f, int S, int align)
{
    const int m = f.m, p = f.p, W = 2 * p + 1;
    if (align < 1) align = 1;
    // fewer segments when the line is short: each segment >= max(p, align)
    while (S > 1 && m / S < std::max(p, align) + align) S /= 2;
    Partition P;
    P.m = m; P.p = p; P.S = S;
    P.b.resize(S + 1);
    for (int s = 0; s <= S; ++s) {
        int v = (int)((long long)m * s / S);
        if (s > 0 && s < S) v = v / align * align;
        P.b[s] = v;
    }
    fill_partition(f, P);
    return P;
}

}  // namespace ads
