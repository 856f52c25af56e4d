// Host check of the library's 1D set-up (Sec. 2 matrices, Appendix line
// solves), run by tests/test_host_setup.py on the CPU:
//   setup1d_check ne p natural d seg
// builds one axis with the library's own host code (setup1d.cpp) and prints
//   band M|K <m> <2p+1> values...   the 1D mass and stiffness bands
//   lohi <lo> <hi>                   Toeplitz interior rows
//   lu_resid <r>                     max |L U - (M + d K)| / max |M + d K|
//   part_err <e>                     partitioned solve with segments of `seg`
//                                    rows vs plain banded substitution, max
//                                    relative difference over three right-hand sides
// The partitioned solve below restates the segment algorithm from its
// definition (local substitutions with zero carry-in, carries through the
// transfer matrices, corrections by the fundamental solutions).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "setup1d.h"

namespace {

void print_band(const char *name, const ads::Band &b)
{
    std::printf("band %s %d %d", name, b.m, 2 * b.p + 1);
    for (double v : b.v) std::printf(" %.17g", v);
    std::printf("\n");
}

// plain forward then back substitution with the factor rows
// [l_p .. l_1 | 1/u_0 | u_1 .. u_p]
std::vector<double> plain_solve(const ads::Factor &f, const std::vector<double> &r)
{
    const int m = f.m, p = f.p, W = 2 * p + 1;
    std::vector<double> w(m), x(m);
    for (int i = 0; i < m; ++i) {
        double a = r[i];
        for (int k = 1; k <= p && i - k >= 0; ++k) a -= f.v[(size_t)i * W + p - k] * w[i - k];
        w[i] = a;
    }
    for (int i = m - 1; i >= 0; --i) {
        double a = w[i];
        for (int k = 1; k <= p && i + k < m; ++k) a -= f.v[(size_t)i * W + p + k] * x[i + k];
        x[i] = a * f.v[(size_t)i * W + p];
    }
    return x;
}

std::vector<double> partitioned_solve(const ads::Factor &f, const ads::Partition &P, const std::vector<double> &r)
{
    const int m = f.m, p = f.p, W = 2 * p + 1, S = P.S;
    std::vector<double> w(m), x(m);
    // forward: local substitution per segment, zero carry-in
    for (int s = 0; s < S; ++s)
        for (int i = P.b[s]; i < P.b[s + 1]; ++i) {
            double a = r[i];
            for (int k = 1; k <= p && i - k >= P.b[s]; ++k) a -= f.v[(size_t)i * W + p - k] * w[i - k];
            w[i] = a;
        }
    // carries c_s (last p values of the true w before segment s), then corrections
    std::vector<double> c(p, 0.0), t(p), n(p);
    std::vector<std::vector<double>> carry(S, std::vector<double>(p, 0.0));
    for (int s = 0; s + 1 < S; ++s) {
        for (int k = 0; k < p; ++k) t[k] = w[P.b[s + 1] - 1 - k];
        for (int k = 0; k < p; ++k) {
            double a = t[k];
            for (int j = 0; j < p; ++j) a += P.Phi[((size_t)s * p + k) * p + j] * c[j];
            n[k] = a;
        }
        c = n;
        carry[s + 1] = c;
    }
    for (int s = 0; s < S; ++s)
        for (int i = P.b[s]; i < P.b[s + 1]; ++i)
            for (int k = 0; k < p; ++k) w[i] += carry[s][k] * P.phi[(size_t)i * p + k];
    // backward: local substitution per segment, zero carry-in from the right
    for (int s = 0; s < S; ++s)
        for (int i = P.b[s + 1] - 1; i >= P.b[s]; --i) {
            double a = w[i];
            for (int k = 1; k <= p && i + k < P.b[s + 1]; ++k) a -= f.v[(size_t)i * W + p + k] * x[i + k];
            x[i] = a * f.v[(size_t)i * W + p];
        }
    std::vector<double> e(p, 0.0), h(p);
    std::vector<std::vector<double>> ecarry(S, std::vector<double>(p, 0.0));
    for (int s = S - 1; s > 0; --s) {
        for (int k = 0; k < p; ++k) h[k] = x[P.b[s] + k];
        for (int k = 0; k < p; ++k) {
            double a = h[k];
            for (int j = 0; j < p; ++j) a += P.Psi[((size_t)s * p + k) * p + j] * e[j];
            n[k] = a;
        }
        e = n;
        ecarry[s - 1] = e;
    }
    for (int s = 0; s < S; ++s)
        for (int i = P.b[s]; i < P.b[s + 1]; ++i)
            for (int k = 0; k < p; ++k) x[i] += ecarry[s][k] * P.psi[(size_t)i * p + k];
    return x;
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc != 6) {
        std::fprintf(stderr, "usage: %s ne p natural d seg\n", argv[0]);
        return 2;
    }
    const int ne = std::atoi(argv[1]), p = std::atoi(argv[2]), natural = std::atoi(argv[3]);
    const double d = std::atof(argv[4]);
    const int seg = std::atoi(argv[5]);
    const ads::Axis1D ax = ads::build_axis(ne, p, 1.0, natural != 0);
    print_band("M", ax.M);
    print_band("K", ax.K);
    std::printf("lohi %d %d\n", ax.lo, ax.hi);

    const ads::Factor f = ads::factor_axis(ax, d);
    const int m = ax.m, W = 2 * p + 1;
    // L U against A = M + d K, entry by entry inside the band
    double amax = 0.0, rmax = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = std::max(0, i - p); j <= std::min(m - 1, i + p); ++j) {
            const double a = ax.M.at(i, j - i) + d * ax.K.at(i, j - i);
            double lu = 0.0;
            for (int k = std::max(0, std::max(i, j) - p); k <= std::min(i, j); ++k) {
                const double l = k == i ? 1.0 : f.v[(size_t)i * W + p - (i - k)];
                const double u = k == j ? 1.0 / f.v[(size_t)k * W + p] : f.v[(size_t)k * W + p + (j - k)];
                lu += l * u;
            }
            amax = std::fmax(amax, std::fabs(a));
            rmax = std::fmax(rmax, std::fabs(lu - a));
        }
    std::printf("lu_resid %.3e\n", rmax / amax);

    const ads::Partition P = ads::partition_fixed(f, seg);
    double err = 0.0;
    for (int t = 0; t < 3; ++t) {
        std::vector<double> r(m);
        for (int i = 0; i < m; ++i) r[i] = std::sin(0.37 * (i + 1) * (t + 1)) + 0.01 * t * i;
        const std::vector<double> x0 = plain_solve(f, r), x1 = partitioned_solve(f, P, r);
        double nx = 0.0, nd = 0.0;
        for (int i = 0; i < m; ++i) {
            nx = std::fmax(nx, std::fabs(x0[i]));
            nd = std::fmax(nd, std::fabs(x1[i] - x0[i]));
        }
        err = std::fmax(err, nd / nx);
    }
    std::printf("segments %d\n", P.S);
    std::printf("part_err %.3e\n", err);
    return 0;
}
