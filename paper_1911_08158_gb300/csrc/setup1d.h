// setup1d.h -- host FP64 construction of the 1D spline operators (Sec. 2,
// Appendix) in band storage, and their pivot-free banded LU factors.
#pragma once
#include <utility>
#include <vector>

namespace ads {

// Band of an m x m matrix with half-bandwidth p: row i holds A[i][i+k] at
// column (k + p), k = -p..p; entries outside the matrix are 0.
struct Band {
    int m = 0, p = 0;
    std::vector<double> v;   // m * (2p+1)
    double &at(int i, int k) { return v[(size_t)i * (2 * p + 1) + (k + p)]; }
    double at(int i, int k) const { return v[(size_t)i * (2 * p + 1) + (k + p)]; }
};

// 1D operators of one axis on its unknowns: the interior functions
// (Dirichlet restriction, off = 1) or all of them (natural boundary, off = 0).
struct Axis1D {
    int ne = 0, p = 0, n = 0, m = 0, off = 1;
    double L = 1.0;
    Band M, K, B;            // (N_a,N_c), (N'_a,N'_c), (N'_a,N_c)
    Band Bt;                 // B^T (= -B up to rounding with the Dirichlet restriction)
    int lo = 0, hi = 0;      // rows [lo, hi) of M, K and B are the Toeplitz interior row
};

// Factor row layout used by the device sweeps, 2p+1 entries per row:
//   [ l_p .. l_1 | 1/u_0 | u_1 .. u_p ]
// with A = L U, L unit lower (l_k = L[i][i-k]), U upper (u_k = U[i][i+k]).
// Forward:  w_i = r_i - sum_k l_k w_{i-k};  backward: x_i = (w_i - sum_k u_k x_{i+k}) / u_0.
struct Factor {
    int m = 0, p = 0;
    std::vector<double> v;   // m * (2p+1)
};

// Partitioned line solve (segment-parallel substitution).  A line of length
// m is cut into S segments [b_s, b_{s+1}) (lengths >= p, starts multiples of
// `align`).  Each segment is solved with zero carry-in; the true solution is
// the local one plus a combination of fundamental solutions that depend only
// on the factors, hence are shared by every line:
//   forward  (L w = r): carry c_s[k] = w_{b_s-1-k};   w = w_loc + sum_k c_s[k] phi[i][k]
//            c_{s+1} = t_s + Phi_s c_s,  t_s[k] = w_loc_{b_{s+1}-1-k}
//   backward (U x = w): carry e_s[k] = x_{b_{s+1}+k}; x = x_loc + sum_k e_s[k] psi[i][k]
//            e_{s-1} = h_s + Psi_s e_s,  h_s[k] = x_loc_{b_s+k}
struct Partition {
    int m = 0, p = 0, S = 1;
    std::vector<int> b;          // S+1 boundaries
    std::vector<double> phi;     // m*p (zero on segment 0)
    std::vector<double> psi;     // m*p (zero on the last segment)
    std::vector<double> Phi;     // S*p*p, Phi[s][k][j]
    std::vector<double> Psi;     // S*p*p, Psi[s][k][j]
};
Partition partition(const Factor &f, int S, int align);
// Segments of fixed width `seg` (the last one may be shorter): b_s = s*seg.
Partition partition_fixed(const Factor &f, int seg);

// Interior rows of the uniform-grid 1D matrices are Toeplitz (same stencil
// row shifted).  Rows [lo, hi) that agree with the middle row up to the
// quadrature's rounding (1e-12 of the row) are set to exactly that row, so
// that kernels may keep one interior row in registers.  Returns {lo, hi}.
std::pair<int, int> canonicalize_interior(Band &b);

void gauss_legendre(int q, double *x, double *w);
Axis1D build_axis(int ne, int p, double L, bool natural = false);
// The axis of a 2D problem's missing dimension: one constant function, M = [1],
// K = B = [0] (band width of degree p), so 3D operators act as their 2D ones.
Axis1D trivial_axis(int p);
// A = M + d K, factored
Factor factor_axis(const Axis1D &ax, double d);
// interior load (exp(-(x-c)^2/den), N_i) with the (p+1)-point rule
std::vector<double> gaussian_load(const Axis1D &ax, double c, double den);

}  // namespace ads
