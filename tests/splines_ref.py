"""Independent 1D reference for the oracle pins: SciPy's B-spline evaluator
and NumPy's Gauss-Legendre rule.  Nothing here comes from the oracle."""
import numpy as np
from scipy.interpolate import BSpline


def knots(ne, p, L=1.0):
    return np.r_[[0.0] * p, np.linspace(0.0, L, ne + 1), [L] * p]


def basis_funcs(ne, p, L=1.0):
    t = knots(ne, p, L)
    n = ne + p
    return [BSpline(t, np.eye(n)[i], p, extrapolate=False) for i in range(n)], t


def mats(ne, p, L=1.0):
    """Full 1D M, K, B (B[a,c] = (N'_a, N_c)) by SciPy evaluation + NumPy Gauss."""
    fs, t = basis_funcs(ne, p, L)
    n = ne + p
    g, w = np.polynomial.legendre.leggauss(p + 1)
    M = np.zeros((n, n)); K = np.zeros((n, n)); B = np.zeros((n, n))
    for e in range(ne):
        a, b = L * e / ne, L * (e + 1) / ne
        x = 0.5 * (a + b) + 0.5 * (b - a) * g
        ww = 0.5 * (b - a) * w
        V = np.nan_to_num(np.array([f(x) for f in fs]))
        D = np.nan_to_num(np.array([f.derivative()(x) for f in fs]))
        M += (V * ww) @ V.T
        K += (D * ww) @ D.T
        B += (D * ww) @ V.T
    return M, K, B


def restricted(ne, p, L=1.0):
    M, K, B = mats(ne, p, L)
    s = slice(1, -1)
    return M[s, s], K[s, s], B[s, s]


def load1d(ne, p, c, den, L=1.0):
    """Interior 1D load (exp(-(x-c)^2/den), N_i) with the same (p+1)-point rule."""
    fs, t = basis_funcs(ne, p, L)
    g, w = np.polynomial.legendre.leggauss(p + 1)
    out = np.zeros(ne + p)
    for e in range(ne):
        a, b = L * e / ne, L * (e + 1) / ne
        x = 0.5 * (a + b) + 0.5 * (b - a) * g
        ww = 0.5 * (b - a) * w * np.exp(-(x - c) ** 2 / den)
        V = np.nan_to_num(np.array([f(x) for f in fs]))
        out += V @ ww
    return out[1:-1]


def kron3(Ax, Ay, Az):
    """Operator on x-fastest [z][y][x] flattening: A_z (x) A_y (x) A_x in NumPy order."""
    return np.kron(np.kron(Az, Ay), Ax)


def tables(ne, p, L=1.0):
    """Per-element Gauss points: values V[e, g, b] and derivatives D[e, g, b] of
    the p+1 functions e..e+p that live on element e, weights W[e, g]."""
    fs, t = basis_funcs(ne, p, L)
    g, w = np.polynomial.legendre.leggauss(p + 1)
    V = np.zeros((ne, p + 1, p + 1)); D = np.zeros_like(V); W = np.zeros((ne, p + 1))
    for e in range(ne):
        a, b = L * e / ne, L * (e + 1) / ne
        x = 0.5 * (a + b) + 0.5 * (b - a) * g
        W[e] = 0.5 * (b - a) * w
        for k in range(p + 1):
            V[e, :, k] = np.nan_to_num(fs[e + k](x))
            D[e, :, k] = np.nan_to_num(fs[e + k].derivative()(x))
    return V, D, W


def elastic_dense(ne, p, lam, mu, L=(1.0, 1.0, 1.0), natural=False):
    """Dense elasticity stiffness on the unknowns (interior DOFs with the
    Dirichlet restriction, every DOF with natural=True), assembled by direct
    3D quadrature of  mu (d_ab grad phi_A . grad phi_B + d_b phi_A d_a phi_B)
    + lam d_a phi_A d_b phi_B  (the bilinear form 2mu e(w):e(u) + lam div w div u
    for w = phi_A e_a, u = phi_B e_b).  Component-major, x fastest."""
    T = [tables(ne[a], p, L[a]) for a in range(3)]
    n = [ne[a] + p for a in range(3)]
    off = 0 if natural else 1
    m = [v - 2 * off for v in n]
    N = m[0] * m[1] * m[2]
    S = np.zeros((3 * N, 3 * N))
    q = p + 1
    for ez in range(ne[2]):
        for ey in range(ne[1]):
            for ex in range(ne[0]):
                # local functions (bx, by, bz) -> interior global index or -1
                idx = []
                for bz in range(q):
                    for by in range(q):
                        for bx in range(q):
                            i, j, k = ex + bx - off, ey + by - off, ez + bz - off
                            ok = 0 <= i < m[0] and 0 <= j < m[1] and 0 <= k < m[2]
                            idx.append((k * m[1] + j) * m[0] + i if ok else -1)
                idx = np.array(idx)
                for gz in range(q):
                    for gy in range(q):
                        for gx in range(q):
                            w = T[0][2][ex, gx] * T[1][2][ey, gy] * T[2][2][ez, gz]
                            vx, dx = T[0][0][ex, gx], T[0][1][ex, gx]
                            vy, dy = T[1][0][ey, gy], T[1][1][ey, gy]
                            vz, dz = T[2][0][ez, gz], T[2][1][ez, gz]
                            G = np.stack([
                                np.einsum("k,j,i->kji", vz, vy, dx).ravel(),
                                np.einsum("k,j,i->kji", vz, dy, vx).ravel(),
                                np.einsum("k,j,i->kji", dz, vy, vx).ravel()])   # (3, q^3)
                            keep = idx >= 0
                            Gk, I = G[:, keep], idx[keep]
                            gg = Gk.T @ Gk
                            for a in range(3):
                                for b in range(3):
                                    blk = mu * np.outer(Gk[b], Gk[a]) + lam * np.outer(Gk[a], Gk[b])
                                    if a == b:
                                        blk = blk + mu * gg
                                    S[np.ix_(a * N + I, b * N + I)] += w * blk
    return S


def elastic_dense_2d(ne, p, lam, mu, L=(1.0, 1.0)):
    """Dense plane-strain elasticity stiffness (components x, y) on the
    interior DOFs of a 2D spline space, by direct 2D quadrature of
    2 mu e(w):e(u) + lam div w div u.  Component-major, x fastest."""
    T = [tables(ne[a], p, L[a]) for a in range(2)]
    m = [ne[a] + p - 2 for a in range(2)]
    N = m[0] * m[1]
    S = np.zeros((2 * N, 2 * N))
    q = p + 1
    for ey in range(ne[1]):
        for ex in range(ne[0]):
            idx = []
            for by in range(q):
                for bx in range(q):
                    i, j = ex + bx - 1, ey + by - 1
                    idx.append(j * m[0] + i if 0 <= i < m[0] and 0 <= j < m[1] else -1)
            idx = np.array(idx)
            keep = idx >= 0
            I = idx[keep]
            for gy in range(q):
                for gx in range(q):
                    w = T[0][2][ex, gx] * T[1][2][ey, gy]
                    vx, dx = T[0][0][ex, gx], T[0][1][ex, gx]
                    vy, dy = T[1][0][ey, gy], T[1][1][ey, gy]
                    G = np.stack([np.outer(vy, dx).ravel(), np.outer(dy, vx).ravel()])[:, keep]   # grad of each function
                    gg = G.T @ G
                    for a in range(2):
                        for b in range(2):
                            blk = mu * np.outer(G[b], G[a]) + lam * np.outer(G[a], G[b])
                            if a == b:
                                blk = blk + mu * gg
                            S[np.ix_(a * N + I, b * N + I)] += w * blk
    return S
