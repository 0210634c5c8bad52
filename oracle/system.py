"""The collective-scattering linear system, App. I-C (Eq. final_linear_eqs)
with the block-diagonal T preconditioner of App. I-C/I-D.

Unknowns: outgoing coefficients s_i (shape (N, P)). The field incident on
scatterer i is a_i = a0_i + sum_{j != i} A_ij s_j with A_ij = xi(k(x_i - x_j))^T
(target i, source j), and s_i = T_i a_i. Multiplying Omega s = a0 by the
preconditioner M = diag(T_i) gives the system that is iterated:

    K s = b,   K = I - T A,   b = T a0.

The adjoint operator (App. IV, Omega^T) in the same preconditioned form is
K^T-like: (I - A^T T) mu = v with (A^T)_ij = (A_ji)^T = xi(k(x_j - x_i)).
Interactions are restricted to the neighbour list (all pairs when cutoff <= 0).

Optional coupling window (a parameter of this implementation, not of the
paper): window = (cutoff, taper) multiplies the block of a pair at distance d
by w(d) = 1 for d <= cutoff - taper and 0.5 (1 + cos(pi (d - cutoff + taper) /
taper)) up to the cutoff; window = None (or taper = 0) is the hard cutoff.
"""
import math

import numpy as np

from .geometry import neighbours
from .translation import xi_matrix

_WINDOW = [None]  # (cutoff, taper) in force for _block, set by the callers below


def coupling_weight(d, cutoff, taper):
    """Raised-cosine window of the pair coupling (1 inside cutoff - taper)."""
    if not taper or cutoff <= 0:
        return 1.0
    d0 = cutoff - taper
    if d <= d0:
        return 1.0
    if d >= cutoff:
        return 0.0
    return 0.5 * (1.0 + math.cos(math.pi * (d - d0) / taper))


def _block(nmax, k, xt, xs):
    d = np.asarray(xt, dtype=np.float64) - np.asarray(xs, dtype=np.float64)
    B = xi_matrix(nmax, nmax, k, d).T
    if _WINDOW[0] is not None:
        B = B * coupling_weight(float(np.linalg.norm(d)), *_WINDOW[0])
    return B


class window:
    """Context manager: `with window(cutoff, taper): ...` applies the coupling
    window inside the block."""

    def __init__(self, cutoff, taper):
        self.w = (cutoff, taper) if taper else None

    def __enter__(self):
        self.prev = _WINDOW[0]
        _WINDOW[0] = self.w
        return self

    def __exit__(self, *a):
        _WINDOW[0] = self.prev


def apply_A(nmax, k, pos, x, nbr):
    """(A x)_i = sum_{j in N(i)} A_ij x_j."""
    row_ptr, col = nbr
    N, P = x.shape
    y = np.zeros_like(x, dtype=np.complex128)
    for i in range(N):
        acc = np.zeros(P, dtype=np.complex128)
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            acc += _block(nmax, k, pos[i], pos[j]) @ x[j]
        y[i] = acc
    return y


def apply_AT(nmax, k, pos, x, nbr):
    """(A^T x)_i = sum_{j in N(i)} (A_ji)^T x_j (neighbour lists are symmetric)."""
    row_ptr, col = nbr
    N, P = x.shape
    y = np.zeros_like(x, dtype=np.complex128)
    for i in range(N):
        acc = np.zeros(P, dtype=np.complex128)
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            acc += _block(nmax, k, pos[j], pos[i]).T @ x[j]
        y[i] = acc
    return y


def apply_K(nmax, k, pos, tdiag, x, nbr):
    """y = x - T (A x)  (the preconditioned Maxwell operator M Omega)."""
    return x - tdiag * apply_A(nmax, k, pos, x, nbr)


def apply_KT(nmax, k, pos, tdiag, x, nbr):
    """y = x - A^T (T x)  (adjoint of apply_K under the bilinear form)."""
    return x - apply_AT(nmax, k, pos, tdiag * x, nbr)


def apply_K_rows(nmax, k, pos, tdiag, x, nbr, rows):
    """apply_K evaluated only at the target rows listed (for sampled checks of
    large problems)."""
    row_ptr, col = nbr
    P = x.shape[1]
    out = np.zeros((len(rows), P), dtype=np.complex128)
    for r, i in enumerate(rows):
        acc = np.zeros(P, dtype=np.complex128)
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            acc += _block(nmax, k, pos[i], pos[j]) @ x[j]
        out[r] = x[i] - tdiag[i] * acc
    return out


def apply_KT_rows(nmax, k, pos, tdiag, x, nbr, rows):
    row_ptr, col = nbr
    P = x.shape[1]
    out = np.zeros((len(rows), P), dtype=np.complex128)
    for r, i in enumerate(rows):
        acc = np.zeros(P, dtype=np.complex128)
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            acc += _block(nmax, k, pos[j], pos[i]).T @ (tdiag[j] * x[j])
        out[r] = x[i] - acc
    return out


def dense_A(nmax, k, pos, nbr):
    row_ptr, col = nbr
    N = pos.shape[0]
    P = 2 * nmax * (nmax + 2)
    A = np.zeros((N * P, N * P), dtype=np.complex128)
    for i in range(N):
        for j in col[row_ptr[i]:row_ptr[i + 1]]:
            A[i * P:(i + 1) * P, j * P:(j + 1) * P] = _block(nmax, k, pos[i], pos[j])
    return A


def dense_K(nmax, k, pos, tdiag, nbr):
    A = dense_A(nmax, k, pos, nbr)
    t = tdiag.reshape(-1)
    return np.eye(A.shape[0], dtype=np.complex128) - t[:, None] * A


def solve_dense(nmax, k, pos, tdiag, a0, cutoff=0.0):
    """Direct solve of K s = T a0 by LU (numpy/LAPACK as the library step)."""
    nbr = neighbours(pos, cutoff)
    K = dense_K(nmax, k, pos, tdiag, nbr)
    b = (tdiag * a0).reshape(-1)
    return np.linalg.solve(K, b).reshape(a0.shape)


def gmres(matvec, b, tol=1e-13, restart=50, maxiter=2000):
    """Restarted GMRES(m), x0 = 0, Arnoldi with modified Gram-Schmidt and Givens
    rotations (Saad, Iterative Methods, Alg. 6.9 / 6.11). Stops when the true
    relative residual ||b - K x|| / ||b|| <= tol. Returns (x, iterations, relres)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, 0.0
    its = 0
    r = b.copy()
    while True:
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or its >= maxiter:
            return x, its, beta / bnorm
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        jlast = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            # rotation G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]] zeroes H[i+1, i]
            for i in range(j):  # apply the previous rotations to column j
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            cs[j] = H[j, j] / den if den else 1.0
            sn[j] = H[j + 1, j] / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            jlast = j + 1
            if abs(g[j + 1]) / bnorm <= tol * 0.5 or its >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:jlast, :jlast]), g[:jlast])
        x = x + V[:jlast].T @ y
        r = b - matvec(x)


def solve_gmres(nmax, k, pos, tdiag, a0, cutoff=0.0, tol=1e-13, restart=50, maxiter=5000):
    nbr = neighbours(pos, cutoff)
    shape = a0.shape
    b = (tdiag * a0).reshape(-1)

    def mv(v):
        return apply_K(nmax, k, pos, tdiag, v.reshape(shape), nbr).reshape(-1)

    x, its, rr = gmres(mv, b, tol=tol, restart=restart, maxiter=maxiter)
    return x.reshape(shape), its, rr


# ----------------------------------------------------------------------------
# Full per-scatterer T-blocks (App. I-B, Eq. def_tmatrix: s_i = T_i a_i with T_i a
# P x P matrix, e.g. a null-field cylinder). The same system with block-diagonal
# T = diag(T_1 .. T_N) instead of a diagonal:
#     K = I - T A,  b = T a0;  adjoint (transpose) K^T = I - A^T T^T.
# Tb has shape (N, P, P), rows = outgoing index, columns = incident index.
# ----------------------------------------------------------------------------

def apply_K_blocks(nmax, k, pos, Tb, x, nbr):
    """y_i = x_i - T_i (A x)_i."""
    Ax = apply_A(nmax, k, pos, x, nbr)
    return x - np.einsum("nab,nb->na", Tb, Ax)


def apply_KT_blocks(nmax, k, pos, Tb, x, nbr):
    """y = x - A^T (T^T x), the transpose of apply_K_blocks."""
    return x - apply_AT(nmax, k, pos, np.einsum("nba,nb->na", Tb, x), nbr)


def dense_K_blocks(nmax, k, pos, Tb, nbr):
    A = dense_A(nmax, k, pos, nbr)
    N, P, _ = Tb.shape
    Tfull = np.zeros((N * P, N * P), dtype=np.complex128)
    for i in range(N):
        Tfull[i * P:(i + 1) * P, i * P:(i + 1) * P] = Tb[i]
    return np.eye(N * P, dtype=np.complex128) - Tfull @ A


def solve_dense_blocks(nmax, k, pos, Tb, a0, cutoff=0.0):
    """Direct solve of (I - T A) s = T a0 with full T-blocks (LU, the library step)."""
    nbr = neighbours(pos, cutoff)
    K = dense_K_blocks(nmax, k, pos, Tb, nbr)
    b = np.einsum("nab,nb->na", Tb, a0).reshape(-1)
    return np.linalg.solve(K, b).reshape(a0.shape)
