"""Adjoint sensitivity of a point figure of merit, App. IV.

Figure of merit (App. IV, Eq. performance_metric with sigma a point detector and
f = |.|^2 summed over the three Cartesian components; reading: the total field
E = E_inc + E_sca at the focal point x_f):
    FoM = sum_c |E_c(x_f)|^2,  E_c = E_inc,c(x_f) + sum_i s_i^T Phi_c(k(x_f - x_i)).
Its differential is dFoM = 2 Re[ v^T ds ] with v_i = sum_c conj(E_c) Phi_c(k(x_f - x_i))
(the Wirtinger derivative d|z|^2/dz = conj(z); reading of f').

Position gradient (App. IV with the in-plane positions as the geometry parameters):
dFoM/d(x_i, y_i) by central differences of the figure of merit, every side a direct
solve (`position_gradient_fd`), the derivative by its definition for small arrays.

Geometry gradient (App. IV, Eq. grad_geometry_overlap): only the diagonal
blocks of Omega depend on the radius. With the preconditioned unknowns
s = T e, e = a0 + A s, and the adjoint solve
    (I - A^T T) mu = v        (Omega^T lambda = v with lambda = T^{-1}... , no inverse needed),
the radius gradient is
    dFoM/dr_i = 2 Re[ sum_n mu_{i,n} (dT_{i,n}/dr_i) e_{i,n} ].
"""
import numpy as np

from .system import apply_A, apply_KT, gmres
from .geometry import neighbours
from .vswf import vswf


def total_field_at(nmax, k, pos, s, x_f, E_inc_f):
    E = np.array(E_inc_f, dtype=np.complex128).copy()
    for i in range(pos.shape[0]):
        E += s[i] @ vswf(nmax, k, np.asarray(x_f) - pos[i])
    return E


def fom(nmax, k, pos, s, x_f, E_inc_f):
    E = total_field_at(nmax, k, pos, s, x_f, E_inc_f)
    return float(np.sum(np.abs(E) ** 2))


def adjoint_source(nmax, k, pos, s, x_f, E_inc_f):
    """v (N, P): v_{i,n} = sum_c conj(E_c(x_f)) Phi_{n,c}(k(x_f - x_i))."""
    E = total_field_at(nmax, k, pos, s, x_f, E_inc_f)
    v = np.zeros(s.shape, dtype=np.complex128)
    for i in range(pos.shape[0]):
        v[i] = vswf(nmax, k, np.asarray(x_f) - pos[i]) @ np.conj(E)
    return v


def radius_gradient(nmax, k, pos, tdiag, dtdiag_dr, a0, s, v, cutoff=0.0, tol=1e-13, mu=None):
    """dFoM/dr for every scatterer given the forward solution s and the adjoint
    source v. Solves (I - A^T T) mu = v by GMRES unless mu is given."""
    nbr = neighbours(pos, cutoff)
    shape = s.shape
    if mu is None:
        def mv(x):
            return apply_KT(nmax, k, pos, tdiag, x.reshape(shape), nbr).reshape(-1)
        mu, _, _ = gmres(mv, v.reshape(-1), tol=tol)
        mu = mu.reshape(shape)
    e = a0 + apply_A(nmax, k, pos, s, nbr)
    return 2.0 * np.real(np.sum(mu * dtdiag_dr * e, axis=1)), mu


def position_gradient_fd(nmax, k, pos, tdiag, a0_of, x_f, E_inc_f, h=1e-5, cutoff=0.0, taper=0.0):
    """dFoM/d(x_i, y_i) for every scatterer by central differences of the figure of merit,
    each side a direct (LU) solve of the system with that one position moved: the derivative
    by its definition, for small arrays. a0_of(pos) -> (N, P) incident coefficients of the
    moved positions (the incident field at x_f does not depend on them). Returns (N, 2)."""
    from .system import solve_dense, window

    pos = np.asarray(pos, dtype=np.float64)

    def F(p):
        with window(cutoff, taper):
            s = solve_dense(nmax, k, p, tdiag, a0_of(p), cutoff)
        return fom(nmax, k, p, s, x_f, E_inc_f)

    g = np.zeros((pos.shape[0], 2))
    for i in range(pos.shape[0]):
        for d in range(2):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            g[i, d] = (F(pp) - F(pm)) / (2.0 * h)
    return g


def focus_gradient_fd(nmax, k, pos, s, x_f, E_inc_f, h=1e-5):
    """dFoM/d(x_f, y_f) with s and the incident field held fixed (central differences)."""
    g = np.zeros(2)
    for d in range(2):
        xp, xm = np.array(x_f, dtype=np.float64), np.array(x_f, dtype=np.float64)
        xp[d] += h
        xm[d] -= h
        g[d] = (fom(nmax, k, pos, s, xp, E_inc_f) - fom(nmax, k, pos, s, xm, E_inc_f)) / (2.0 * h)
    return g
