"""Pins of the oracle's position gradient of the point figure of merit (App. IV with the
in-plane positions as the geometry parameters): step convergence of the central
differences, mirror symmetry of a symmetric array, and translation invariance (moving
every scatterer and the focus together leaves the figure of merit unchanged under normal
incidence)."""
import math

import numpy as np

from oracle import adjoint, incident, mie, system

K0 = 2 * math.pi
NMAX = 2


def _setup(nx=3, ny=3, beta=0.0, offset=(0.0, 0.0)):
    iy, ix = np.divmod(np.arange(nx * ny), nx)
    pos = np.zeros((nx * ny, 3))
    pos[:, 0] = (ix - (nx - 1) / 2) * 0.5 + offset[0]
    pos[:, 1] = (iy - (ny - 1) / 2) * 0.5 + offset[1]
    T = np.array([mie.tmatrix_diag(NMAX, K0, 0.18, 2.0) for _ in range(nx * ny)])
    A = np.array([math.cos(beta), 0.0, -math.sin(beta)], dtype=complex)
    a0_of = lambda p: incident.planewave_incident(NMAX, K0, p, beta, 0.0, A)
    x_f = np.array([offset[0] + 0.1, offset[1] - 0.05, 3.0])
    E_inc_f = incident.planewave_field(K0, beta, 0.0, A, x_f[None, :])[0]
    return pos, T, a0_of, x_f, E_inc_f


def test_step_convergence():
    pos, T, a0_of, x_f, E = _setup(3, 2, beta=math.radians(10))
    g1 = adjoint.position_gradient_fd(NMAX, K0, pos, T, a0_of, x_f, E, h=1e-5)
    g2 = adjoint.position_gradient_fd(NMAX, K0, pos, T, a0_of, x_f, E, h=2e-5)
    assert np.linalg.norm(g1) > 1e-3
    assert np.linalg.norm(g1 - g2) <= 1e-7 * np.linalg.norm(g1)


def test_mirror_symmetry():
    """3 x 3 array, normal incidence (x-polarised), focus on the axis: mirroring x -> -x
    maps the array and the problem onto themselves, so d/dx flips sign between mirror
    partners and vanishes on the mirror line; d/dy is even."""
    pos, T, a0_of, _, E = _setup(3, 3)
    x_f = np.array([0.0, 0.0, 3.0])
    E = incident.planewave_field(K0, 0.0, 0.0, np.array([1, 0, 0], complex), x_f[None, :])[0]
    g = adjoint.position_gradient_fd(NMAX, K0, pos, T, a0_of, x_f, E)
    scale = np.max(np.abs(g))
    assert scale > 1e-3
    for i in range(9):
        j = [q for q in range(9) if np.allclose(pos[q, :2], [-pos[i, 0], pos[i, 1]])][0]
        assert abs(g[i, 0] + g[j, 0]) <= 1e-6 * scale
        assert abs(g[i, 1] - g[j, 1]) <= 1e-6 * scale


def test_translation_invariance():
    """Normal incidence: the incident coefficients and the incident field at the focus are
    unchanged by in-plane translations, so sum_i dFoM/dx_i = -dFoM/dx_f."""
    pos, T, a0_of, x_f, E = _setup(3, 2)
    g = adjoint.position_gradient_fd(NMAX, K0, pos, T, a0_of, x_f, E)
    s = system.solve_dense(NMAX, K0, pos, T, a0_of(pos))
    gf = adjoint.focus_gradient_fd(NMAX, K0, pos, s, x_f, E)
    assert np.linalg.norm(g.sum(axis=0) + gf) <= 1e-7 * np.linalg.norm(gf) + 1e-9
    assert np.linalg.norm(gf) > 1e-3
