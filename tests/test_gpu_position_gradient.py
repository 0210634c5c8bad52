"""GPU position gradient of the point figure of merit (App. IV with the in-plane positions
as the geometry parameters) against the oracle's central differences of direct solves."""
import math

import numpy as np
import pytest

from gpu_common import K0, atoms, ctx, rel_l2
from oracle import adjoint, incident, mie
from paper_2107_09879_b300 import _lib
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _grad_case(nx, ny, nmax, cutoff, taper, beta_deg, xf):
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.1, 0.22, 11 + nx)
    beta = math.radians(beta_deg)
    A = incident.beta_hat(beta, 0.0).astype(complex)
    dirs = np.array([[beta, 0.0]])
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, A[None])
    T, dT = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax, with_dr=True)
    opts = _lib.make_opts(tol=1e-12, cutoff=cutoff, taper=taper, precision=0, path=_lib.PATH_LATTICE,
                          lattice_nx=nx, lattice_ny=ny, lattice_pitch=0.5)
    s, info, sol, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
    assert rc == 0
    Einc = incident.planewave_field(K0, beta, 0.0, A, xf[None])[0]
    fom, v = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, Einc)
    Ef = np.ascontiguousarray(Einc + ctx().tmat_field(pos, 1.0, 1.0, nmax, s[0], xf[None])[0])
    _, mu, _ = ctx().tmat_adjoint(sol, v, dT, want_mu=True)
    kinc = K0 * incident.direction(beta, 0.0)
    da0x = np.ascontiguousarray(1j * kinc[0] * a0[0])
    da0y = np.ascontiguousarray(1j * kinc[1] * a0[0])
    g = ctx().tmat_position_gradient(sol, mu, xf, Ef, da0x, da0y)
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    a0_of = lambda p: incident.planewave_incident(nmax, K0, p, beta, 0.0, A)
    go = adjoint.position_gradient_fd(nmax, K0, pos, To, a0_of, xf, Einc, h=1e-5, cutoff=cutoff, taper=taper)
    return g, go, sol, mu, xf, Ef


@pytest.mark.parametrize("fft", [True, False])
@pytest.mark.parametrize("nx,ny,nmax,cutoff,taper,beta", [(4, 3, 3, 1.2, 1.2, 10.0), (3, 3, 2, 0.0, 0.0, 0.0),
                                                         (5, 2, 3, 1.6, 0.6, 20.0)])
def test_position_gradient_vs_oracle(nx, ny, nmax, cutoff, taper, beta, fft):
    """Every pair or a windowed cutoff, normal and oblique incidence (the incident term),
    ragged lattices, derivative operators by FFT convolution or by the direct kernel: the
    adjoint gradient against central differences of direct solves."""
    xf = np.array([0.6, 0.3, 2.5])
    ctx().set_lattice_fft(fft)
    try:
        g, go, *_ = _grad_case(nx, ny, nmax, cutoff, taper, beta, xf)
    finally:
        ctx().set_lattice_fft(True)
    assert np.max(np.abs(go)) > 1e-3
    assert rel_l2(g, go) <= 1e-6


def test_position_gradient_neighbour_path_not_supported():
    pos = W.lattice_positions(2, 2)
    T = ctx().tmat_build(atoms(np.full(4, 0.15)), 1.0, 1.0, 2)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, 2, np.array([[0.0, 0.0]]), np.array([[1.0, 0, 0]], complex))
    s, info, sol, rc = ctx().tmat_solve(pos, 1.0, 1.0, 2, T, a0, _lib.make_opts(tol=1e-10, precision=0), keep=True)
    mu = np.zeros_like(s[0])
    with pytest.raises(_lib.TMatError):
        ctx().tmat_position_gradient(sol, mu, np.array([0.0, 0.0, 2.0]), np.zeros(3, complex))
