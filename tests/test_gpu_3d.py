"""General 3-D positions (no common plane): the neighbour-path apply with full blocks, the
solve and the adjoint radius gradient against the oracle (which is 3-D throughout)."""
import math

import numpy as np
import pytest

from gpu_common import C64_APPLY_TOL, K0, atoms, ctx, rand_c, rel_l2
from oracle import adjoint, geometry, incident, mie, system
from paper_2107_09879_b300 import _lib
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _positions(nx, ny, seed, dz=0.3):
    """A lattice with every scatterer lifted by a seeded height in [-dz, dz] (a corrugated
    array: no two layers share a plane)."""
    pos = W.lattice_positions(nx, ny).copy()
    pos[:, 2] = (W.uniform_radii(nx * ny, 0.0, 1.0, seed) - 0.5) * 2 * dz
    return pos


@pytest.mark.parametrize("nmax,nx,ny,cutoff,taper,R", [(3, 4, 3, 1.2, 0.0, 1), (2, 3, 3, 0.0, 0.0, 3),
                                                       (4, 3, 2, 1.4, 0.6, 2), (5, 2, 2, 0.0, 0.0, 1)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_apply_3d_vs_oracle(nmax, nx, ny, cutoff, taper, R, op):
    pos = _positions(nx, ny, 3 + nmax)
    r = W.uniform_radii(nx * ny, 0.08, 0.2, 9 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 17 + nmax)
    nbr = geometry.neighbours(pos, cutoff)
    rp, col = ctx().tmat_neighbors(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    with system.window(cutoff, taper):
        ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(R)])
    y64 = ctx().tmat_apply(op, _lib.PREC_FP64, pos, K0, nmax, T, rp, col, x, cutoff=cutoff, taper=taper)
    y32 = ctx().tmat_apply(op, _lib.PREC_MIXED, pos, K0, nmax, T, rp, col, x, cutoff=cutoff, taper=taper)
    assert rel_l2(y64, ref) <= 1e-12
    assert rel_l2(y32, ref) <= C64_APPLY_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_and_radius_gradient_3d(precision):
    nmax, cutoff = 3, 0.0
    pos = _positions(3, 2, 21)
    r = W.uniform_radii(6, 0.1, 0.22, 7)
    xf = np.array([0.5, 0.25, 3.0])
    A = np.array([1.0, 0.0, 0.0], dtype=complex)
    Einc = incident.planewave_field(K0, 0.0, 0.0, A, xf[None])[0]
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), A[None])
    T, dT = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax, with_dr=True)
    opts = _lib.make_opts(tol=1e-12 if precision == 0 else 1e-9, cutoff=cutoff, precision=precision)
    s, info, sol, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
    assert rc == 0
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    a0o = incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, A)  # the oracle's own
    so = system.solve_dense(nmax, K0, pos, To, a0o, cutoff)
    assert rel_l2(s[0], so) <= (1e-9 if precision == 0 else 1e-6)
    fom, v = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, Einc)
    vo = adjoint.adjoint_source(nmax, K0, pos, so, xf, Einc)
    grad, mu, _ = ctx().tmat_adjoint(sol, v, dT, want_mu=True)
    dTo = np.array([mie.tmatrix_diag_dr(nmax, K0, x, 2.0) for x in r])
    go, _ = adjoint.radius_gradient(nmax, K0, pos, To, dTo, a0o, so, vo, cutoff=cutoff)
    assert rel_l2(grad, go) <= (1e-9 if precision == 0 else 1e-6)


def test_lattice_path_needs_a_plane():
    pos = _positions(3, 3, 5)
    T = ctx().tmat_build(atoms(np.full(9, 0.1)), 1.0, 1.0, 2)
    a0 = np.ones((1, 9, 16), complex)
    opts = _lib.make_opts(tol=1e-8, path=_lib.PATH_LATTICE, lattice_nx=3, lattice_ny=3, lattice_pitch=0.5)
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve(pos, 1.0, 1.0, 2, T, a0, opts)
    assert e.value.code == _lib.EINVAL
