"""GPU parity with the raised-cosine coupling window (taper) against the oracle."""
import math

import numpy as np
import pytest

from gpu_common import C64_APPLY_TOL, K0, atoms, ctx, rand_c, rel_l2
from oracle import incident, geometry, mie, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cutoff,taper", [(1.6, 1.6), (2.1, 0.7), (1.2, 0.5)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_windowed_apply_both_paths(cutoff, taper, op):
    nx, ny, nmax = 9, 8, 3
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 5)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((2, nx * ny, T.shape[1]), 6)
    nbr = geometry.neighbours(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    with system.window(cutoff, taper):
        ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(2)])
    rp, col = ctx().tmat_neighbors(pos, cutoff)
    for prec, bound in ((0, 1e-12), (1, C64_APPLY_TOL)):
        y = ctx().tmat_apply(op, prec, pos, K0, nmax, T, rp, col, x, cutoff=cutoff, taper=taper)
        assert rel_l2(y, ref) <= bound
        y = ctx().tmat_apply_lattice(op, prec, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=taper)
        assert rel_l2(y, ref) <= bound


@pytest.mark.parametrize("path", [1, 2])
def test_windowed_solve_vs_oracle(path):
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax, cutoff = 9, 7, 4, 2.0
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 8)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), np.array([[1, 0, 0]], complex))
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    with system.window(cutoff, cutoff):
        ref = system.solve_dense(nmax, K0, pos, To,
                                 incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, np.array([1, 0, 0], complex)),
                                 cutoff)
    for prec, tol, bound in ((0, 1e-11, 1e-9), (1, 1e-8, 1e-6)):
        opts = _lib.make_opts(tol=tol, cutoff=cutoff, taper=cutoff, precision=prec, path=path, lattice_nx=nx,
                              lattice_ny=ny, lattice_pitch=0.5)
        s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
        assert rc == 0 and rel_l2(s[0], ref) <= bound
