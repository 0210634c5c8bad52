"""GPU enclosing-sphere overlap check (tmat_check_overlap, TMAT_EOVERLAP from tmat_solve with
enclosing radii and from tmat_sweep) against the oracle's brute-force definition: the first
intersecting pair is integer output, compared exactly."""
import math

import numpy as np
import pytest

from gpu_common import K0, atoms, ctx
from oracle import geometry
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,rlo,rhi,seed,flat", [(200, 10.0, 0.05, 0.2, 1, True), (300, 4.0, 0.05, 0.12, 2, False),
                                                  (150, 30.0, 0.01, 0.1, 3, True), (2, 1.0, 0.4, 0.6, 4, False),
                                                  (500, 6.0, 0.0, 0.08, 5, False)])
def test_first_pair_matches_oracle(n, box, rlo, rhi, seed, flat):
    g = W.SplitMix64(seed)
    pos = np.stack([g.uniforms(n) * box, g.uniforms(n) * box, np.zeros(n) if flat else g.uniforms(n) * box], 1)
    r = rlo + (rhi - rlo) * g.uniforms(n)
    assert ctx().tmat_check_overlap(np.ascontiguousarray(pos), r) == geometry.first_overlap(pos, r)


def test_lattice_edge_cases():
    pos = W.lattice_positions(40, 30)
    r = np.full(len(pos), 0.25)  # exactly touching neighbours
    assert ctx().tmat_check_overlap(pos, r) is None
    assert geometry.first_overlap(pos[:60], r[:60]) is None
    r[613] = 0.25 + 1e-9  # now touches-and-overlaps its four lattice neighbours; the lowest is 573
    assert ctx().tmat_check_overlap(pos, r) == (573, 613) == geometry.first_overlap(pos, r)
    big = np.array([0.1] * len(pos))
    big[1199] = 3.0  # one large sphere at the last site reaches many others; first pair is the lowest i
    got = ctx().tmat_check_overlap(pos, big)
    i = min(k for k in range(len(pos) - 1) if np.sum((pos[k] - pos[1199]) ** 2) < 3.1 ** 2)
    assert got == (i, 1199)


def test_solve_and_sweep_refuse_overlapping_spheres():
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 4, 3, 2
    pos = W.lattice_positions(nx, ny)
    r = np.full(nx * ny, 0.2)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.zeros((1, 2)), np.array([[1, 0, 0]], complex))
    ok = _lib.make_opts(tol=1e-10, precision=0, enclosing_radii=r)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, ok)
    assert rc == 0
    rb = r.copy()
    rb[5] = 0.31
    bad = _lib.make_opts(tol=1e-10, precision=0, enclosing_radii=rb)
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, bad)
    assert e.value.code == _lib.EOVERLAP
    # sweep over spheres that overlap
    at = atoms(np.full(nx * ny, 0.26))
    src = np.ones((1, nx * ny, 2), complex)
    sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=2, core_y=2, buffer=1, z0=-1.0, n_beta=20, n_alpha=24)
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_sweep(sw, at, 1.0, 1.0, nmax, src, _lib.make_opts(tol=1e-8, precision=0), np.array([[0.5, 0.5, 3.0]]))
    assert e.value.code == _lib.EOVERLAP
