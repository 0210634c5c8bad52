"""GPU sub-region sweep (tmat_sweep) against direct solves and the oracle."""
import math

import numpy as np
import pytest

from gpu_common import K0, atoms, ctx, rand_c, rel_l2
from oracle import incident, sweep
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu
Z0 = -1.0


def _setup(nx, ny, seed, R=1):
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.2, seed)
    at = atoms(r)
    # sources sample a normally incident x-polarised plane wave (and a tilted one for R = 2)
    src = np.zeros((R, nx * ny, 2), complex)
    for q in range(R):
        th = math.radians(10 * q)
        ph = np.exp(1j * K0 * (math.sin(th) * pos[:, 0] + math.cos(th) * Z0))
        src[q, :, 0] = math.cos(th) * ph
    pts = np.array([[1.0, 1.2, 3.0], [2.5, 0.5, 4.0], [0.3, 2.0, -2.5]])
    return pos, r, at, src, pts


def _direct(pos, at, src, pts, nmax, opts, nb, na):
    from paper_2107_09879_b300 import _lib
    T = ctx().tmat_build(at, 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_jinc(pos, 1.0, 1.0, nmax, pos[:, :2].copy(), src, Z0, nb, na, precision=opts.precision)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    assert rc == 0
    return np.array([ctx().tmat_field(pos, 1.0, 1.0, nmax, s[q], pts) for q in range(src.shape[0])])


def test_one_subregion_equals_direct_pipeline():
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 7, 6, 3
    pos, r, at, src, pts = _setup(nx, ny, 1, R=2)
    opts = _lib.make_opts(tol=1e-12, cutoff=0.0, precision=0)
    sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=nx, core_y=ny, buffer=0, z0=Z0, n_beta=40, n_alpha=56)
    E, info, rc = ctx().tmat_sweep(sw, at, 1.0, 1.0, nmax, src, opts, pts)
    assert rc == 0 and info.subregions == 1
    o2 = _lib.make_opts(tol=1e-12, cutoff=0.0, precision=0, path=2, lattice_nx=nx, lattice_ny=ny, lattice_pitch=0.5)
    ref = _direct(pos, at, src, pts, nmax, o2, 40, 56)
    assert rel_l2(E, ref) <= 1e-12


def test_full_buffer_decomposition_is_linear():
    """Buffers that cover the whole array: each sub-region solves the full array for its
    core's sources, so the sum over sub-regions equals one solve with all sources."""
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 8, 6, 2
    pos, r, at, src, pts = _setup(nx, ny, 2)
    opts = _lib.make_opts(tol=1e-13, cutoff=0.0, precision=0)
    sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=3, core_y=4, buffer=8, z0=Z0, n_beta=40, n_alpha=56)
    E, info, rc = ctx().tmat_sweep(sw, at, 1.0, 1.0, nmax, src, opts, pts)
    assert rc == 0 and info.subregions == 6
    o2 = _lib.make_opts(tol=1e-13, cutoff=0.0, precision=0)
    ref = _direct(pos, at, src, pts, nmax, o2, 40, 56)
    assert rel_l2(E, ref) <= 1e-9


def test_sweep_vs_oracle():
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 6, 4, 2
    pos, r, at, src, pts = _setup(nx, ny, 3)
    opts = _lib.make_opts(tol=1e-13, cutoff=0.0, precision=0)
    sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=3, core_y=2, buffer=1, z0=Z0, n_beta=36, n_alpha=48)
    E, info, rc = ctx().tmat_sweep(sw, at, 1.0, 1.0, nmax, src, opts, pts)
    rule = incident.jinc_rule(36, 48)
    ref = sweep.sweep_fields(nmax, K0, nx, ny, 0.5, 0.0, r, 2.0, src[0], Z0, (3, 2), 1, pts, lambda p, s: rule)
    assert rc == 0 and rel_l2(E[0], ref) <= 1e-9


def test_sweep_resume_in_pieces():
    """A sweep split into [first, first+count) pieces accumulates the same field."""
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 9, 6, 2
    pos, r, at, src, pts = _setup(nx, ny, 4)
    opts = _lib.make_opts(tol=1e-12, cutoff=0.0, precision=0)
    kw = dict(nx=nx, ny=ny, pitch=0.5, core_x=3, core_y=3, buffer=2, z0=Z0, n_beta=36, n_alpha=48)
    E_all, _, _ = ctx().tmat_sweep(_lib.make_sweep(**kw), at, 1.0, 1.0, nmax, src, opts, pts)
    E = None
    for first in (0, 2, 4):
        E, info, rc = ctx().tmat_sweep(_lib.make_sweep(first=first, count=2, **kw), at, 1.0, 1.0, nmax, src, opts,
                                       pts, E=E)
        assert info.subregions == 2
    assert np.array_equal(E, E_all)


def test_buffer_convergence():
    """Synthetic analog of the paper's padding study (Fig. 2b): the error of the
    decomposed field against the full-array solve falls as the padding grows."""
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax = 20, 20, 2
    pos, r, at, src, pts = _setup(nx, ny, 5)
    pts = np.array([[4.75, 4.75, 4.0], [2.0, 7.0, 5.0], [8.0, 3.0, 6.0]])
    opts = _lib.make_opts(tol=1e-10, cutoff=0.0, precision=0)
    full = _direct(pos, at, src, pts, nmax, _lib.make_opts(tol=1e-10, cutoff=0.0, precision=0), 0, 0)
    errs = []
    for buf in (0, 3, 6, 12):
        sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=10, core_y=10, buffer=buf, z0=Z0)
        E, info, rc = ctx().tmat_sweep(sw, at, 1.0, 1.0, nmax, src, opts, pts)
        assert rc == 0
        errs.append(rel_l2(E, full))
    assert errs[-1] < 0.5 * errs[0] and errs[-1] < 1e-6, errs
