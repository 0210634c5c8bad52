"""GPU null-field cylinder T-matrices (tmat_build_cylinder) and the solve / adjoint with full
per-scatterer T-blocks (tmat_solve_tblocks, tmat_adjoint_tblocks) against the oracle."""
import math

import numpy as np
import pytest

from gpu_common import K0, ctx, rel_l2
from oracle import incident, mie, nullfield, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _cyl(rows):
    return np.ascontiguousarray(np.array(rows, dtype=np.float64))


@pytest.mark.parametrize("nmax", [1, 2, 4, 6])
@pytest.mark.parametrize("index", [(2.0, 0.0), (1.5, 0.2), (3.5, 0.0)])
def test_cylinder_tmatrix_vs_oracle(nmax, index):
    """Same rule on both sides (24 Gauss nodes per face; the oracle's trapezoid azimuth is exact
    for the m = m' integrands), so the two agree to rounding."""
    geo = [(0.12, 0.25), (0.2, 0.1), (0.07, 0.3)]
    T = ctx().tmat_build_cylinder(_cyl([[a, h, index[0], index[1]] for a, h in geo]), 1.0, 1.0, nmax, n_quad=24)
    for i, (a, h) in enumerate(geo):
        ref = nullfield.cylinder_tmatrix(nmax, K0, complex(*index), a, h, n_face=24)
        assert np.abs(T[i] - ref).max() <= 1e-10 * np.abs(ref).max()


def test_cylinder_radius_derivative_vs_oracle_differences():
    nmax, a, h = 3, 0.13, 0.22
    T, dT = ctx().tmat_build_cylinder(_cyl([[a, h, 2.0, 0.0]]), 1.0, 1.0, nmax, n_quad=32, with_dr=True)
    st = 1e-4
    fd = (nullfield.cylinder_tmatrix(nmax, K0, 2.0, a + st, h, n_face=32) -
          nullfield.cylinder_tmatrix(nmax, K0, 2.0, a - st, h, n_face=32)) / (2 * st)
    assert np.abs(dT[0] - fd).max() <= 1e-6 * np.abs(fd).max()


def test_sphere_limit_on_the_gpu_path_is_not_assumed():
    """A cylinder is not a sphere: the GPU T has couplings l != l' (off-diagonal entries) that
    a diagonal Mie T lacks, and equals the oracle there too."""
    T = ctx().tmat_build_cylinder(_cyl([[0.12, 0.25, 2.0, 0.0]]), 1.0, 1.0, 3, n_quad=24)[0]
    off = T - np.diag(np.diag(T))
    assert np.abs(off).max() > 1e-3 * np.abs(T).max()


def _array(nx, ny, nmax, seed, z0=0.0):
    """Cylinders of three kinds on a 0.5-wavelength lattice (types), oracle T-blocks; z0 != 0
    shifts every cylinder along its axis (blocks coupling the parity classes)."""
    pos = W.lattice_positions(nx, ny)
    g = W.SplitMix64(seed)
    types = np.array([min(2, int(3 * g.uniform())) for _ in range(nx * ny)], dtype=np.int32)
    kinds = [(0.08, 0.2), (0.12, 0.22), (0.15, 0.18)]
    if z0:
        Tb = np.array([nullfield.tmatrix(nmax, K0, 2.0, nullfield.surface_cylinder(a, h, 24, 2 * nmax + 4, z0=z0))
                       for a, h in kinds])
    else:
        Tb = np.array([nullfield.cylinder_tmatrix(nmax, K0, 2.0, a, h, n_face=24) for a, h in kinds])
    return pos, types, Tb


def _a0(nmax, pos, angles):
    return np.array([incident.planewave_incident(nmax, K0, pos, math.radians(b), 0.0,
                                                 incident.beta_hat(math.radians(b), 0.0)) for b in angles])


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-9), (1, 1e-8, 1e-6)])
@pytest.mark.parametrize("nx,ny,nmax,cutoff,z0", [(4, 3, 3, 0.0, 0.0), (5, 4, 4, 1.2, 0.0), (3, 3, 2, 0.8, 0.05)])
def test_solve_tblocks_vs_oracle(path, precision, tol, bound, nx, ny, nmax, cutoff, z0):
    from paper_2107_09879_b300 import _lib
    pos, types, Tb = _array(nx, ny, nmax, 31 + nx, z0)
    a0 = _a0(nmax, pos, (0.0, 10.0))
    opts = _lib.make_opts(tol=tol, restart=80, max_iter=3000, cutoff=cutoff, precision=precision, path=path,
                          lattice_nx=nx, lattice_ny=ny, lattice_pitch=0.5)
    s, info, _, rc = ctx().tmat_solve_tblocks(pos, 1.0, 1.0, nmax, Tb, a0, opts, types=types)
    assert rc == 0 and info.converged
    for q in range(2):
        ref = system.solve_dense_blocks(nmax, K0, pos, Tb[types], a0[q], cutoff)
        assert rel_l2(s[q], ref) <= bound


def test_diagonal_blocks_reproduce_tmat_solve():
    from paper_2107_09879_b300 import _lib
    nmax, nx, ny = 3, 6, 5
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 9)
    t = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    Tb = np.ascontiguousarray(np.array([np.diag(v) for v in t]))
    a0 = _a0(nmax, pos, (0.0,))
    for path in (1, 2):
        opts = _lib.make_opts(tol=1e-12, cutoff=1.5, precision=0, path=path, lattice_nx=nx, lattice_ny=ny,
                              lattice_pitch=0.5)
        s1, _, _, rc1 = ctx().tmat_solve(pos, 1.0, 1.0, nmax, np.ascontiguousarray(t), a0, opts)
        s2, _, _, rc2 = ctx().tmat_solve_tblocks(pos, 1.0, 1.0, nmax, Tb, a0, opts)
        assert rc1 == 0 and rc2 == 0 and rel_l2(s2, s1) <= 1e-10


@pytest.mark.parametrize("path,precision", [(2, 0), (1, 0), (2, 1)])
def test_adjoint_tblocks_radius_gradient(path, precision):
    """dFoM/d(radius) of every cylinder (its own T-block) by the adjoint, against the oracle's
    gradient formula on its own solution and against central differences of the FoM of
    GPU fp64 solves."""
    from paper_2107_09879_b300 import _lib
    nmax, nx, ny = 3, 3, 2
    pos = W.lattice_positions(nx, ny)
    radii = W.uniform_radii(nx * ny, 0.09, 0.15, 17)
    cyl = _cyl([[a, 0.2, 2.0, 0.0] for a in radii])
    T, dT = ctx().tmat_build_cylinder(cyl, 1.0, 1.0, nmax, n_quad=24, with_dr=True)
    xf = np.array([0.5, 0.25, 3.0])
    A = np.array([1.0, 0.0, 0.0], dtype=complex)
    Einc = incident.planewave_field(K0, 0.0, 0.0, A, xf[None])[0]
    a0 = incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, A)[None]
    opts = _lib.make_opts(tol=1e-12 if precision == 0 else 1e-9, restart=60, cutoff=0.0, precision=precision,
                          path=path, lattice_nx=nx, lattice_ny=ny, lattice_pitch=0.5)
    s, info, sol, rc = ctx().tmat_solve_tblocks(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
    assert rc == 0
    fom, v = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, Einc)
    g, mu, ainfo = ctx().tmat_adjoint_tblocks(sol, v, dT, want_mu=True)
    sol.free()
    # central differences of the FoM (fp64 GPU solves, T rebuilt for the moved radius)
    opts64 = _lib.make_opts(tol=1e-13, restart=60, cutoff=0.0, precision=0, path=path, lattice_nx=nx,
                            lattice_ny=ny, lattice_pitch=0.5)
    h = 1e-5
    for i in (0, 3, 5):
        f = []
        for sgn in (1, -1):
            c2 = cyl.copy()
            c2[i, 0] += sgn * h
            T2 = ctx().tmat_build_cylinder(c2, 1.0, 1.0, nmax, n_quad=24)
            s2, _, _, _ = ctx().tmat_solve_tblocks(pos, 1.0, 1.0, nmax, T2, a0, opts64)
            f.append(ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s2[0], xf, Einc)[0])
        fd = (f[0] - f[1]) / (2 * h)
        assert abs(g[i] - fd) <= (1e-5 if precision == 0 else 1e-4) * np.abs(g).max()
    # the oracle's gradient: mu from the transposed dense system, e = a0 + A s, dT by central
    # differences of the oracle's null-field T
    from oracle import adjoint, geometry
    To = np.array([nullfield.cylinder_tmatrix(nmax, K0, 2.0, a, 0.2, n_face=24) for a in radii])
    st = 1e-4
    dTo = np.array([(nullfield.cylinder_tmatrix(nmax, K0, 2.0, a + st, 0.2, n_face=24) -
                     nullfield.cylinder_tmatrix(nmax, K0, 2.0, a - st, 0.2, n_face=24)) / (2 * st) for a in radii])
    so = system.solve_dense_blocks(nmax, K0, pos, To, a0[0])
    vo = adjoint.adjoint_source(nmax, K0, pos, so, xf, Einc)
    nbr = geometry.neighbours(pos, 0.0)
    K = system.dense_K_blocks(nmax, K0, pos, To, nbr)
    muo = np.linalg.solve(K.T, vo.reshape(-1)).reshape(so.shape)
    e = a0[0] + system.apply_A(nmax, K0, pos, so, nbr)
    go = np.array([2 * np.real(muo[i] @ dTo[i] @ e[i]) for i in range(len(pos))])
    assert rel_l2(g, go) <= (1e-6 if precision == 0 else 1e-5)


def test_tblock_argument_errors():
    from paper_2107_09879_b300 import _lib
    pos, types, Tb = _array(3, 2, 2, 5)
    a0 = _a0(2, pos, (0.0,))
    opts = _lib.make_opts(tol=1e-10, precision=0)
    bad = types.copy()
    bad[2] = 3
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve_tblocks(pos, 1.0, 1.0, 2, Tb, a0, opts, types=bad)
    assert e.value.code == _lib.EINVAL
    opts.precision = 2
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve_tblocks(pos, 1.0, 1.0, 2, Tb, a0, opts, types=types)
    assert e.value.code == _lib.ENOTSUP
