"""GPU parity of the building-block kernels against the oracle (through the C-ABI)."""
import math

import numpy as np
import pytest

from gpu_common import C64_APPLY_TOL, K0, atoms, ctx, rand_c, rel_l2
from oracle import geometry, incident, mie, system, translation
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["lattice", "random", "dense", "empty", "single"])
def test_neighbors_bit_exact(case):
    if case == "lattice":
        pos, cut = W.lattice_positions(13, 11), 2.0
    elif case == "random":
        pos, cut = W.random_positions(57, 5.0, 0.4, 3), 1.37
    elif case == "dense":
        pos, cut = W.lattice_positions(8, 8), 0.0
    elif case == "empty":
        pos, cut = np.zeros((0, 3)), 1.0
    else:
        pos, cut = np.zeros((1, 3)), 1.0
    rp, col = ctx().tmat_neighbors(pos, cut)
    orp, ocol = geometry.neighbours(pos, cut)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)


def test_neighbors_cutoff_boundary_inclusive():
    # (12,16) pitches -> distance exactly 10.0: inclusive on both sides
    pos = W.lattice_positions(41, 41)
    rp, col = ctx().tmat_neighbors(pos, 10.0)
    orp, ocol = geometry.neighbours(pos, 10.0)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    c = 20 * 41 + 20
    assert rp[c + 1] - rp[c] == 1256


@pytest.mark.parametrize("dims", [(23, 17, 6, 5, 2), (120, 120, 60, 60, 8), (7, 3, 7, 3, 4), (10, 9, 3, 4, 0)])
def test_subregions_bit_exact(dims):
    nx, ny, cx, cy, buf = dims
    core_ptr, core_idx, sim_ptr, sim_idx = ctx().tmat_subregions(nx, ny, cx, cy, buf)
    sets = geometry.subregion_sets(nx, ny, cx, cy, buf)
    assert len(core_ptr) == len(sets) + 1
    for a, (c, s) in enumerate(sets):
        assert np.array_equal(core_idx[core_ptr[a]:core_ptr[a + 1]], c)
        assert np.array_equal(sim_idx[sim_ptr[a]:sim_ptr[a + 1]], s)


@pytest.mark.parametrize("nmax", [1, 3, 4, 6])
def test_mie_build(nmax):
    r = W.uniform_radii(37, 0.05, 0.3, 11)
    for n_im in [0.0, 0.07]:
        T, dT = ctx().tmat_build(atoms(r, 2.0, n_im), 1.0, 1.0, nmax, with_dr=True)
        To = np.array([mie.tmatrix_diag(nmax, K0, x, complex(2.0, n_im)) for x in r])
        dTo = np.array([mie.tmatrix_diag_dr(nmax, K0, x, complex(2.0, n_im)) for x in r])
        assert np.max(np.abs(T - To)) <= 1e-12 * np.max(np.abs(To))
        assert np.max(np.abs(dT - dTo)) <= 1e-11 * np.max(np.abs(dTo))


def test_mie_build_background_index_and_wavelength():
    r = np.array([0.1, 0.2])
    T = ctx().tmat_build(atoms(r, 2.4, 0.0), 1.1, 1.2, 3)
    k = 2 * math.pi * 1.2 / 1.1
    To = np.array([mie.tmatrix_diag(3, k, x, 2.4 / 1.2) for x in r])
    assert np.max(np.abs(T - To)) <= 1e-12 * np.max(np.abs(To))


@pytest.mark.parametrize("nmax", [2, 4, 5])
def test_planewave_incident(nmax):
    pos = W.random_positions(19, 3.0, 0.3, 5)
    pos[:, 2] = np.linspace(-0.2, 0.3, len(pos))
    dirs = np.array([[0.0, 0.0], [math.radians(10), 0.0], [0.7, 1.3]])
    pols = np.array([incident.beta_hat(*d) * (1 + 0.5j) + 0.3 * incident.alpha_hat(*d) for d in dirs])
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pols)
    for r, d in enumerate(dirs):
        ref = incident.planewave_incident(nmax, K0, pos, d[0], d[1], pols[r])
        assert np.max(np.abs(a0[r] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("nmax", [1, 2, 3, 4, 5, 6])
def test_translation_matrices(nmax):
    g = W.SplitMix64(100 + nmax)
    disp = (np.array(g.uniforms(3 * 9)).reshape(9, 3) - 0.5) * 6.0
    disp[0] = [0.5, 0.0, 0.0]      # lattice neighbour, k d = pi (j_0 = 0)
    disp[1] = [3.0, -4.0, 0.0]     # planar, k d = 10 pi
    disp[2] = [0.0, 0.0, 0.7]      # on the axis (theta = 0)
    xi = ctx().tmat_translation(nmax, K0, disp)
    for m in range(len(disp)):
        ref = translation.xi_matrix(nmax, nmax, K0, disp[m])
        assert np.max(np.abs(xi[m] - ref)) <= 1e-11 * np.max(np.abs(ref)), m


def _apply_case(nx, ny, nmax, cutoff, seed, R):
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, seed)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), seed + 1)
    return pos, T, x


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(3, 7, 5, 1.2, 1), (4, 6, 6, 1.6, 2), (2, 5, 3, 0.0, 5),
                                                 (5, 4, 3, 1.1, 1), (6, 3, 3, 0.8, 1)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_apply_neighbour_fp64_and_fp32(nmax, nx, ny, cutoff, R, op):
    from paper_2107_09879_b300 import _lib
    pos, T, x = _apply_case(nx, ny, nmax, cutoff, 31 + nmax, R)
    nbr = geometry.neighbours(pos, cutoff)
    rp, col = ctx().tmat_neighbors(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    ref = np.array([f(nmax, K0, pos, T, x[r], nbr) for r in range(R)])
    y64 = ctx().tmat_apply(op, _lib.PREC_FP64, pos, K0, nmax, T, rp, col, x)
    y32 = ctx().tmat_apply(op, _lib.PREC_MIXED, pos, K0, nmax, T, rp, col, x)
    assert rel_l2(y64, ref) <= 1e-12
    assert rel_l2(y32, ref) <= C64_APPLY_TOL


def test_apply_rejects_non_finite_positions():
    from paper_2107_09879_b300 import _lib
    pos, T, x = _apply_case(3, 3, 2, 1.0, 5, 1)
    rp, col = ctx().tmat_neighbors(pos, 1.0)
    pos = pos.copy()
    pos[4, 2] = float("nan")
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_apply(0, 0, pos, K0, 2, T, rp, col, x)
    assert e.value.code == _lib.EINVAL
