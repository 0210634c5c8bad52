"""Pins of the incident coefficients (App. II-A), the collective system
(App. I-C, Eq. final_linear_eqs), the adjoint gradient (App. IV) and the
integer geometry."""
import math

import numpy as np
import pytest

from oracle import adjoint, geometry, incident, mie, system, vswf
from oracle_pins import K0, energy_balance_error, planewave_error
from paper_2107_09879_b300 import workloads as W


@pytest.mark.parametrize("beta,alpha", [(0.0, 0.0), (math.radians(10), 0.0), (0.4, 1.1), (1.2, -2.0)])
def test_planewave_expansion_pointwise(beta, alpha):
    assert planewave_error(20, beta, alpha) < 1e-10


def test_energy_conservation_lattice():
    """Lossless spheres: extinction from the coefficients equals the scattered
    power from far-field quadrature of the field (solves the coupled system)."""
    assert energy_balance_error(3, 3, 3, 10.0) < 1e-11


def test_energy_conservation_non_planar():
    """Same with sphere centres off the plane (pins the theta dependence of xi)."""
    assert energy_balance_error(2, 3, 3, 25.0, z_jitter=0.3) < 1e-11


def _tiny(nx=3, ny=2, nmax=3, seed=11):
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, seed)
    T = np.array([mie.tmatrix_diag(nmax, K0, rr, 2.0) for rr in r])
    a0 = incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, [1.0, 0.0, 0.0])
    return pos, r, T, a0


@pytest.mark.parametrize("cutoff", [0.0, 0.8])
def test_dense_lu_vs_gmres(cutoff):
    pos, r, T, a0 = _tiny()
    sd = system.solve_dense(3, K0, pos, T, a0, cutoff)
    sg, its, rr = system.solve_gmres(3, K0, pos, T, a0, cutoff, tol=1e-14)
    assert np.linalg.norm(sd - sg) <= 1e-12 * np.linalg.norm(sd)


def test_gmres_restart_path():
    pos, r, T, a0 = _tiny(3, 3)
    sd = system.solve_dense(3, K0, pos, T, a0)
    nbr = geometry.neighbours(pos, 0.0)
    shape = a0.shape
    mv = lambda v: system.apply_K(3, K0, pos, T, v.reshape(shape), nbr).reshape(-1)
    x, its, rr = system.gmres(mv, (T * a0).reshape(-1), tol=1e-13, restart=5)
    assert its > 5 and np.linalg.norm(x.reshape(shape) - sd) <= 1e-11 * np.linalg.norm(sd)


def test_single_scatterer_reduces_to_mie():
    pos = np.zeros((1, 3))
    t = mie.tmatrix_diag(4, K0, 0.2, 2.0)[None, :]
    a0 = incident.planewave_incident(4, K0, pos, 0.3, 0.2, incident.beta_hat(0.3, 0.2))
    s = system.solve_dense(4, K0, pos, t, a0)
    assert np.allclose(s, t * a0, rtol=0, atol=1e-15)


def test_reciprocity():
    """Omega^T = J Omega J with J the m -> -m permutation (reciprocity of the
    Maxwell operator in this basis); checked on K = T Omega through T^-1 K."""
    pos, r, T, a0 = _tiny(2, 2)
    pos = pos + np.array([[0, 0, 0], [0.03, 0, 0.1], [0, -0.05, -0.1], [0.02, 0.04, 0]])
    nbr = geometry.neighbours(pos, 0.0)
    Kd = system.dense_K(3, K0, pos, T, nbr)
    Om = Kd / T.reshape(-1)[:, None]
    lm = vswf.lm_list(3)
    L = len(lm)
    idx = {x: i for i, x in enumerate(lm)}
    perm = [idx[(l, -m)] for (l, m) in lm]
    perm = perm + [L + p for p in perm]
    P = T.shape[1]
    full = np.concatenate([np.array(perm) + i * P for i in range(len(pos))])
    J = np.eye(len(full))[full]
    assert np.max(np.abs(Om.T - J @ Om @ J)) < 1e-12 * np.max(np.abs(Om))


def test_transposed_apply_is_bilinear_transpose():
    pos, r, T, a0 = _tiny(3, 2)
    nbr = geometry.neighbours(pos, 0.8)
    rng = np.random.default_rng(1)
    u = rng.normal(size=a0.shape) + 1j * rng.normal(size=a0.shape)
    x = rng.normal(size=a0.shape) + 1j * rng.normal(size=a0.shape)
    lhs = np.sum(u * system.apply_K(3, K0, pos, T, x, nbr))
    rhs = np.sum(system.apply_KT(3, K0, pos, T, u, nbr) * x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_sampled_rows_match_full_apply():
    pos, r, T, a0 = _tiny(3, 3)
    nbr = geometry.neighbours(pos, 0.8)
    y = system.apply_K(3, K0, pos, T, a0, nbr)
    assert np.allclose(system.apply_K_rows(3, K0, pos, T, a0, nbr, [0, 4, 8]), y[[0, 4, 8]], atol=1e-15)
    yt = system.apply_KT(3, K0, pos, T, a0, nbr)
    assert np.allclose(system.apply_KT_rows(3, K0, pos, T, a0, nbr, [1, 5]), yt[[1, 5]], atol=1e-15)


def test_adjoint_gradient_vs_central_fd():
    nmax = 3
    pos = W.lattice_positions(3, 2)
    r = W.uniform_radii(6, 0.1, 0.22, 7)
    xf = np.array([0.5, 0.25, 3.0])
    A = np.array([1.0, 0.0, 0.0])
    Einc = incident.planewave_field(K0, 0.0, 0.0, A, xf[None])[0]
    a0 = incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, A)

    def fwd(rr):
        T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in rr])
        return T, system.solve_dense(nmax, K0, pos, T, a0, 0.8)

    T, s = fwd(r)
    dT = np.array([mie.tmatrix_diag_dr(nmax, K0, x, 2.0) for x in r])
    v = adjoint.adjoint_source(nmax, K0, pos, s, xf, Einc)
    g, mu = adjoint.radius_gradient(nmax, K0, pos, T, dT, a0, s, v, cutoff=0.8)
    h = 1e-5
    for i in range(6):
        rp, rm = r.copy(), r.copy()
        rp[i] += h
        rm[i] -= h
        fd = (adjoint.fom(nmax, K0, pos, fwd(rp)[1], xf, Einc) - adjoint.fom(nmax, K0, pos, fwd(rm)[1], xf, Einc)) / (2 * h)
        assert abs(g[i] - fd) < 1e-6 * np.max(np.abs(g))


def _lattice_count(c_pitch):
    c2 = c_pitch * c_pitch
    return sum(1 for a in range(-c_pitch, c_pitch + 1) for b in range(-c_pitch, c_pitch + 1)
               if (a, b) != (0, 0) and a * a + b * b <= c2)


@pytest.mark.parametrize("cutoff,expect", [(8.0, 796), (10.0, 1256), (6.0, 440)])
def test_neighbour_counts_interior(cutoff, expect):
    assert _lattice_count(int(round(cutoff / 0.5))) == expect
    n = int(2 * cutoff / 0.5) + 3
    pos = W.lattice_positions(n, n)
    row_ptr, col = geometry.neighbours(pos, cutoff)
    centre = (n // 2) * n + n // 2
    assert row_ptr[centre + 1] - row_ptr[centre] == expect


def test_neighbours_dense_and_symmetric():
    pos = W.lattice_positions(8, 8)
    row_ptr, col = geometry.neighbours(pos, 0.0)
    assert row_ptr[-1] == 64 * 63
    pos = W.random_positions(40, 4.0, 0.45, 9)
    row_ptr, col = geometry.neighbours(pos, 1.3)
    pairs = {(i, int(j)) for i in range(len(pos)) for j in col[row_ptr[i]:row_ptr[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)
    for i in range(len(pos)):
        js = col[row_ptr[i]:row_ptr[i + 1]]
        assert np.all(np.diff(js) > 0) and i not in js


def test_subregions_partition():
    sets = geometry.subregion_sets(23, 17, 6, 5, 2)
    cores = np.concatenate([c for c, s in sets])
    assert np.array_equal(np.sort(cores), np.arange(23 * 17))
    for core, sim in sets:
        assert np.all(np.isin(core, sim))
    # interior sub-region: (6 + 4) x (5 + 4) sites
    assert len(sets[1 * 4 + 1][1]) == 10 * 9


def test_coupling_window_definition():
    """The window is 1 inside cutoff - taper, 1/2 at the taper midpoint, 0 at the
    cutoff, and scales every block of a pair by the same factor."""
    w = system.coupling_weight
    assert w(1.0, 8.0, 2.0) == 1.0 and w(8.0, 8.0, 2.0) == 0.0
    assert abs(w(7.0, 8.0, 2.0) - 0.5) < 1e-15 and w(3.0, 8.0, 0.0) == 1.0
    assert abs(w(4.0, 8.0, 8.0) - 0.5) < 1e-15
    pos = W.lattice_positions(3, 1)
    B0 = system._block(3, K0, pos[0], pos[2])
    with system.window(2.0, 2.0):
        B1 = system._block(3, K0, pos[0], pos[2])
    assert np.allclose(B1, B0 * 0.5 * (1 + math.cos(math.pi * 1.0 / 2.0)), rtol=0, atol=1e-15)
