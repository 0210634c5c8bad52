"""Pins of the oracle's null-field T-matrix (App. I-B: the P and Q surface integrals and
T from them) for spheres and upright cylinders:

  - sphere limit: the surface integrals over a sphere give the Lorenz-Mie T-matrix
    (closed form) for lossless and lossy spheres;
  - first Born limit: for an index m -> 1 the T-matrix tends to
        T[nu, mu] = i (k^3 / pi) (m^2 - 1) volume integral of RPhi_{l,-m,p}(k x) . RPhi_mu(k x),
    a volume integral that shares nothing with the surface integrals; the constant is
    checked on the sphere, then the cylinder's full matrix (off-diagonal couplings
    included) must match;
  - structure: rotational symmetry (T couples m = m' only) and the z-mirror class
    (l + m + p) mod 2 hold exactly;
  - unitarity (lossless) and reciprocity converge as nmax grows;
  - the quadrature is converged;
and the literal printed forms (T = -P Q^-1; a minus between the two terms) fail the
sphere limit."""
import math

import numpy as np
import pytest

from oracle import mie, nullfield
from oracle import vswf as V

K0 = 2 * math.pi


def _born(nmax, pts_w):
    """Volume integral of RPhi_{l,-m,p} . RPhi_mu over quadrature points (x, weight)."""
    _, same = nullfield._partner(nmax)
    P = 2 * nmax * (nmax + 2)
    M = np.zeros((P, P), complex)
    for x, w in pts_w:
        R = V.vswf(nmax, K0, x, regular=True)
        M += w * (R[same] @ R.T)
    return M


def _sphere_volume(a, n, nphi):
    rr, wr = nullfield._gauss(n, 0.0, a)
    ct, wt = np.polynomial.legendre.leggauss(n)
    for r, w1 in zip(rr, wr):
        for c, w2 in zip(ct, wt):
            s = math.sqrt(1 - c * c)
            for ph in 2 * math.pi * np.arange(nphi) / nphi:
                yield r * np.array([s * math.cos(ph), s * math.sin(ph), c]), w1 * w2 * r * r * 2 * math.pi / nphi


def _cylinder_volume(a, h, n, nphi):
    rr, wr = nullfield._gauss(n, 0.0, a)
    zz, wz = nullfield._gauss(n, -h / 2, h / 2)
    for r, w1 in zip(rr, wr):
        for z, w2 in zip(zz, wz):
            for ph in 2 * math.pi * np.arange(nphi) / nphi:
                yield np.array([r * math.cos(ph), r * math.sin(ph), z]), w1 * w2 * r * 2 * math.pi / nphi


def _labels(nmax):
    lmp = [(l, m, p) for p in range(2) for l, m in V.lm_list(nmax)]
    return (np.array([t[0] for t in lmp]), np.array([t[1] for t in lmp]), np.array([t[2] for t in lmp]))


def _J(nmax):
    ls, ms, ps = _labels(nmax)
    P = len(ls)
    idx = {(l, m, p): i for i, (l, m, p) in enumerate(zip(ls, ms, ps))}
    J = np.zeros((P, P))
    for i, (l, m, p) in enumerate(zip(ls, ms, ps)):
        J[i, idx[(l, -m, p)]] = 1.0
    return J


def sphere_limit_error(nmax, m_rel, radius=0.2, form=None):
    surf = nullfield.surface_sphere(radius, 24, 2 * nmax + 4)
    if form is None:
        T = nullfield.tmatrix(nmax, K0, m_rel, surf)
    else:
        Pm, Qm = nullfield.pq_matrices(nmax, K0, m_rel * K0, surf)
        T = form(Pm, Qm)
    Tm = mie.tmatrix_diag(nmax, K0, radius, m_rel)
    return np.abs(T - np.diag(Tm)).max() / np.abs(Tm).max()


@pytest.mark.parametrize("nmax", [2, 4])
@pytest.mark.parametrize("m_rel", [2.0, 1.5 + 0.1j, 3.5])
def test_sphere_limit_is_mie(nmax, m_rel):
    assert sphere_limit_error(nmax, m_rel) <= 1e-12


def test_printed_product_order_is_a_garble():
    assert sphere_limit_error(3, 2.0, form=lambda Pm, Qm: -Pm @ np.linalg.inv(Qm)) > 1e-1


def test_printed_minus_between_the_terms_is_a_garble():
    """The printed integrand subtracts the (k_s / k_b) term; with that sign the sphere limit fails."""
    # direct construction of the literal form
    L = 3 * 5
    flip, same = nullfield._partner(3)
    mu_bar = np.concatenate([np.arange(L, 2 * L), np.arange(0, L)])
    surf = nullfield.surface_sphere(0.2, 24, 10)
    ks = 2.0 * K0
    Pm = np.zeros((2 * L, 2 * L), complex)
    Qm = np.zeros((2 * L, 2 * L), complex)
    for x, n, w in zip(*surf):
        Ri = V.vswf(3, ks, x, regular=True)
        for Out, M in ((V.vswf(3, K0, x), Pm), (V.vswf(3, K0, x, regular=True), Qm)):
            t1 = np.cross(Ri[None, :, :], Out[flip][:, None, :]) @ n
            t2 = np.cross(Ri[mu_bar][None, :, :], Out[same][:, None, :]) @ n
            M += w * (t1 - (ks / K0) * t2)
    T = -Qm @ np.linalg.inv(Pm)
    Tm = mie.tmatrix_diag(3, K0, 0.2, 2.0)
    assert np.abs(T - np.diag(Tm)).max() / np.abs(Tm).max() > 1e-1


def test_born_limit_volume_integral():
    nmax, d = 2, 1e-5
    m_rel = 1.0 + d
    nphi = 2 * nmax + 4
    # the constant i k^3 / pi on the sphere (every diagonal entry)
    Ts = nullfield.tmatrix(nmax, K0, m_rel, nullfield.surface_sphere(0.2, 24, nphi))
    Bs = _born(nmax, _sphere_volume(0.2, 14, nphi))
    ratio = np.diag(Ts) / np.diag(Bs) / (m_rel * m_rel - 1)
    assert np.abs(ratio - 1j * K0 ** 3 / math.pi).max() <= 1e-4 * K0 ** 3 / math.pi
    # the cylinder's whole matrix
    Tc = nullfield.cylinder_tmatrix(nmax, K0, m_rel, 0.12, 0.25, n_face=32)
    Bc = 1j * K0 ** 3 / math.pi * (m_rel * m_rel - 1) * _born(nmax, _cylinder_volume(0.12, 0.25, 14, nphi))
    off = np.abs(Tc - np.diag(np.diag(Tc))).max()
    assert off > 1e-3 * np.abs(Tc).max()  # the check covers real off-diagonal couplings
    assert np.abs(Tc - Bc).max() <= 1e-4 * np.abs(Tc).max()


def test_cylinder_structure_is_exact():
    nmax = 4
    T = nullfield.cylinder_tmatrix(nmax, K0, 2.0, 0.12, 0.25, n_face=24)
    ls, ms, ps = _labels(nmax)
    scale = np.abs(T).max()
    assert np.abs(T[ms[:, None] != ms[None, :]]).max() <= 1e-13 * scale
    cls = (ls + ms + ps) % 2
    assert np.abs(T[cls[:, None] != cls[None, :]]).max() <= 1e-13 * scale
    # an off-centre cylinder (shifted along z) breaks the mirror class but keeps m = m'
    Ts = nullfield.tmatrix(nmax, K0, 2.0, nullfield.surface_cylinder(0.12, 0.25, 24, 2 * nmax + 4, z0=0.05))
    assert np.abs(Ts[cls[:, None] != cls[None, :]]).max() > 1e-4 * scale
    assert np.abs(Ts[ms[:, None] != ms[None, :]]).max() <= 1e-13 * scale


def test_unitarity_and_reciprocity_converge_with_nmax():
    errs = []
    for nmax in (3, 6):
        T = nullfield.cylinder_tmatrix(nmax, K0, 2.0, 0.12, 0.25, n_face=40)
        U = T + T.conj().T + 2 * T.conj().T @ T
        J = _J(nmax)
        errs.append((np.abs(U).max() / np.abs(T).max(), np.abs(J @ T.T @ J - T).max() / np.abs(T).max()))
    assert errs[0][0] <= 1e-2 and errs[0][1] <= 1e-2
    assert errs[1][0] <= errs[0][0] / 5 and errs[1][1] <= errs[0][1] / 5
    # the sphere is unitary and reciprocal to rounding
    Ts = nullfield.tmatrix(3, K0, 2.0, nullfield.surface_sphere(0.2, 24, 10))
    assert np.abs(Ts + Ts.conj().T + 2 * Ts.conj().T @ Ts).max() <= 1e-12


def test_quadrature_is_converged():
    a = nullfield.cylinder_tmatrix(3, K0, 2.0 + 0.05j, 0.15, 0.2, n_face=32)
    b = nullfield.cylinder_tmatrix(3, K0, 2.0 + 0.05j, 0.15, 0.2, n_face=48)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


def _cylinder_array(nx, ny, nmax, seed):
    """Lossless cylinders (two radii) on a 0.5-wavelength lattice, each enclosing sphere
    inside its cell; T-blocks from the null-field oracle."""
    from paper_2107_09879_b300 import workloads as W
    pos = W.lattice_positions(nx, ny)
    radii = W.uniform_radii(nx * ny, 0.08, 0.14, seed)
    kinds = {}
    Tb = []
    for r in radii:
        key = 0.08 if r < 0.11 else 0.14
        if key not in kinds:
            kinds[key] = nullfield.cylinder_tmatrix(nmax, K0, 2.0, key, 0.2, n_face=24)
        Tb.append(kinds[key])
    return pos, np.array(Tb)


def test_block_system_energy_conservation(monkeypatch):
    """A lossless cylinder array conserves energy: extinction from the coefficients equals
    the scattered power from far-field quadrature, to the cylinders' own unitarity error
    (null-field truncation, ~4e-3 at nmax 4). A planted mistake in the block system (T on
    the wrong side of the coupling, K = I - A T) breaks the balance by far more."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from oracle import incident, system
    from oracle_pins import far_power
    nmax = 4
    pos, Tb = _cylinder_array(3, 2, nmax, 5)
    beta = math.radians(20.0)
    a0 = incident.planewave_incident(nmax, K0, pos, beta, 0.3, incident.beta_hat(beta, 0.3))

    def balance():
        s = system.solve_dense_blocks(nmax, K0, pos, Tb, a0)
        pext = -np.real(np.vdot(a0, s)) * math.pi / K0 ** 2
        return abs(pext - far_power(nmax, pos, s, nth=30, nph=60)) / pext

    good = balance()
    assert good <= 5e-3

    def wrong_side(nmax_, k, pos_, Tb_, nbr):
        A = system.dense_A(nmax_, k, pos_, nbr)
        N, P, _ = Tb_.shape
        Tf = np.zeros((N * P, N * P), dtype=np.complex128)
        for i in range(N):
            Tf[i * P:(i + 1) * P, i * P:(i + 1) * P] = Tb_[i]
        return np.eye(N * P) - A @ Tf

    monkeypatch.setattr(system, "dense_K_blocks", wrong_side)
    assert balance() > 10 * good


def test_block_system_reduces_to_the_diagonal_system():
    from oracle import geometry, incident, system
    from paper_2107_09879_b300 import workloads as W
    nmax = 3
    pos = W.lattice_positions(3, 2)
    t = np.array([mie.tmatrix_diag(nmax, K0, r, 2.0) for r in W.uniform_radii(6, 0.08, 0.2, 3)])
    Tb = np.array([np.diag(v) for v in t])
    a0 = incident.planewave_incident(nmax, K0, pos, 0.2, 0.0, incident.beta_hat(0.2, 0.0))
    s1 = system.solve_dense(nmax, K0, pos, t, a0, 0.8)
    s2 = system.solve_dense_blocks(nmax, K0, pos, Tb, a0, 0.8)
    assert np.abs(s1 - s2).max() <= 1e-13 * np.abs(s1).max()
    nbr = geometry.neighbours(pos, 0.8)
    x = a0 * 0.3 + 0.1j
    assert np.abs(system.apply_KT_blocks(nmax, K0, pos, Tb, x, nbr) - system.apply_KT(nmax, K0, pos, t, x, nbr)).max() <= 1e-13
