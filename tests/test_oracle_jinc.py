"""Pins of the jinc-source incident coefficients (App. II): the expansion about
a sphere reproduces the closed-form jinc field on the source plane; the
propagated field agrees with a direct angular-spectrum integral; linearity over
source groups; convergence of the quadrature rule."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import incident, vswf

K0 = 2 * math.pi
Z0 = -1.0


def _field_from_coeffs(a, xj, pts, nmax):
    return np.array([a @ vswf.vswf(nmax, K0, p - xj, regular=True) for p in pts])


def test_source_plane_field_is_the_jinc_sum():
    """On z = z0 the transverse field of the group is sum_s A_s (pi/2) J1(k0 rho)/(k0 rho)
    (cylindrical J_1, lambda/2-cell weight): closed form with scipy's J_1."""
    src = np.array([[0.0, 0.0], [0.5, 0.0]])
    A = np.array([[1.0, 0.0], [0.3j, 0.8]])
    xj = np.array([0.3, -0.2, Z0])
    rule = incident.jinc_rule(*incident.jinc_rule_size(K0, 2.0))
    a = incident.jinc_group_coeffs(18, K0, xj[None], src, A, Z0, rule)[0]
    rng = np.random.default_rng(0)
    pts = []
    for _ in range(6):
        p = xj + rng.normal(size=3) * 0.12
        p[2] = Z0
        pts.append(p)
    E = _field_from_coeffs(a, xj, pts, 18)
    for p, e in zip(pts, E):
        ref = np.zeros(2, dtype=complex)
        for s, amp in zip(src, A):
            rho = math.hypot(p[0] - s[0], p[1] - s[1])
            ref += amp * (math.pi / 2) * (sp.j1(K0 * rho) / (K0 * rho) if rho > 0 else 0.5)
        assert np.max(np.abs(e[:2] - ref)) < 1e-11


def test_source_plane_field_on_a_coarser_grid():
    """Grid pitch a != lambda/2: the kernel is (a^2 k0^2 / (2 pi)) J1(k0 rho)/(k0 rho)."""
    a = 0.45 / 0.9 * 1.0  # pitch 0.5 at wavelength 0.9 -> k0 = 2 pi / 0.9
    k0 = 2 * math.pi / 0.9
    src = np.array([[0.0, 0.0]])
    A = np.array([[0.7, -0.2j]])
    xj = np.array([0.2, 0.1, Z0])
    rule = incident.jinc_rule(*incident.jinc_rule_size(k0, 2.0))
    coef = incident.jinc_group_coeffs(16, k0, xj[None], src, A, Z0, rule, pitch=0.5)[0]
    for d in ([0.05, 0.02], [-0.1, 0.08]):
        p = xj + np.array([d[0], d[1], 0.0])
        E = coef @ vswf.vswf(16, k0, p - xj, regular=True)
        rho = math.hypot(p[0], p[1])
        ref = A[0] * (0.5 ** 2 * k0 ** 2 / (2 * math.pi)) * sp.j1(k0 * rho) / (k0 * rho)
        assert np.max(np.abs(E[:2] - ref)) < 1e-11


def test_propagated_field_matches_direct_angular_spectrum():
    """Off the source plane: sum a RPhi equals the angular-spectrum integral of the
    source evaluated directly (no spherical-wave expansion), with a finer rule."""
    src = np.array([[0.2, -0.1]])
    A = np.array([[0.6, 0.4j]])
    xj = np.array([0.4, 0.3, 0.0])
    rule = incident.jinc_rule(*incident.jinc_rule_size(K0, 2.0))
    a = incident.jinc_group_coeffs(16, K0, xj[None], src, A, Z0, rule)[0]
    pts = [xj + np.array([0.1, -0.05, 0.08]), xj + np.array([-0.12, 0.02, -0.1])]
    E = _field_from_coeffs(a, xj, pts, 16)
    beta, wb, alpha, wa = incident.jinc_rule(80, 96)
    for p, e in zip(pts, E):
        ref = np.zeros(3, dtype=complex)
        for ib, b in enumerate(beta):
            for al in alpha:
                kx, ky, kz = K0 * math.sin(b) * math.cos(al), K0 * math.sin(b) * math.sin(al), K0 * math.cos(b)
                S = A[0] * np.exp(-1j * (kx * src[0, 0] + ky * src[0, 1]))
                Avec = np.array([S[0], S[1], -(kx * S[0] + ky * S[1]) / kz])
                ref += 0.25 * wb[ib] * wa * math.sin(b) * math.cos(b) * Avec * np.exp(
                    1j * (kx * p[0] + ky * p[1] + kz * (p[2] - Z0)))
        assert np.max(np.abs(e - ref)) < 1e-9


def test_group_linearity():
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0]])
    s1, A1 = np.array([[0.0, 0.0], [0.5, 0.0]]), np.array([[1.0, 0.0], [0.0, 1.0j]])
    s2, A2 = np.array([[0.0, 0.5]]), np.array([[0.2, 0.3]])
    rule = incident.jinc_rule(30, 40)
    a1 = incident.jinc_group_coeffs(3, K0, pos, s1, A1, Z0, rule)
    a2 = incident.jinc_group_coeffs(3, K0, pos, s2, A2, Z0, rule)
    a12 = incident.jinc_group_coeffs(3, K0, pos, np.vstack([s1, s2]), np.vstack([A1, A2]), Z0, rule)
    assert np.max(np.abs(a1 + a2 - a12)) < 1e-14 * np.max(np.abs(a12))


def test_rule_convergence():
    """The rule sized from the largest sphere-source distance is converged: a finer
    rule changes the coefficients by < 1e-10 relative."""
    pos = np.array([[1.0, 0.5, 0.0], [-0.5, 1.0, 0.0]])
    src = np.array([[0.0, 0.0], [0.5, 0.5], [-0.5, 0.0]])
    A = np.array([[1.0, 0.0], [0.5, 0.5], [0.0, 1.0]])
    ext = max(np.linalg.norm(np.array([p[0] - s[0], p[1] - s[1], p[2] - Z0])) for p in pos for s in src)
    nb, na = incident.jinc_rule_size(K0, ext)
    a = incident.jinc_group_coeffs(3, K0, pos, src, A, Z0, incident.jinc_rule(nb, na))
    b = incident.jinc_group_coeffs(3, K0, pos, src, A, Z0, incident.jinc_rule(nb + nb // 2, na + na // 2))
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(a))
