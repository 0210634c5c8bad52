"""Pin metrics for the oracle, shared by the pin tests and by the planted-
mistake tests (which patch a mistake into the oracle and check that some pin
catches it). Each function returns an error measure that is ~1e-12 for a
correct oracle."""
import math

import numpy as np
import scipy.special as sp

from oracle import field, incident, mie, system, translation, vswf
from paper_2107_09879_b300 import workloads as W

K0 = 2 * math.pi


def addition_theorem_error(nmax=3, d=(0.5, 0.2, 0.3), npts=6, seed=0, extra=20):
    """max relative error of Phi(k(x - x_a)) = sum xi(k(x_b - x_a)) RPhi(k(x - x_b))."""
    rng = np.random.default_rng(seed)
    xa = np.zeros(3)
    xb = np.asarray(d, dtype=np.float64)
    nbig = nmax + extra
    X = translation.xi_matrix(nmax, nbig, K0, xb - xa)
    err = 0.0
    for _ in range(npts):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x = xb + 0.25 * np.linalg.norm(xb - xa) * rng.uniform(0.1, 1.0) * u
        lhs = vswf.vswf(nmax, K0, x - xa)
        rhs = X @ vswf.vswf(nbig, K0, x - xb, regular=True)
        err = max(err, np.max(np.abs(lhs - rhs)) / np.max(np.abs(lhs)))
    return err


def planewave_error(nmax=20, beta=0.4, alpha=1.1, npts=5, seed=1):
    rng = np.random.default_rng(seed)
    bh = incident.beta_hat(beta, alpha)
    ah = incident.alpha_hat(beta, alpha)
    A = 0.6 * bh + 0.8j * ah
    a = incident.planewave_coeffs(nmax, beta, alpha, A)
    err = 0.0
    for _ in range(npts):
        x = rng.normal(size=3) * 0.2
        E = incident.planewave_field(K0, beta, alpha, A, x[None])[0]
        err = max(err, np.max(np.abs(E - a @ vswf.vswf(nmax, K0, x, regular=True))))
    return err


def far_power(nmax, pos, s, nth=40, nph=80):
    """Scattered power by Gauss-Legendre x trapezoid quadrature of |F|^2 / k^2."""
    xg, wg = np.polynomial.legendre.leggauss(nth)
    dirs = [(math.acos(x), 2 * math.pi * j / nph) for x in xg for j in range(nph)]
    F = field.far_field(nmax, K0, pos, s, dirs)
    w = np.repeat(wg, nph) * 2 * math.pi / nph
    return float(np.sum(w * np.sum(np.abs(F) ** 2, axis=1)) / K0 ** 2)


def energy_balance_error(nx=3, ny=3, nmax=3, beta_deg=10.0, seed=123, z_jitter=0.0):
    """|P_ext - P_sca| / P_sca for a lossless array, P_ext from coefficients
    (extinction, -(pi/k^2) Re sum a0^H s) and P_sca from far-field quadrature."""
    pos = W.lattice_positions(nx, ny)
    if z_jitter:
        g = W.SplitMix64(seed + 1)
        pos[:, 2] = z_jitter * (g.uniforms(len(pos)) - 0.5)
    r = W.uniform_radii(nx * ny, 0.08, 0.2, seed)
    T = np.array([mie.tmatrix_diag(nmax, K0, rr, 2.0) for rr in r])
    beta = math.radians(beta_deg)
    a0 = incident.planewave_incident(nmax, K0, pos, beta, 0.0, incident.beta_hat(beta, 0.0))
    s = system.solve_dense(nmax, K0, pos, T, a0)
    pext = -np.real(np.vdot(a0, s)) * math.pi / K0 ** 2
    psca = far_power(nmax, pos, s, nth=30, nph=60)
    return abs(pext - psca) / psca


def mie_dipole_pattern_ratio(x=0.05, m=1.5):
    """A small sphere under x-polarised normal incidence radiates like an electric
    dipole along x: the far field vanishes along +x and is maximal along +y.
    Returns |F(+x)|^2 / |F(+y)|^2 (should be ~ (b1/a1)^2 ~ x^4)."""
    nmax = 2
    t = mie.tmatrix_diag(nmax, K0, x / K0, m)
    a0 = incident.planewave_coeffs(nmax, 0.0, 0.0, [1.0, 0.0, 0.0])
    s = (t * a0)[None, :]
    F = field.far_field(nmax, K0, np.zeros((1, 3)), s, [(math.pi / 2, 0.0), (math.pi / 2, math.pi / 2)])
    return float(np.sum(np.abs(F[0]) ** 2) / np.sum(np.abs(F[1]) ** 2))


def mie_extinction_error(x=1.3, m=2.0, nmax=8):
    """Single sphere: extinction from coefficients vs Bohren-Huffman C_ext =
    (2 pi / k^2) sum (2l+1) Re(a_l + b_l), and far-field quadrature vs C_sca."""
    r = x / K0
    a, b = mie.mie_ab(nmax, K0, r, m)
    cext = 2 * math.pi / K0 ** 2 * sum((2 * l + 1) * (a[l] + b[l]).real for l in range(1, nmax + 1))
    csca = 2 * math.pi / K0 ** 2 * sum((2 * l + 1) * (abs(a[l]) ** 2 + abs(b[l]) ** 2) for l in range(1, nmax + 1))
    t = mie.tmatrix_diag(nmax, K0, r, m)
    a0 = incident.planewave_coeffs(nmax, 0.0, 0.0, [1.0, 0.0, 0.0])
    s = t * a0
    pext = -np.real(np.vdot(a0, s)) * math.pi / K0 ** 2
    psca = far_power(nmax, np.zeros((1, 3)), s[None, :], nth=20, nph=40)
    return max(abs(pext - cext) / cext, abs(psca - csca) / csca)
