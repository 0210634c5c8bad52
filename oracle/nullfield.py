"""T-matrix of a single scatterer by the null-field method (App. I-B, Eq. def_tmatrix and
the P, Q surface integrals). Test infrastructure, like the rest of this package.

With k_s the wave number inside the scatterer and k_b outside, for every pair of indices
nu = (l, m, p) (outside function) and mu = (l', m', p') (inside function):

  P[nu, mu] = surface integral of
      [ RPhi_{l' m' p'}(k_s x) x Phi_{l, -m, 1-p}(k_b x)
        + (k_s / k_b) RPhi_{l' m', 1-p'}(k_s x) x Phi_{l, -m, p}(k_b x) ] . n(x) dA
  Q[nu, mu] = the same with the regular RPhi(k_b x) in place of Phi(k_b x)

and T = -Q P^-1.

Readings (each pinned by a test in tests/test_oracle_nullfield.py):
  G16  The integrals run over the scatterer's own surface (the paper writes the enclosing
       sphere dS, on which the null-field equations do not hold for a non-spherical body).
  G17  The paper prints T = -P Q^-1 with P the matrix of outgoing functions. The
       null-field derivation (inside: the incident field is cancelled by the outgoing
       expansion of the surface currents, coefficients P c; outside: the scattered field
       is the regular expansion, -Q c) gives T = -Q P^-1; for a sphere it reduces to
       -(regular)/(outgoing), the Lorenz-Mie form, while the printed order gives its
       inverse.
  G18  The two terms of the integrand are added. On a sphere the p = 0 rows then reduce to
       b_l = [psi_l(mx) psi_l'(x) - m psi_l(x) psi_l'(mx)] / [the same with xi_l for psi_l at x]
       (Riccati-Bessel psi_l = x j_l, xi_l = x h_l), the Mie coefficient; the printed minus
       turns both inner minus signs into plus signs.
The surface integral is computed by quadrature over a surface given as points, unit
outward normals and area weights (Gauss-Legendre along each face, trapezoid in the
azimuth); nothing assumes rotational symmetry, so the axisymmetric structure of the
result (m = m' only) is a check, not an input.
"""
import math

import numpy as np

from . import vswf as V


def _gauss(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def surface_cylinder(radius, height, n_face, n_phi, z0=0.0):
    """An upright circular cylinder (axis along z, centred at (0, 0, z0)): points (Q, 3),
    outward unit normals (Q, 3) and area weights (Q,) of the bottom disc, the side and the
    top disc; n_face Gauss-Legendre nodes along each face's profile, n_phi azimuths."""
    phis = 2 * math.pi * np.arange(n_phi) / n_phi
    wphi = 2 * math.pi / n_phi
    pts, nrm, wts = [], [], []
    rho, wr = _gauss(n_face, 0.0, radius)
    zs, wz = _gauss(n_face, -0.5 * height, 0.5 * height)
    for ph in phis:
        c, s = math.cos(ph), math.sin(ph)
        for r, w in zip(rho, wr):  # discs: dA = rho drho dphi
            for zc, nz in ((-0.5 * height, -1.0), (0.5 * height, 1.0)):
                pts.append([r * c, r * s, z0 + zc])
                nrm.append([0.0, 0.0, nz])
                wts.append(w * r * wphi)
        for zz, w in zip(zs, wz):  # side: dA = radius dz dphi
            pts.append([radius * c, radius * s, z0 + zz])
            nrm.append([c, s, 0.0])
            wts.append(w * radius * wphi)
    return np.array(pts), np.array(nrm), np.array(wts)


def surface_sphere(radius, n_theta, n_phi):
    """A sphere of the given radius about the origin (points, normals, weights)."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    pts, nrm, wts = [], [], []
    for ph in 2 * math.pi * np.arange(n_phi) / n_phi:
        for c, w in zip(ct, wt):
            s = math.sqrt(1.0 - c * c)
            u = np.array([s * math.cos(ph), s * math.sin(ph), c])
            pts.append(radius * u)
            nrm.append(u)
            wts.append(w * radius * radius * 2 * math.pi / n_phi)
    return np.array(pts), np.array(nrm), np.array(wts)


def _partner(nmax):
    """For every flat index nu = (l, m, p): the flat indices of (l, -m, 1-p) and (l, -m, p)."""
    L = nmax * (nmax + 2)
    flip, same = np.zeros(2 * L, int), np.zeros(2 * L, int)
    for p in range(2):
        for l, m in V.lm_list(nmax):
            nu = p * L + V.n_index(l, m)
            flip[nu] = (1 - p) * L + V.n_index(l, -m)
            same[nu] = p * L + V.n_index(l, -m)
    return flip, same


def pq_matrices(nmax, k_b, k_s, surface):
    """P and Q (P x P, rows nu = outside index, columns mu = inside index) by quadrature."""
    pts, nrm, wts = surface
    L = nmax * (nmax + 2)
    flip, same = _partner(nmax)
    mu_bar = np.concatenate([np.arange(L, 2 * L), np.arange(0, L)])  # (l', m', 1 - p')
    Pm = np.zeros((2 * L, 2 * L), complex)
    Qm = np.zeros((2 * L, 2 * L), complex)
    for x, n, w in zip(pts, nrm, wts):
        Ri = V.vswf(nmax, k_s, x, regular=True)      # RPhi(k_s x), rows mu
        Ho = V.vswf(nmax, k_b, x, regular=False)     # Phi(k_b x)
        Ro = V.vswf(nmax, k_b, x, regular=True)      # RPhi(k_b x)
        for Out, M in ((Ho, Pm), (Ro, Qm)):
            # [RPhi_mu x Out_{nu~,1-p} + (k_s/k_b) RPhi_{mu bar} x Out_{nu~,p}] . n
            t1 = np.cross(Ri[None, :, :], Out[flip][:, None, :]) @ n
            t2 = np.cross(Ri[mu_bar][None, :, :], Out[same][:, None, :]) @ n
            M += w * (t1 + (k_s / k_b) * t2)
    return Pm, Qm


def tmatrix(nmax, k_b, m_rel, surface):
    """Full T-matrix (P x P, flat indices) of a homogeneous scatterer of relative
    refractive index m_rel bounded by `surface`: T = -Q P^-1 (G17)."""
    Pm, Qm = pq_matrices(nmax, k_b, m_rel * k_b, surface)
    return -Qm @ np.linalg.inv(Pm)


def cylinder_tmatrix(nmax, k_b, m_rel, radius, height, n_face=48, n_phi=None):
    """T-matrix of an upright cylinder centred at the origin."""
    n_phi = n_phi or 2 * nmax + 4  # exact for the azimuthal factors e^{i(m' - m) phi}
    return tmatrix(nmax, k_b, m_rel, surface_cylinder(radius, height, n_face, n_phi))
