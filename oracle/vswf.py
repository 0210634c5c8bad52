"""Vector spherical wave functions, App. I-A (Eq. vector_spherical_wf).

Scalar waves  phi_lm  = h_l(kr) Pbar_l^{|m|}(cos th) e^{i m ph},
              Rphi_lm = j_l(kr) Pbar_l^{|m|}(cos th) e^{i m ph}.
Vector waves  Phi_{lm0} = (1/sqrt(2l(l+1))) grad(phi_lm) x r
              Phi_{lm1} = (1/k) curl Phi_{lm0}
(and the regular versions RPhi with j_l). Written out in spherical components:
  Phi_{lm0} = c_l z_l(kr) [ i m pi_l^{|m|} th^ - tau_l^{|m|} ph^ ] e^{i m ph}
  Phi_{lm1} = c_l [ l(l+1) z_l(kr)/(kr) Pbar_l^{|m|} r^
                   + ((kr z_l)'/(kr)) ( tau_l^{|m|} th^ + i m pi_l^{|m|} ph^ ) ] e^{i m ph}
with c_l = 1/sqrt(2l(l+1)), z_l = h_l^(1) (Phi) or j_l (RPhi). These closed forms
are pinned in the tests against a finite-difference curl of the definition.

Coefficient order (used everywhere in this repository):
  n(l, m) = l(l+1) + m - 1  in [0, L),  L = nmax(nmax+2),
  flat index = p * L + n(l, m)   (polarisation-major), P = 2L.
"""
import math

import numpy as np

from .specfun import legendre_norm, sph_h1_all, sph_jn_all


def n_index(l, m):
    return l * (l + 1) + m - 1


def num_coeffs(nmax):
    return 2 * nmax * (nmax + 2)


def lm_list(nmax):
    """[(l, m)] in n(l, m) order."""
    return [(l, m) for l in range(1, nmax + 1) for m in range(-l, l + 1)]


def _sph_to_cart(th, ph):
    st, ct, sp, cp = math.sin(th), math.cos(th), math.sin(ph), math.cos(ph)
    rhat = np.array([st * cp, st * sp, ct])
    thhat = np.array([ct * cp, ct * sp, -st])
    phhat = np.array([-sp, cp, 0.0])
    return rhat, thhat, phhat


def vswf(nmax, k, x, regular=False):
    """Phi (regular=False) or RPhi (regular=True) at the point x (3-vector,
    relative to the expansion centre), wave number k (complex allowed for RPhi:
    the field inside a lossy scatterer). Returns complex array of shape (P, 3):
    row p*L + n(l,m) holds the Cartesian vector."""
    x = np.asarray(x, dtype=np.float64)
    r = float(np.linalg.norm(x))
    if r == 0.0:
        raise ValueError("VSWF evaluated at the expansion centre")
    th = math.acos(max(-1.0, min(1.0, x[2] / r)))
    ph = math.atan2(x[1], x[0])
    rho = k * r
    if regular:
        # a complex wave number (lossy medium, inside a scatterer) keeps complex j_l
        z = sph_jn_all(nmax, rho)
        if np.imag(k) == 0:
            z = z.real.astype(np.complex128)
    else:
        if np.imag(k) != 0:
            raise ValueError("outgoing waves need a real wave number")
        z = sph_h1_all(nmax, float(np.real(rho)))
    # (rho z_l)'/rho = z_{l-1} - l z_l / rho
    P, pi, tau = legendre_norm(nmax, th)
    rhat, thhat, phhat = _sph_to_cart(th, ph)
    L = nmax * (nmax + 2)
    out = np.zeros((2 * L, 3), dtype=np.complex128)
    for l in range(1, nmax + 1):
        cl = 1.0 / math.sqrt(2.0 * l * (l + 1))
        dz = z[l - 1] - l * z[l] / rho
        for m in range(-l, l + 1):
            am = abs(m)
            e = complex(math.cos(m * ph), math.sin(m * ph))
            pim = pi[l, am] * m  # m * pi_l^{|m|}
            M = cl * z[l] * (1j * pim * thhat - tau[l, am] * phhat) * e
            N = cl * (l * (l + 1) * z[l] / rho * P[l, am] * rhat
                      + dz * (tau[l, am] * thhat + 1j * pim * phhat)) * e
            n = n_index(l, m)
            out[n] = M
            out[L + n] = N
    return out
