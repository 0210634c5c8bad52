"""Field evaluation, App. I-C (Eq. sca_fld_concise):
    E_sca(x) = sum_i s_i^T Phi(k(x - x_i)),
and the far-field amplitude F of the same field, defined by
    E_sca(r r^) -> e^{ikr}/(kr) F(r^)   (r -> infinity),
obtained from the large-argument form h_l(z) -> (-i)^{l+1} e^{iz}/z
(A&S 10.1.16; the paper's Eq. asymptotic omits the phase (-i)^{l+1}):
    M-type (p=0): F_n = c_l (-i)^{l+1} [ i m pi th^ - tau ph^ ] e^{i m ph}
    N-type (p=1): F_n = c_l (-i)^l     [ tau th^ + i m pi ph^ ] e^{i m ph}
and each scatterer contributes with the phase e^{-i k r^.x_i}.
"""
import math

import numpy as np

from .specfun import legendre_norm
from .vswf import _sph_to_cart, vswf


def scattered_field(nmax, k, pos, s, pts):
    """E_sca at points pts (M, 3) from coefficients s (N, P)."""
    pts = np.asarray(pts, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    E = np.zeros((pts.shape[0], 3), dtype=np.complex128)
    for a in range(pts.shape[0]):
        for i in range(pos.shape[0]):
            E[a] += s[i] @ vswf(nmax, k, pts[a] - pos[i])
    return E


def far_amplitudes(nmax, th, ph):
    """F_n(r^) for one direction: (P, 3) complex."""
    P_, pi, tau = legendre_norm(nmax, th)
    _, thhat, phhat = _sph_to_cart(th, ph)
    L = nmax * (nmax + 2)
    out = np.zeros((2 * L, 3), dtype=np.complex128)
    for l in range(1, nmax + 1):
        cl = 1.0 / math.sqrt(2.0 * l * (l + 1))
        for m in range(-l, l + 1):
            am = abs(m)
            e = complex(math.cos(m * ph), math.sin(m * ph))
            n = l * (l + 1) + m - 1
            out[n] = cl * ((-1j) ** ((l + 1) % 4)) * (1j * m * pi[l, am] * thhat - tau[l, am] * phhat) * e
            out[L + n] = cl * ((-1j) ** (l % 4)) * (tau[l, am] * thhat + 1j * m * pi[l, am] * phhat) * e
    return out


def far_field(nmax, k, pos, s, dirs):
    """Far-field amplitude F(r^) for each direction (theta, phi) in dirs."""
    pos = np.asarray(pos, dtype=np.float64)
    out = np.zeros((len(dirs), 3), dtype=np.complex128)
    for a, (th, ph) in enumerate(dirs):
        rhat = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        Fn = far_amplitudes(nmax, th, ph)
        for i in range(pos.shape[0]):
            out[a] += np.exp(-1j * k * (rhat @ pos[i])) * (s[i] @ Fn)
    return out
