"""Special functions for the oracle (fp64 / complex128), written from their
textbook definitions. App. I-A of the paper defines the wave functions in terms
of these; App. I-C uses the Wigner-3j symbols in the translation coefficients.

Nothing here calls scipy/sympy/mpmath: those libraries are only used by the
tests to pin these functions.
"""
import math
from fractions import Fraction

import numpy as np


# ----------------------------------------------------------------------------
# Spherical Bessel functions (Abramowitz & Stegun 10.1)
# ----------------------------------------------------------------------------

def sph_jn_all(lmax, z):
    """j_0..j_lmax at (real or complex) z. Scalar z.

    Upward recurrence j_{l+1} = (2l+1)/z j_l - j_{l-1} is unstable for l > |z|,
    so the values are obtained by Miller's downward recurrence started well
    above lmax and normalised to j_0 = sin z / z (A&S 10.1.19 / 10.5).
    """
    z = complex(z)
    out = np.zeros(lmax + 1, dtype=np.complex128)
    if abs(z) < 1e-300:
        out[0] = 1.0
        return out
    start = lmax + int(abs(z)) + 40
    jp1 = 0.0 + 0.0j
    jc = 1e-300 + 0.0j
    vals = {}
    for l in range(start, 0, -1):
        jm1 = (2 * l + 1) / z * jc - jp1
        jp1, jc = jc, jm1
        if l - 1 <= max(lmax, 1):
            vals[l - 1] = jc
        if abs(jc) > 1e250:  # rescale to avoid overflow
            jp1 /= 1e250
            jc /= 1e250
            for key in vals:
                vals[key] /= 1e250
    # normalise with whichever of j_0 = sin z / z, j_1 = sin z / z^2 - cos z / z
    # is larger (their zeros interlace, so one of them is never small)
    j0 = np.sin(z) / z
    j1 = np.sin(z) / (z * z) - np.cos(z) / z
    if abs(j0) >= abs(j1) or lmax < 1 and abs(j0) > 0:
        scale = j0 / vals[0]
    else:
        v1 = vals[1] if 1 in vals else (3.0 / z * vals[0])  # never reached for lmax >= 1
        scale = j1 / v1
    for l in range(lmax + 1):
        out[l] = vals[l] * scale
    return out


def sph_yn_all(lmax, z):
    """y_0..y_lmax at z by the (stable) upward recurrence, A&S 10.1.12/10.1.19."""
    z = complex(z)
    out = np.zeros(lmax + 1, dtype=np.complex128)
    out[0] = -np.cos(z) / z
    if lmax >= 1:
        out[1] = -np.cos(z) / (z * z) - np.sin(z) / z
    for l in range(1, lmax):
        out[l + 1] = (2 * l + 1) / z * out[l] - out[l - 1]
    return out


def sph_h1_all(lmax, x):
    """Spherical Hankel functions of the first kind h_l^(1) = j_l + i y_l for
    real x > 0 (App. I-A, outgoing waves for exp(-i omega t))."""
    j = sph_jn_all(lmax, x).real
    y = sph_yn_all(lmax, x).real
    return j + 1j * y


def riccati_psi_all(lmax, z):
    """psi_l(z) = z j_l(z) and its derivative psi_l'(z) = z j_{l-1}(z) - l j_l(z)."""
    j = sph_jn_all(lmax + 1, z)
    psi = z * j[: lmax + 1]
    dpsi = np.zeros(lmax + 1, dtype=np.complex128)
    dpsi[0] = np.cos(z)  # d/dz sin z
    for l in range(1, lmax + 1):
        dpsi[l] = z * j[l - 1] - l * j[l]
    return psi, dpsi


def riccati_xi_all(lmax, x):
    """xi_l(x) = x h_l^(1)(x) and xi_l'(x) = x h_{l-1}(x) - l h_l(x), real x."""
    h = sph_h1_all(lmax + 1, x)
    xi = x * h[: lmax + 1]
    dxi = np.zeros(lmax + 1, dtype=np.complex128)
    dxi[0] = np.cos(x) + 1j * np.sin(x)  # d/dx (-i e^{ix}) = e^{ix}
    for l in range(1, lmax + 1):
        dxi[l] = x * h[l - 1] - l * h[l]
    return xi, dxi


# ----------------------------------------------------------------------------
# Normalised associated Legendre functions (App. I-A; the normalisation is the
# one of Doicu et al., App. B, which the paper says it follows):
#   Pbar_l^m(x) = sqrt((2l+1)/2 * (l-m)!/(l+m)!) P_l^m(x),  m >= 0,
#   P_l^m(x) = (1-x^2)^{m/2} d^m/dx^m P_l(x)   (no Condon-Shortley phase).
# ----------------------------------------------------------------------------

def legendre_norm(lmax, theta):
    """Return (P, pi, tau), each of shape (lmax+1, lmax+1) indexed [l, m]:
    P[l,m]   = Pbar_l^m(cos theta)
    pi[l,m]  = Pbar_l^m(cos theta) / sin theta   (m >= 1; 0 for m = 0)
    tau[l,m] = d Pbar_l^m(cos theta) / d theta
    computed by the standard three-term recurrence in l (pi by the same
    recurrence, which keeps it finite at the poles)."""
    c = math.cos(theta)
    s = math.sin(theta)
    P = np.zeros((lmax + 1, lmax + 1))
    pi = np.zeros((lmax + 1, lmax + 1))
    tau = np.zeros((lmax + 1, lmax + 1))
    for m in range(0, lmax + 1):
        # Pbar_m^m = sqrt((2m+1)/2 / (2m)!) (2m-1)!! s^m
        dfact = 1.0
        for k in range(1, 2 * m, 2):
            dfact *= k
        pmm_over_s = math.sqrt((2 * m + 1) / 2.0 / math.factorial(2 * m)) * dfact  # times s^(m-1)
        # pi-type sequence Q_l = Pbar_l^m / s (for m >= 1), P sequence = Q * s
        q_prev2 = 0.0
        q_prev1 = pmm_over_s * (s ** (m - 1) if m >= 1 else 0.0)
        p_prev2 = 0.0
        p_prev1 = pmm_over_s * (s ** m)
        P[m, m] = p_prev1
        if m >= 1:
            pi[m, m] = q_prev1
        for l in range(m + 1, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            p_new = a * (c * p_prev1 - b * p_prev2)
            q_new = a * (c * q_prev1 - b * q_prev2)
            P[l, m] = p_new
            if m >= 1:
                pi[l, m] = q_new
            p_prev2, p_prev1 = p_prev1, p_new
            q_prev2, q_prev1 = q_prev1, q_new
    # tau from the derivative identities of the normalised functions:
    #   m >= 1: tau_l^m = l cos(theta) pi_l^m - sqrt((2l+1)(l^2-m^2)/(2l-1)) pi_{l-1}^m
    #   m = 0 : tau_l^0 = -sqrt(l(l+1)) Pbar_l^1
    for l in range(0, lmax + 1):
        tau[l, 0] = -math.sqrt(l * (l + 1.0)) * P[l, 1] if (l >= 1 and lmax >= 1) else 0.0
        for m in range(1, l + 1):
            prev = pi[l - 1, m] if l - 1 >= m else 0.0
            tau[l, m] = l * c * pi[l, m] - math.sqrt((2.0 * l + 1) * (l * l - m * m) / (2.0 * l - 1)) * prev
    return P, pi, tau


# ----------------------------------------------------------------------------
# Wigner-3j symbols (App. I-C, Eq. tran_coeff), Racah's closed form evaluated in
# exact rational arithmetic, then one square root in floating point.
# ----------------------------------------------------------------------------

def wigner3j(j1, j2, j3, m1, m2, m3):
    """( j1 j2 j3 ; m1 m2 m3 ) for integer arguments, Racah's formula."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    if min(j1, j2, j3) < 0:
        return 0.0
    f = math.factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pref = tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    ssum = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(j3 - j2 + k + m1) * f(j3 - j1 + k - m2) * f(j1 + j2 - j3 - k)
               * f(j1 - k - m1) * f(j2 - k + m2))
        ssum += Fraction((-1) ** k, den)
    sign = (-1) ** (j1 - j2 - m3)
    # value = sign * sqrt(pref) * ssum ; keep exactness until the single sqrt
    val2 = pref * ssum * ssum
    mag = math.sqrt(float(val2))  # val2 <= 1: Fraction -> float is correctly rounded
    return float(sign * (1 if ssum >= 0 else -1) * mag)
