"""Translation (addition) theorem coefficients, App. I-C (Eqs. tran_coeff).

    Phi_{lmp}(k(x - x_a)) = sum_{l'm'p'} xi_{lmp; l'm'p'}(k d) RPhi_{l'm'p'}(k(x - x_b)),
    d = x_b - x_a,  valid for |x - x_b| < |d|,

    xi = delta_{pp'} alpha + (1 - delta_{pp'}) beta,
    alpha_{lm;l'm'}(kd) = e^{i(m-m') phi_d} sum_q a5(l,m|l',m'|q) h_q(k|d|) Pbar_q^{|m-m'|}(cos th_d)
    beta_{lm;l'm'}(kd)  = e^{i(m-m') phi_d} sum_q b5(l,m|l',m'|q) h_q(k|d|) Pbar_q^{|m-m'|}(cos th_d)

Readings of the printed equations (each confirmed by the pointwise addition-
theorem test, which fails for the literal alternatives):
  * the expansion on the right is in REGULAR waves RPhi about x_b, and the
    displacement argument is x_b - x_a (the new centre minus the old one);
  * the last argument of a5/b5 is the summation order q (not the polarisation);
  * the denominator under the square root is 2 l(l+1) l'(l'+1);
  * beta's second 3j symbol is (l l' q-1; 0 0 0).
With j_q in place of h_q the same formula gives the regular-to-regular
translation R xi (valid everywhere).
"""
import math
from functools import lru_cache

import numpy as np

from .specfun import legendre_norm, sph_h1_all, sph_jn_all, wigner3j
from .vswf import lm_list


def a5b5(l, m, lp, mp, q):
    """Coupling constants a5(l,m|l',m'|q), b5(l,m|l',m'|q) of Eq. tran_coeff."""
    ipow = abs(m - mp) - abs(m) - abs(mp) + lp - l + q
    jf = (1j ** (ipow % 4)) * (-1) ** ((m - mp) % 2)
    f1 = math.sqrt((2 * l + 1) * (2 * lp + 1) / (2.0 * l * (l + 1) * lp * (lp + 1)))
    fa = (l * (l + 1) + lp * (lp + 1) - q * (q + 1)) * math.sqrt(2 * q + 1)
    arg = (l + lp + 1 + q) * (l + lp + 1 - q) * (q + l - lp) * (q - l + lp) * (2 * q + 1)
    fb = math.sqrt(arg) if arg > 0 else 0.0
    w1 = wigner3j(l, lp, q, m, -mp, mp - m)
    a = jf * f1 * fa * w1 * wigner3j(l, lp, q, 0, 0, 0)
    b = jf * f1 * fb * w1 * wigner3j(l, lp, q - 1, 0, 0, 0) if q >= 1 else 0.0
    return complex(a), complex(b)


@lru_cache(maxsize=None)
def coupling_tables(nmax_row, nmax_col):
    """Tables CA[n, n', q] = a5, CB[n, n', q] = b5 for all row (l,m) up to
    nmax_row, column (l',m') up to nmax_col and q = 0..nmax_row+nmax_col."""
    rows = lm_list(nmax_row)
    cols = lm_list(nmax_col)
    Q = nmax_row + nmax_col + 1
    CA = np.zeros((len(rows), len(cols), Q), dtype=np.complex128)
    CB = np.zeros((len(rows), len(cols), Q), dtype=np.complex128)
    MU = np.zeros((len(rows), len(cols)), dtype=np.int64)
    for i, (l, m) in enumerate(rows):
        for j, (lp, mp) in enumerate(cols):
            MU[i, j] = m - mp
            for q in range(abs(l - lp), l + lp + 1):
                if abs(m - mp) > q:
                    continue  # Pbar_q^{|m-m'|} = 0
                CA[i, j, q], CB[i, j, q] = a5b5(l, m, lp, mp, q)
    return CA, CB, MU


def xi_matrix(nmax_row, nmax_col, k, d, regular=False):
    """xi(k d) as a (2 L_row) x (2 L_col) matrix in the flat (p, n) order.
    regular=False: outgoing -> regular (h_q); regular=True: R xi (j_q)."""
    d = np.asarray(d, dtype=np.float64)
    r = float(np.linalg.norm(d))
    th = math.acos(max(-1.0, min(1.0, d[2] / r)))
    ph = math.atan2(d[1], d[0])
    Q = nmax_row + nmax_col
    z = sph_jn_all(Q, k * r).real.astype(np.complex128) if regular else sph_h1_all(Q, k * r)
    P, _, _ = legendre_norm(Q, th)
    CA, CB, MU = coupling_tables(nmax_row, nmax_col)
    absmu = np.abs(MU)
    # radial-polar factor per (n, n', q): z_q * Pbar_q^{|mu|}(cos th)
    fac = z[None, None, :] * P[:, absmu].transpose(1, 2, 0)
    phase = np.exp(1j * MU * ph)
    alpha = phase * np.sum(CA * fac, axis=2)
    beta = phase * np.sum(CB * fac, axis=2)
    Lr, Lc = alpha.shape
    X = np.zeros((2 * Lr, 2 * Lc), dtype=np.complex128)
    X[:Lr, :Lc] = alpha
    X[Lr:, Lc:] = alpha
    X[:Lr, Lc:] = beta
    X[Lr:, :Lc] = beta
    return X


def coupling_block(nmax, k, x_target, x_source):
    """Block A_ts of the interaction operator: the regular-wave coefficients at
    the target produced by unit outgoing coefficients at the source,
    a_t += A_ts s_s with A_ts = xi(k (x_t - x_s))^T (App. I-C, Eq. final_linear_eqs)."""
    d = np.asarray(x_target, dtype=np.float64) - np.asarray(x_source, dtype=np.float64)
    return xi_matrix(nmax, nmax, k, d).T
