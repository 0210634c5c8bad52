"""Sphere T-matrix: the closed-form (Mie) special case of the per-scatterer
T-matrix of App. I-B (Eq. def_tmatrix, s = T a). For a sphere T is diagonal in
(l, m, p) and independent of m:

    t_{l, p=0} = -b_l     (p = 0 waves are the magnetic / M-type ones)
    t_{l, p=1} = -a_l     (p = 1 waves are the electric / N-type ones)

with the Lorenz-Mie coefficients (Bohren & Huffman, Eq. 4.53) in terms of the
Riccati-Bessel functions psi_l(z) = z j_l(z), xi_l(x) = x h_l^(1)(x),
size parameter x = k r and relative index m_s = n_sphere / n_background:

    a_l = [m psi(mx) psi'(x) - psi(x) psi'(mx)] / [m psi(mx) xi'(x) - xi(x) psi'(mx)]
    b_l = [psi(mx) psi'(x) - m psi(x) psi'(mx)] / [psi(mx) xi'(x) - m xi(x) psi'(mx)]

The radius derivative (App. IV, dT/dp for the geometric parameter p = radius)
follows by the chain rule through x = k r and m x, using the Riccati-Bessel
equation f''(z) = (l(l+1)/z^2 - 1) f(z) for f = psi, xi.
"""
import numpy as np

from .specfun import riccati_psi_all, riccati_xi_all


def mie_ab(nmax, k, radius, m_rel):
    """(a_l, b_l) for l = 1..nmax (index 0 unused), complex arrays of length nmax+1."""
    x = k * radius
    mx = m_rel * x
    psi_x, dpsi_x = riccati_psi_all(nmax, x)
    xi_x, dxi_x = riccati_xi_all(nmax, x)
    psi_mx, dpsi_mx = riccati_psi_all(nmax, mx)
    a = np.zeros(nmax + 1, dtype=np.complex128)
    b = np.zeros(nmax + 1, dtype=np.complex128)
    for l in range(1, nmax + 1):
        a[l] = ((m_rel * psi_mx[l] * dpsi_x[l] - psi_x[l] * dpsi_mx[l])
                / (m_rel * psi_mx[l] * dxi_x[l] - xi_x[l] * dpsi_mx[l]))
        b[l] = ((psi_mx[l] * dpsi_x[l] - m_rel * psi_x[l] * dpsi_mx[l])
                / (psi_mx[l] * dxi_x[l] - m_rel * xi_x[l] * dpsi_mx[l]))
    return a, b


def mie_ab_dr(nmax, k, radius, m_rel):
    """d a_l / d r and d b_l / d r (quotient rule, chain rule via x = k r)."""
    x = k * radius
    mx = m_rel * x
    psi_x, dpsi_x = riccati_psi_all(nmax, x)
    xi_x, dxi_x = riccati_xi_all(nmax, x)
    psi_mx, dpsi_mx = riccati_psi_all(nmax, mx)
    da = np.zeros(nmax + 1, dtype=np.complex128)
    db = np.zeros(nmax + 1, dtype=np.complex128)
    m = m_rel
    for l in range(1, nmax + 1):
        ll = l * (l + 1.0)
        d2psi_x = (ll / x ** 2 - 1.0) * psi_x[l]
        d2xi_x = (ll / x ** 2 - 1.0) * xi_x[l]
        d2psi_mx = (ll / mx ** 2 - 1.0) * psi_mx[l]
        # d/dr of each factor: f(x) -> k f'(x), g(mx) -> m k g'(mx)
        p_x, dp_x, dd_p_x = psi_x[l], dpsi_x[l], d2psi_x
        q_x, dq_x, dd_q_x = xi_x[l], dxi_x[l], d2xi_x
        p_m, dp_m, dd_p_m = psi_mx[l], dpsi_mx[l], d2psi_mx
        # a_l = Na / Da
        Na = m * p_m * dp_x - p_x * dp_m
        Da = m * p_m * dq_x - q_x * dp_m
        dNa = k * (m * m * dp_m * dp_x + m * p_m * dd_p_x - dp_x * dp_m - p_x * m * dd_p_m)
        dDa = k * (m * m * dp_m * dq_x + m * p_m * dd_q_x - dq_x * dp_m - q_x * m * dd_p_m)
        da[l] = (dNa * Da - Na * dDa) / Da ** 2
        # b_l = Nb / Db
        Nb = p_m * dp_x - m * p_x * dp_m
        Db = p_m * dq_x - m * q_x * dp_m
        dNb = k * (m * dp_m * dp_x + p_m * dd_p_x - m * dp_x * dp_m - m * m * p_x * dd_p_m)
        dDb = k * (m * dp_m * dq_x + p_m * dd_q_x - m * dq_x * dp_m - m * m * q_x * dd_p_m)
        db[l] = (dNb * Db - Nb * dDb) / Db ** 2
    return da, db


def tmatrix_diag(nmax, k, radius, m_rel):
    """Diagonal of the sphere T-matrix in the flat order p*L + n(l, m)."""
    a, b = mie_ab(nmax, k, radius, m_rel)
    L = nmax * (nmax + 2)
    t = np.zeros(2 * L, dtype=np.complex128)
    for l in range(1, nmax + 1):
        for m in range(-l, l + 1):
            n = l * (l + 1) + m - 1
            t[n] = -b[l]
            t[L + n] = -a[l]
    return t


def tmatrix_diag_dr(nmax, k, radius, m_rel):
    """d/dr of tmatrix_diag."""
    da, db = mie_ab_dr(nmax, k, radius, m_rel)
    L = nmax * (nmax + 2)
    t = np.zeros(2 * L, dtype=np.complex128)
    for l in range(1, nmax + 1):
        for m in range(-l, l + 1):
            n = l * (l + 1) + m - 1
            t[n] = -db[l]
            t[L + n] = -da[l]
    return t
