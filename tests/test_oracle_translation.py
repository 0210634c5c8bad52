"""Pins of the translation coefficients (App. I-C, Eqs. tran_coeff) and of the
readings taken of the printed equations."""
import math

import numpy as np
import pytest

from oracle import translation, vswf
from oracle_pins import K0, addition_theorem_error


@pytest.mark.parametrize("d", [(0.5, 0.2, 0.3), (-0.4, 0.9, 0.0), (0.0, 0.0, 0.7), (1.5, -2.0, 0.0), (0.3, 0.1, -0.8)])
def test_addition_theorem_pointwise(d):
    """Phi(k(x-x_a)) = sum xi(k(x_b-x_a)) RPhi(k(x-x_b)) at random points."""
    assert addition_theorem_error(3, d) < 1e-10


def test_addition_theorem_nmax5():
    assert addition_theorem_error(5, (0.6, -0.35, 0.1), extra=20) < 1e-10


def test_printed_argument_sign_is_a_garble():
    """With the displacement x_a - x_b (as printed) the identity fails: the
    reading d = x_b - x_a is the one the mathematics fixes."""
    rng = np.random.default_rng(0)
    nmax, nbig = 3, 17
    xb = np.array([0.5, 0.2, 0.3])
    X = translation.xi_matrix(nmax, nbig, K0, -xb)
    x = xb + 0.1 * rng.normal(size=3)
    lhs = vswf.vswf(nmax, K0, x)
    rhs = X @ vswf.vswf(nbig, K0, x - xb, regular=True)
    assert np.max(np.abs(lhs - rhs)) / np.max(np.abs(lhs)) > 0.1


def test_regular_addition_theorem_pointwise():
    """RPhi(k(x - x_a)) = sum Rxi(k(x_b - x_a)) RPhi(k(x - x_b)) everywhere."""
    rng = np.random.default_rng(2)
    nmax, nbig = 3, 25
    xb = np.array([0.3, -0.2, 0.25])
    X = translation.xi_matrix(nmax, nbig, K0, xb, regular=True)
    for _ in range(4):
        x = rng.normal(size=3) * 0.3
        lhs = vswf.vswf(nmax, K0, x, regular=True)
        rhs = X @ vswf.vswf(nbig, K0, x - xb, regular=True)
        assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(lhs))


def test_regular_translation_there_and_back():
    """Rxi(d) Rxi(-d) restricted to the nmax block tends to the identity as the
    intermediate truncation grows."""
    nmax = 3
    d = np.array([0.35, 0.2, 0.0])
    errs = []
    for mid in [4, 8, 14]:
        F = translation.xi_matrix(nmax, mid, K0, d, regular=True)
        B = translation.xi_matrix(mid, nmax, K0, -d, regular=True)
        errs.append(np.max(np.abs(F @ B - np.eye(F.shape[0]))))
    assert errs[-1] < 1e-10 and errs[0] > errs[-1]


def test_planar_parity_decoupling():
    """At theta = pi/2 entries linking (l+m+p) classes of different parity vanish."""
    nmax = 4
    L = nmax * (nmax + 2)
    X = translation.xi_matrix(nmax, nmax, K0, np.array([1.1, -0.7, 0.0]))
    cls = np.array([(l + m) % 2 for (l, m) in vswf.lm_list(nmax)] + [(l + m + 1) % 2 for (l, m) in vswf.lm_list(nmax)])
    mask = cls[:, None] != cls[None, :]
    assert np.max(np.abs(X[mask])) < 1e-15
    assert np.min(np.abs(X[~mask])) >= 0  # the rest is generically non-zero
    assert np.count_nonzero(np.abs(X) > 1e-14) <= (2 * L) ** 2 // 2


def test_inversion_symmetry():
    """xi(-d) = S xi(d) S with S = diag((-1)^{l+p})."""
    nmax = 4
    S = np.diag([(-1) ** l for (l, m) in vswf.lm_list(nmax)] + [(-1) ** (l + 1) for (l, m) in vswf.lm_list(nmax)])
    d = np.array([0.7, -0.3, 0.2])
    assert np.max(np.abs(translation.xi_matrix(nmax, nmax, K0, -d) - S @ translation.xi_matrix(nmax, nmax, K0, d) @ S)) < 1e-13


@pytest.mark.parametrize("d", [(1.0, 0.5), (0.3, -1.7), (2.5, 1.0), (-0.8, 0.0), (0.0, 1.3)])
def test_mirror_symmetries_of_planar_blocks(d):
    """Mirror reflections of the plane map a coupling block to a signed permutation of itself:
    B(-dx, dy) = Dx J B(dx, dy) J Dx with Dx = diag((-1)^(m+p)) and B(dx, -dy) = Dy J B J Dy
    with Dy = diag((-1)^p), J the m -> -m permutation. The FFT lattice operator reads one
    block spectrum for the pair (kx, +-ky) on the strength of the second identity."""
    nmax = 4
    lm = vswf.lm_list(nmax)
    L = len(lm)
    jn = [lm.index((l, -m)) for (l, m) in lm]
    J = np.concatenate([jn, np.array(jn) + L])
    m = np.array([mm for (_, mm) in lm] * 2)
    p = np.array([0] * L + [1] * L)
    Dx, Dy = np.diag((-1.0) ** (m + p)), np.diag((-1.0) ** p)
    dx, dy = d
    B = translation.coupling_block(nmax, K0, np.array([dx, dy, 0.0]), np.zeros(3))
    Bx = translation.coupling_block(nmax, K0, np.array([-dx, dy, 0.0]), np.zeros(3))
    By = translation.coupling_block(nmax, K0, np.array([dx, -dy, 0.0]), np.zeros(3))
    scale = np.max(np.abs(B))
    assert np.max(np.abs(Bx - Dx @ B[np.ix_(J, J)] @ Dx)) <= 1e-13 * scale
    assert np.max(np.abs(By - Dy @ B[np.ix_(J, J)] @ Dy)) <= 1e-13 * scale
    # the signs matter: without them neither identity holds (off the symmetry axes)
    if dx != 0 and dy != 0:
        assert np.max(np.abs(By - B[np.ix_(J, J)])) > 1e-3 * scale
