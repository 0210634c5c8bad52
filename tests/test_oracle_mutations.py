"""Planted mistakes: each test patches one plausible mistake into the ORACLE
(on the CPU) and checks that at least one of the pins catches it. This shows
the pins are strong enough to certify the oracle."""
import math

import numpy as np
import pytest

from oracle import incident, mie, system, translation
from oracle_pins import (addition_theorem_error, energy_balance_error, mie_dipole_pattern_ratio,
                         planewave_error)

ORIG_A5B5 = translation.a5b5


@pytest.fixture(autouse=True)
def _clear_tables():
    translation.coupling_tables.cache_clear()
    yield
    translation.coupling_tables.cache_clear()


def _patch_a5b5(monkeypatch, fn):
    monkeypatch.setattr(translation, "a5b5", fn)
    translation.coupling_tables.cache_clear()


@pytest.mark.parametrize("mutation", ["beta_sign", "drop_minus1_power", "ipow_l_minus_lp", "beta_3j_q", "denominator"])
def test_translation_mistakes_are_caught(monkeypatch, mutation):
    def bad(l, m, lp, mp, q):
        a, b = ORIG_A5B5(l, m, lp, mp, q)
        if mutation == "beta_sign":
            return a, -b
        if mutation == "drop_minus1_power":
            s = (-1) ** ((m - mp) % 2)
            return a * s, b * s
        if mutation == "ipow_l_minus_lp":
            s = (-1) ** ((l - lp) % 2)
            return a * s, b * s
        if mutation == "beta_3j_q":  # the literal printed (l l' q; 0 0 0) in beta
            return a, 0.0 * b
        if mutation == "denominator":  # literal 2 l (l+1)(l'+1)
            return a * math.sqrt(lp), b * math.sqrt(lp)
        raise AssertionError

    _patch_a5b5(monkeypatch, bad)
    assert addition_theorem_error(3, (0.5, 0.2, 0.3), npts=3) > 1e-3


def test_untransposed_coupling_block_is_caught(monkeypatch):
    monkeypatch.setattr(system, "_block", lambda nmax, k, xt, xs: translation.xi_matrix(nmax, nmax, k, np.asarray(xt) - np.asarray(xs)))
    assert energy_balance_error(2, 2, 2, 10.0) > 1e-4


def test_reversed_displacement_in_system_is_caught(monkeypatch):
    monkeypatch.setattr(system, "_block", lambda nmax, k, xt, xs: translation.xi_matrix(nmax, nmax, k, np.asarray(xs) - np.asarray(xt)).T)
    assert energy_balance_error(2, 2, 2, 10.0) > 1e-4


def test_swapped_mie_polarisations_are_caught(monkeypatch):
    orig = mie.mie_ab
    monkeypatch.setattr(mie, "mie_ab", lambda nmax, k, r, m: orig(nmax, k, r, m)[::-1])
    assert mie_dipole_pattern_ratio() > 1.0


def test_planewave_i_power_m_is_caught(monkeypatch):
    """The printed first equality uses 4 i^m; the explicit i^l form is the right one."""
    orig = incident.planewave_coeffs

    def bad(nmax, beta, alpha, A):
        a = orig(nmax, beta, alpha, A)
        L = nmax * (nmax + 2)
        for l in range(1, nmax + 1):
            for m in range(-l, l + 1):
                n = l * (l + 1) + m - 1
                f = (1j ** (m % 4)) / (1j ** (l % 4))
                a[n] *= f
                a[L + n] *= f
        return a

    monkeypatch.setattr(incident, "planewave_coeffs", bad)
    assert planewave_error(12, 0.4, 1.1, npts=2) > 1e-3


def test_mie_radius_derivative_dropped_factor_is_caught(monkeypatch):
    orig = mie.mie_ab_dr
    monkeypatch.setattr(mie, "mie_ab_dr", lambda nmax, k, r, m: tuple(v / m for v in orig(nmax, k, r, m)))
    r, h = 0.16, 1e-4
    d = mie.tmatrix_diag_dr(3, 2 * math.pi, r, 2.0)
    f = lambda rr: mie.tmatrix_diag(3, 2 * math.pi, rr, 2.0)
    fd = (f(r + h) - f(r - h)) / (2 * h)
    assert np.max(np.abs(d - fd)) > 1e-3 * np.max(np.abs(fd))
