"""Pins of the oracle's sub-region sweep (main text, "Low-overhead multi-GPU simulation
strategy"; Fig. 3; App. II jinc sources): the decomposition is linear in the sources, so

  - one sub-region covering the whole array with no padding is the direct pipeline
    (all sources -> jinc-group coefficients -> dense solve -> field), and
  - padding rings that cover the whole array make every sub-region simulate every sphere
    with only its core's sources; the groups partition the sources, so the summed field
    equals the single all-source solve exactly (up to rounding).

The source grid pitch (0.4) differs from the lambda/2 default, so a sweep that drops the
pitch is caught; planted mistakes (sources taken from the padded set, the pitch dropped,
a sub-region skipped) must fail these pins."""
import math

import numpy as np
import pytest

from oracle import field, geometry, incident, mie, sweep, system
from paper_2107_09879_b300 import workloads as W

K0 = 2 * math.pi
Z0 = -1.0
PITCH = 0.4


def _case(nx, ny, nmax, seed):
    r = W.uniform_radii(nx * ny, 0.08, 0.18, seed)
    g = W.SplitMix64(seed + 1)
    src = np.stack([g.uniforms(nx * ny) - 0.5 + 1j * (g.uniforms(nx * ny) - 0.5),
                    0.3 * (g.uniforms(nx * ny) - 0.5) + 0.2j * g.uniforms(nx * ny)], axis=1)
    pts = np.array([[0.2, 0.3, 2.0], [0.9, 0.1, 3.5], [-0.4, 0.7, 1.5]])
    return r, src, pts


def _direct(nmax, nx, ny, r, src, pts, rule, cutoff=0.0, taper=0.0):
    """All sources at once on the whole array (no decomposition)."""
    pos = W.lattice_positions(nx, ny, PITCH)
    a0 = incident.jinc_group_coeffs(nmax, K0, pos, pos[:, :2], src, Z0, rule, pitch=PITCH)
    T = np.array([mie.tmatrix_diag(nmax, K0, ri, 2.0) for ri in r])
    with system.window(cutoff, taper):
        s = system.solve_dense(nmax, K0, pos, T, a0, cutoff)
    return field.scattered_field(nmax, K0, pos, s, pts)


def _sweep(nmax, nx, ny, r, src, pts, rule, core, buf, cutoff=0.0, taper=0.0):
    return sweep.sweep_fields(nmax, K0, nx, ny, PITCH, 0.0, r, 2.0, src, Z0, core, buf, pts, lambda p, s: rule,
                              cutoff=cutoff, taper=taper)


RULE = incident.jinc_rule(20, 28)


def single_region_error(nmax=2, nx=3, ny=2):
    r, src, pts = _case(nx, ny, nmax, 5)
    E = _sweep(nmax, nx, ny, r, src, pts, RULE, (nx, ny), 0)
    ref = _direct(nmax, nx, ny, r, src, pts, RULE)
    return np.linalg.norm(E - ref) / np.linalg.norm(ref)


def linearity_error(nmax=2, nx=4, ny=3, cutoff=0.0, taper=0.0):
    r, src, pts = _case(nx, ny, nmax, 9)
    E = _sweep(nmax, nx, ny, r, src, pts, RULE, (2, 2), max(nx, ny), cutoff, taper)
    ref = _direct(nmax, nx, ny, r, src, pts, RULE, cutoff, taper)
    return np.linalg.norm(E - ref) / np.linalg.norm(ref)


def test_single_subregion_without_padding_is_the_direct_pipeline():
    assert single_region_error() <= 1e-12


@pytest.mark.parametrize("cutoff,taper", [(0.0, 0.0), (0.9, 0.3)])
def test_covering_rings_sum_to_the_all_source_solve(cutoff, taper):
    assert linearity_error(cutoff=cutoff, taper=taper) <= 1e-11


def test_sources_from_the_padded_set_are_caught(monkeypatch):
    orig = geometry.subregion_sets
    monkeypatch.setattr(geometry, "subregion_sets",
                        lambda *a, **k: [(sim, sim) for _, sim in orig(*a, **k)])
    assert linearity_error() > 1e-3


def test_dropped_pitch_is_caught(monkeypatch):
    orig = incident.jinc_group_coeffs
    monkeypatch.setattr(incident, "jinc_group_coeffs",
                        lambda nmax, k0, pos, xy, A, z0, rule, pitch=None: orig(nmax, k0, pos, xy, A, z0, rule))
    # the direct pipeline keeps the explicit pitch (it calls the original through a closure)
    r, src, pts = _case(3, 2, 2, 5)
    E = _sweep(2, 3, 2, r, src, pts, RULE, (3, 2), 0)
    pos = W.lattice_positions(3, 2, PITCH)
    a0 = orig(2, K0, pos, pos[:, :2], src, Z0, RULE, pitch=PITCH)
    T = np.array([mie.tmatrix_diag(2, K0, ri, 2.0) for ri in r])
    ref = field.scattered_field(2, K0, pos, system.solve_dense(2, K0, pos, T, a0), pts)
    assert np.linalg.norm(E - ref) / np.linalg.norm(ref) > 1e-3


def test_skipped_subregion_is_caught(monkeypatch):
    orig = geometry.subregion_sets
    monkeypatch.setattr(geometry, "subregion_sets", lambda *a, **k: list(orig(*a, **k))[1:])
    assert linearity_error() > 1e-3
