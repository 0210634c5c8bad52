"""GPU parity of the jinc-group incident coefficients (App. II) against the oracle."""
import math

import numpy as np
import pytest

from gpu_common import K0, ctx, rand_c, rel_l2
from oracle import incident
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu
Z0 = -1.0


def _case(nsx, nsy, nx, ny, R, seed):
    pos = W.lattice_positions(nx, ny)
    src = W.lattice_positions(nsx, nsy)[:, :2] + np.array([0.25, 0.0])
    A = rand_c((R, nsx * nsy, 2), seed)
    return pos, src, A


def _extent(pos, src):
    ex = max(pos[:, 0].max() - src[:, 0].min(), src[:, 0].max() - pos[:, 0].min())
    ey = max(pos[:, 1].max() - src[:, 1].min(), src[:, 1].max() - pos[:, 1].min())
    ez = max(abs(pos[:, 2].max() - Z0), abs(pos[:, 2].min() - Z0))
    return math.sqrt(ex * ex + ey * ey + ez * ez)


@pytest.mark.parametrize("nmax,R", [(3, 2), (4, 1), (2, 4)])
def test_jinc_group_vs_oracle(nmax, R):
    pos, src, A = _case(4, 3, 5, 4, R, 10 + nmax)
    nb, na = incident.jinc_rule_size(K0, _extent(pos, src))
    rule = incident.jinc_rule(nb, na)
    ref = np.array([incident.jinc_group_coeffs(nmax, K0, pos, src, A[r], Z0, rule) for r in range(R)])
    a64 = ctx().tmat_incident_jinc(pos, 1.0, 1.0, nmax, src, A, Z0, nb, na, precision=0)
    a32 = ctx().tmat_incident_jinc(pos, 1.0, 1.0, nmax, src, A, Z0, nb, na, precision=1)
    auto = ctx().tmat_incident_jinc(pos, 1.0, 1.0, nmax, src, A, Z0, 0, 0, precision=0)  # same sizing rule
    assert rel_l2(a64, ref) <= 1e-12
    assert rel_l2(a32, ref) <= 1e-6
    assert rel_l2(auto, ref) <= 1e-12


def test_jinc_coarser_grid_weight():
    pos, src, A = _case(3, 2, 3, 2, 1, 7)
    k0 = 2 * math.pi / 0.9
    nb, na = incident.jinc_rule_size(k0, _extent(pos, src))
    ref = incident.jinc_group_coeffs(3, k0, pos, src, A[0], Z0, incident.jinc_rule(nb, na), pitch=0.5)
    a = ctx().tmat_incident_jinc(pos, 0.9, 1.0, 3, src, A, Z0, nb, na, precision=0, src_pitch=0.5)
    assert rel_l2(a[0], ref) <= 1e-12


def test_jinc_single_source_and_empty_group():
    pos, src, A = _case(1, 1, 3, 3, 1, 3)
    a = ctx().tmat_incident_jinc(pos, 1.0, 1.0, 3, src, A, Z0)
    nb, na = incident.jinc_rule_size(K0, _extent(pos, src))
    ref = incident.jinc_group_coeffs(3, K0, pos, src, A[0], Z0, incident.jinc_rule(nb, na))
    assert rel_l2(a[0], ref) <= 1e-12
    z = ctx().tmat_incident_jinc(pos, 1.0, 1.0, 3, np.zeros((0, 2)), np.zeros((1, 0, 2), complex), Z0, 10, 12)
    assert np.all(z == 0)


@pytest.mark.parametrize("offset", [0.0, 480.0])
def test_jinc_complex64_chunked_group(offset):
    """The complex64 path on a group that needs several node chunks of the phase matrix and a
    GEMM split over nodes (40 x 40 spheres, 30 x 30 sources, 26,312 rule nodes, 2 RHS):
    against the fp64 path at every sphere (complex64 tolerance) and the fp64 path against
    the oracle at sampled spheres. The offset (480 wavelengths) puts the phases k.x in the
    thousands of radians, where the double-float argument and its reduction modulo 2 pi
    must still hold the complex64 accuracy."""
    side, core = 40, 30
    pos = W.lattice_positions(side, side, origin=(offset, 0.7 * offset))
    src = np.ascontiguousarray(W.lattice_positions(core, core, origin=(offset + 2.5, 0.7 * offset + 2.5))[:, :2])
    A = rand_c((2, core * core, 2), 77)
    a32 = ctx().tmat_incident_jinc(pos, 1.0, 1.0, 3, src, A, Z0, precision=1, src_pitch=0.5)
    a64 = ctx().tmat_incident_jinc(pos, 1.0, 1.0, 3, src, A, Z0, precision=0, src_pitch=0.5)
    assert rel_l2(a32, a64) <= 1e-6
    idx = [0, 777, side * side - 1]
    nb, na = incident.jinc_rule_size(K0, _extent(pos, src))
    assert nb * na > 3 * 8192  # several node chunks of the complex64 path
    ref = incident.jinc_group_coeffs(3, K0, pos[idx], src, A[1], Z0, incident.jinc_rule(nb, na), pitch=0.5)
    assert rel_l2(a64[1][idx], ref) <= 1e-10
