"""tmat_field_noalloc: the field evaluation for callers that cannot allocate
device memory during a call (a host application whose device memory is owned
by another framework's fixed budget, or a loop where the device-wide
synchronisation a cudaMalloc/cudaFree may cause would stall other streams).
It must give the same field as tmat_field. Collected last on purpose."""
import ctypes as ct

import numpy as np
import pytest

from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(nx, ny, nmax, M, seed):
    import torch
    from gpu_common import rand_c
    pos = W.lattice_positions(nx, ny)
    P = 2 * nmax * (nmax + 2)
    s = rand_c((nx * ny, P), seed)
    g = W.SplitMix64(seed + 1)
    pts = np.stack([g.uniforms(M) * 3 - 0.5, g.uniforms(M) * 3 - 0.5, 1.0 + g.uniforms(M)], axis=1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return pos, s, pts, dev(pos), dev(s), dev(pts)


def test_noalloc_field_matches_tmat_field_on_two_calls_in_a_row():
    import torch
    from paper_2107_09879_b300 import _lib
    ctx = _lib.Context(0)
    # two calls with different sizes: the second must not see the first's scratch contents
    for (nx, ny, nmax, M, seed) in [(5, 4, 3, 37, 1), (3, 3, 4, 300, 2)]:
        pos, s, pts, d_pos, d_s, d_pts = _case(nx, ny, nmax, M, seed)
        ref = ctx.tmat_field(pos, 1.0, 1.0, nmax, s, pts)
        E = torch.full((M, 3), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        rc = _lib.lib.tmat_field_noalloc(None, _lib.ptr(d_pos), len(pos), 1.0, 1.0, nmax, _lib.ptr(d_s),
                                         _lib.ptr(d_pts), M, _lib.ptr(E))
        torch.cuda.synchronize()
        assert rc == _lib.OK
        got = E.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_noalloc_field_rejects_oversize_and_host_pointers():
    import torch
    from paper_2107_09879_b300 import _lib
    pos, s, pts, d_pos, d_s, d_pts = _case(2, 2, 2, 4, 3)
    too_many = _lib.NOALLOC_FIELD_SLOTS // 3 + 1
    E = torch.empty((4, 3), dtype=torch.complex128, device="cuda")
    assert _lib.lib.tmat_field_noalloc(None, _lib.ptr(d_pos), 4, 1.0, 1.0, 2, _lib.ptr(d_s), _lib.ptr(d_pts),
                                       too_many, _lib.ptr(E)) == _lib.EINVAL
    assert _lib.lib.tmat_field_noalloc(None, _lib.ptr(pos), 4, 1.0, 1.0, 2, _lib.ptr(d_s), _lib.ptr(d_pts),
                                       4, _lib.ptr(E)) == _lib.EINVAL
