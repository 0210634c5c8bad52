"""Full-size checks on the 200 x 200 lattice (40,000 spheres, nmax = 4, cutoff
8 wavelengths) in the launch configuration the benchmark times: sampled rows of
one operator application against the oracle, computed one by one."""
import math

import numpy as np
import pytest

from gpu_common import K0, atoms, ctx, rand_c
from oracle import mie, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu

SAMPLE_ROWS = [0, 199, 20000 + 100, 39999, 150 * 200 + 3, 7 * 200 + 191, 100 * 200 + 100]


def _rows_csr(pos, rows, cutoff):
    N = len(pos)
    out = []
    for i in rows:
        d = pos - pos[i]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        d2 = d2 + d[:, 2] * d[:, 2]
        js = np.nonzero(d2 <= cutoff * cutoff)[0]
        out.append(js[js != i].astype(np.int32))
    return out


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("taper", [0.0, 8.0])
def test_fullsize_lattice_apply_sampled_rows(op, taper):
    """taper = 8 (window over the whole cutoff) is the benchmark's configuration."""
    w = W.lattice_200x200()
    pos, nmax, cutoff = w["pos"], w["nmax"], w["cutoff"]
    N = len(pos)
    T = ctx().tmat_build(atoms(w["radius"]), 1.0, 1.0, nmax)
    x = rand_c((2, N, 48), 77)
    # fp32: unit roundoff 6e-8 x sqrt(~19k accumulated terms per output) ~ 8e-6
    # precision 2: fp64-class tensor-core apply (exact bf16-slice products); its
    # truncation (~2^-48 of the operand scales) is norm-wise ~1e-12, a single row
    # of small norm (lattice corner) sees ~1e-11
    for precision, bound in ((0, 1e-12), (1, 1e-5), (2, 5e-11)):
        y = ctx().tmat_apply_lattice(op, precision, 200, 200, 0.5, cutoff, K0, nmax, T, x, taper=taper)
        for i, js in zip(SAMPLE_ROWS, _rows_csr(pos, SAMPLE_ROWS, cutoff)):
            rp = np.zeros(N + 1, dtype=np.int64)
            rp[i + 1:] = len(js)
            f = system.apply_K_rows if op == 0 else system.apply_KT_rows
            for q in range(2):
                with system.window(cutoff, taper):
                    ref = f(nmax, K0, pos, T, x[q], (rp, js), [i])[0]
                err = np.linalg.norm(y[q, i] - ref) / np.linalg.norm(ref)
                assert err <= bound, (i, q, precision, err)


def test_fullsize_mixed_solve_matches_fp64_solve():
    """The benchmark's solve (complex64 tensor-core apply, fp64 refinement to 1e-7) against
    the plain complex128 GPU solve of the same 40,000-sphere system, both incidences:
    relative L2 error <= 1e-6. Also the fp64 true residual of both, recomputed here
    through the fp64 operator."""
    from paper_2107_09879_b300 import _lib
    import torch
    w = W.lattice_200x200()
    pos, nmax, cutoff = w["pos"], w["nmax"], w["cutoff"]
    d_pos = torch.from_numpy(pos).cuda()
    T = ctx().tmat_build(torch.from_numpy(atoms(w["radius"])).cuda(), 1.0, 1.0, nmax)
    dirs = np.array([[math.radians(d), 0.0] for d in w["angles_deg"]])
    pols = np.array([[math.cos(d[0]), 0.0, -math.sin(d[0])] for d in dirs], dtype=complex)
    a0 = ctx().tmat_incident_planewave(d_pos, 1.0, 1.0, nmax, torch.from_numpy(dirs).cuda(),
                                       torch.from_numpy(pols).cuda())
    lat = dict(cutoff=cutoff, taper=cutoff, path=_lib.PATH_LATTICE, lattice_nx=200, lattice_ny=200,
               lattice_pitch=0.5, restart=300, max_iter=6000)
    s_mx, i_mx, _, rc1 = ctx().tmat_solve(d_pos, 1.0, 1.0, nmax, T, a0,
                                          _lib.make_opts(tol=1e-7, precision=_lib.PREC_MIXED, inner_tol=1e-4, **lat))
    s_64, i_64, _, rc2 = ctx().tmat_solve(d_pos, 1.0, 1.0, nmax, T, a0,
                                          _lib.make_opts(tol=1e-10, precision=_lib.PREC_FP64, **lat))
    assert rc1 == 0 and rc2 == 0
    for q in range(2):
        err = (torch.linalg.vector_norm(s_mx[q] - s_64[q]) / torch.linalg.vector_norm(s_64[q])).item()
        assert err <= 1e-6, (q, err, i_mx.iterations, i_64.iterations)
    # residuals through the fp64 operator: b - K s with b = T a0
    b = (T.unsqueeze(0) * a0).contiguous()
    for s in (s_mx, s_64):
        Ks = ctx().tmat_apply_lattice(0, 0, 200, 200, 0.5, cutoff, K0, nmax, T, s.contiguous(), taper=cutoff)
        rel = (torch.linalg.vector_norm(b - Ks, dim=(1, 2)) / torch.linalg.vector_norm(b, dim=(1, 2))).max().item()
        assert rel <= 1.1e-7, rel
    print(f"mixed: {i_mx.iterations} iterations, {i_mx.refinements} refinements, {i_mx.seconds:.2f} s; "
          f"fp64: {i_64.iterations} iterations, {i_64.seconds:.2f} s")
