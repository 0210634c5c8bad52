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
    for precision, bound in ((0, 1e-12), (1, 1e-5)):
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
