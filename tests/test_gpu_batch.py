"""Batched independent lattice problems (tmat_solve_batch): every problem against its own solve
and the oracle, and the same problem alone and inside a batch."""
import math

import numpy as np
import pytest

from gpu_common import atoms, ctx, rel_l2
from oracle import incident, mie, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _problems(specs, nmax, seed):
    """specs: (nx, ny, wavelength); plane wave at 5 degrees (p-polarised) per problem."""
    out = []
    for q, (nx, ny, w) in enumerate(specs):
        pos = W.lattice_positions(nx, ny)
        r = W.uniform_radii(nx * ny, 0.08, 0.24, seed + q)
        T = ctx().tmat_build(atoms(r), w, 1.0, nmax)
        b = math.radians(5.0)
        a0 = ctx().tmat_incident_planewave(pos, w, 1.0, nmax, np.array([[b, 0.0]]),
                                           np.array([[math.cos(b), 0, -math.sin(b)]], complex))[0]
        out.append(dict(nx=nx, ny=ny, wavelength=w, T=np.ascontiguousarray(T), a0=np.ascontiguousarray(a0), r=r,
                        pos=pos))
    return out


SPECS = [(6, 5, 1.0), (9, 9, 0.93), (4, 7, 1.07), (12, 8, 1.02), (3, 3, 0.9)]


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-9), (1, 1e-8, 1e-6)])
def test_batch_matches_single_solves_and_oracle(precision, tol, bound):
    from paper_2107_09879_b300 import _lib
    nmax, cut = 3, 1.6
    probs = _problems(SPECS, nmax, 300)
    opts = _lib.make_opts(tol=tol, restart=80, max_iter=3000, cutoff=cut, taper=cut, precision=precision)
    outs, infos, rc = ctx().tmat_solve_batch(probs, 1.0, nmax, 0.5, opts)
    assert rc == 0 and all(i.converged for i in infos)
    for p, s in zip(probs, outs):
        o1 = _lib.make_opts(tol=tol, restart=80, max_iter=3000, cutoff=cut, taper=cut, precision=precision,
                            path=_lib.PATH_LATTICE, lattice_nx=p["nx"], lattice_ny=p["ny"], lattice_pitch=0.5)
        s1, _, _, rc1 = ctx().tmat_solve(p["pos"], p["wavelength"], 1.0, nmax, p["T"], p["a0"][None], o1)
        assert rc1 == 0 and rel_l2(s, s1[0]) <= bound
    # the oracle on two of them (its own T and incident coefficients at that wavelength)
    for q in (0, 2):
        p = probs[q]
        k = 2 * math.pi / p["wavelength"]
        To = np.array([mie.tmatrix_diag(nmax, k, x, 2.0) for x in p["r"]])
        b = math.radians(5.0)
        a0o = incident.planewave_incident(nmax, k, p["pos"], b, 0.0, incident.beta_hat(b, 0.0))
        with system.window(cut, cut):
            ref = system.solve_dense(nmax, k, p["pos"], To, a0o, cut)
        assert rel_l2(outs[q], ref) <= bound


@pytest.mark.parametrize("precision,bound", [(0, 1e-12), (1, 1e-6)])
def test_problem_alone_and_in_a_batch(precision, bound):
    """On a fixed canvas a problem's result does not depend on the other problems of the batch:
    to rounding in fp64; within the mixed path's solution tolerance in mixed precision, where
    the refinement steps (how far each complex64 inner solve runs, which residuals are checked
    in complex64) are decided for the batch as a whole."""
    from paper_2107_09879_b300 import _lib
    nmax = 3
    probs = _problems(SPECS, nmax, 400)
    opts = _lib.make_opts(tol=1e-10 if precision == 0 else 1e-7, restart=60, max_iter=3000, cutoff=2.0, taper=2.0,
                          precision=precision)
    outs, infos, rc = ctx().tmat_solve_batch(probs, 1.0, nmax, 0.5, opts, canvas=(12, 9))
    assert rc == 0
    for q in (1, 4):
        alone, _, rc1 = ctx().tmat_solve_batch([probs[q]], 1.0, nmax, 0.5, opts, canvas=(12, 9))
        assert rc1 == 0 and rel_l2(outs[q], alone[0]) <= bound


def test_batch_argument_errors():
    from paper_2107_09879_b300 import _lib
    probs = _problems(SPECS[:2], 2, 500)
    opts = _lib.make_opts(tol=1e-8, cutoff=1.0, precision=2)
    with pytest.raises(_lib.TMatError):
        ctx().tmat_solve_batch(probs, 1.0, 2, 0.5, opts)
    opts.precision = 1
    with pytest.raises(_lib.TMatError):
        ctx().tmat_solve_batch(probs, 1.0, 2, 0.5, opts, canvas=(8, 8))  # the 9 x 9 problem exceeds it
