"""GPU parity of the solve, fields and adjoint (through the C-ABI) against the oracle."""
import math

import numpy as np
import pytest

from gpu_common import K0, atoms, ctx, rand_c, rel_l2
from oracle import adjoint, field, incident, mie, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(nx, ny, nmax, seed, angles=(0.0,), lo=0.08, hi=0.24, const_r=None):
    pos = W.lattice_positions(nx, ny)
    r = np.full(nx * ny, const_r) if const_r else W.uniform_radii(nx * ny, lo, hi, seed)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    dirs = np.array([[math.radians(a), 0.0] for a in angles])
    pols = np.array([incident.beta_hat(d[0], 0.0).astype(complex) for d in dirs])
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pols)
    return pos, r, T, a0, dirs, pols


def _oracle_a0(nmax, pos, angles):
    """Incident coefficients computed by the oracle itself (never the GPU's): p-polarised
    plane waves in the xz plane at the given angles."""
    return np.array([incident.planewave_incident(nmax, K0, pos, math.radians(a), 0.0,
                                                 incident.beta_hat(math.radians(a), 0.0)) for a in angles])


def _oracle_solve(nmax, pos, r, a0, cutoff, angles=None):
    """Oracle inputs -> oracle answer: T from the oracle's Mie, a0 from the oracle's plane-wave
    expansion when `angles` is given (a0 is then used only for its shape)."""
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    if angles is not None:
        a0 = _oracle_a0(nmax, pos, angles)
    return np.array([system.solve_dense(nmax, K0, pos, To, a0[q], cutoff) for q in range(a0.shape[0])])


def _opts(**kw):
    from paper_2107_09879_b300 import _lib
    return _lib.make_opts(**kw)


def test_dense_8x8_fp64_vs_oracle_lu():
    """64 identical spheres r = 0.2, nmax = 3, every pair, tol 1e-10: rel. L2 <= 1e-9."""
    pos, r, T, a0, _, _ = _problem(8, 8, 3, 0, const_r=0.2)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 3, T, a0, _opts(tol=1e-10, cutoff=0.0, precision=0))
    assert rc == 0 and info.converged and info.rel_residual[0] <= 1e-10
    ref = _oracle_solve(3, pos, r, a0, 0.0, angles=(0.0,))
    assert rel_l2(s, ref) <= 1e-9


@pytest.mark.parametrize("nmax,nx,ny,cutoff", [(3, 5, 4, 0.0), (4, 9, 7, 1.6), (5, 4, 3, 1.1)])
def test_fp64_and_mixed_vs_oracle(nmax, nx, ny, cutoff):
    pos, r, T, a0, _, _ = _problem(nx, ny, nmax, 10 + nmax, angles=(0.0, 10.0))
    ref = _oracle_solve(nmax, pos, r, a0, cutoff, angles=(0.0, 10.0))
    s64, i64, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, _opts(tol=1e-11, cutoff=cutoff, precision=0))
    assert rc == 0 and rel_l2(s64, ref) <= 1e-9
    smx, imx, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0,
                                       _opts(tol=1e-8, cutoff=cutoff, precision=1, inner_tol=1e-4))
    assert rc == 0 and imx.converged and imx.refinements >= 1
    for q in range(2):
        assert rel_l2(smx[q], ref[q]) <= 1e-6


def test_restart_and_many_rhs():
    pos, r, T, a0, _, _ = _problem(6, 5, 3, 77, angles=(0.0, 3.0, 6.0, 9.0, 12.0))
    ref = _oracle_solve(3, pos, r, a0, 1.2, angles=(0.0, 3.0, 6.0, 9.0, 12.0))
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 3, T, a0, _opts(tol=1e-11, cutoff=1.2, restart=4))
    assert rc == 0 and rel_l2(s, ref) <= 1e-9


def test_iteration_cap_reports_enoconv():
    from paper_2107_09879_b300 import _lib
    pos, r, T, a0, _, _ = _problem(6, 6, 3, 5)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 3, T, a0, _opts(tol=1e-12, cutoff=0.0, max_iter=3))
    assert rc == _lib.ENOCONV and not info.converged and info.iterations == 3
    assert 0 < info.rel_residual[0] < 1


def test_zero_rhs_and_single_scatterer():
    pos = np.zeros((1, 3))
    T = ctx().tmat_build(atoms([0.2]), 1.0, 1.0, 4)
    a0 = np.zeros((1, 1, 48), complex)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 4, T, a0, _opts(tol=1e-10))
    assert rc == 0 and np.all(s == 0)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, 4, np.array([[0.3, 0.2]]),
                                       np.array([incident.beta_hat(0.3, 0.2).astype(complex)]))
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 4, T, a0, _opts(tol=1e-12))
    assert rc == 0 and np.max(np.abs(s[0] - T * a0[0])) <= 1e-14


def test_field_and_farfield_vs_oracle():
    pos, r, T, a0, _, _ = _problem(3, 3, 4, 21)
    s = rand_c((9, 48), 4)
    pts = np.array([[0.3, 0.4, 1.5], [5.0, -2.0, 0.7], [0.5, 0.5, -2.0], [0.25, 0.25, 0.0]])
    E = ctx().tmat_field(pos, 1.0, 1.0, 4, s, pts)
    Eo = field.scattered_field(4, K0, pos, s, pts)
    assert rel_l2(E, Eo) <= 1e-12
    dirs = np.array([[0.0, 0.0], [0.4, 1.0], [math.pi / 2, 2.0], [2.9, -1.0]])
    F = ctx().tmat_farfield(pos, 1.0, 1.0, 4, s, dirs)
    Fo = field.far_field(4, K0, pos, s, [tuple(d) for d in dirs])
    assert rel_l2(F, Fo) <= 1e-12


def test_energy_conservation_on_gpu():
    """Lossless array, every pair coupled: extinction from the GPU coefficients
    equals the scattered power from quadrature of the GPU far field."""
    pos, r, T, a0, _, _ = _problem(4, 3, 3, 8, angles=(10.0,))
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, 3, T, a0, _opts(tol=1e-12, cutoff=0.0))
    pext = -np.real(np.vdot(a0[0], s[0])) * math.pi / K0 ** 2
    xg, wg = np.polynomial.legendre.leggauss(40)
    nph = 80
    dirs = np.array([[math.acos(x), 2 * math.pi * j / nph] for x in xg for j in range(nph)])
    F = ctx().tmat_farfield(pos, 1.0, 1.0, 3, s[0], dirs)
    psca = np.sum(np.repeat(wg, nph) * 2 * math.pi / nph * np.sum(np.abs(F) ** 2, axis=1)) / K0 ** 2
    assert abs(pext - psca) <= 1e-10 * psca


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_gradient_vs_oracle_and_fd(precision):
    nmax, cutoff = 3, 0.8
    pos = W.lattice_positions(3, 2)
    r = W.uniform_radii(6, 0.1, 0.22, 7)
    xf = np.array([0.5, 0.25, 3.0])
    A = np.array([1.0, 0.0, 0.0], dtype=complex)
    Einc = incident.planewave_field(K0, 0.0, 0.0, A, xf[None])[0]
    dirs = np.array([[0.0, 0.0]])
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, A[None])
    tol = 1e-12 if precision == 0 else 1e-9
    opts = _opts(tol=tol, cutoff=cutoff, precision=precision)

    def fwd(rr, keep=False):
        T, dT = ctx().tmat_build(atoms(rr), 1.0, 1.0, nmax, with_dr=True)
        s, info, sol, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=keep)
        assert rc == 0
        return T, dT, s, sol

    T, dT, s, sol = fwd(r, keep=True)
    fom, v = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, Einc)
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    so = system.solve_dense(nmax, K0, pos, To, a0[0], cutoff)
    assert abs(fom - adjoint.fom(nmax, K0, pos, so, xf, Einc)) <= 1e-9 * fom
    vo = adjoint.adjoint_source(nmax, K0, pos, so, xf, Einc)
    assert rel_l2(v, vo) <= (1e-9 if precision == 0 else 1e-6)
    grad, mu, info = ctx().tmat_adjoint(sol, v, dT, want_mu=True)
    dTo = np.array([mie.tmatrix_diag_dr(nmax, K0, x, 2.0) for x in r])
    go, muo = adjoint.radius_gradient(nmax, K0, pos, To, dTo, a0[0], so, vo, cutoff=cutoff)
    assert rel_l2(grad, go) <= (1e-9 if precision == 0 else 1e-6)
    h = 1e-5
    for i in range(6):
        rp, rm = r.copy(), r.copy()
        rp[i] += h
        rm[i] -= h
        fp = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, fwd(rp)[2][0], xf, Einc)[0]
        fm = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, fwd(rm)[2][0], xf, Einc)[0]
        assert abs(grad[i] - (fp - fm) / (2 * h)) <= 1e-4 * np.max(np.abs(grad))


@pytest.mark.parametrize("nmax,height", [(2, 3.0), (4, 20.0), (5, 150.0)])
def test_mixed_precision_near_field(nmax, height):
    """tmat_ctx_set_field_precision(MIXED): fp32 waves with fp64 phases against the oracle's
    field (detectors up to 150 wavelengths away: the phase reduction matters) to 1e-6."""
    from paper_2107_09879_b300 import _lib
    nx, ny = 9, 7
    pos = W.lattice_positions(nx, ny)
    P = 2 * nmax * (nmax + 2)
    s = rand_c((nx * ny, P), 700 + nmax)
    g = W.SplitMix64(710 + nmax)
    pts = np.stack([g.uniforms(16) * 6 - 1, g.uniforms(16) * 5 - 1, height + g.uniforms(16)], axis=1)
    c = _lib.Context(0)
    c.set_field_precision(_lib.PREC_MIXED)
    E32 = c.tmat_field(pos, 1.0, 1.0, nmax, s, pts)
    c.close()
    ref = field.scattered_field(nmax, K0, pos, s, pts)
    assert rel_l2(E32, ref) <= 1e-6
    E64 = ctx().tmat_field(pos, 1.0, 1.0, nmax, s, pts)
    assert rel_l2(E64, ref) <= 1e-8  # the fp64 field (pinned at 1e-12 near the array elsewhere)
    assert rel_l2(E32, E64) <= 1e-6


@pytest.mark.parametrize("space", ["host", "device"])
def test_forward_call_matches_the_separate_calls(space):
    """tmat_forward (build + incident + solve + fields in one call) against the four calls, on
    host arrays and on device tensors, and its field against the oracle's field of the
    oracle's solution."""
    import torch
    from paper_2107_09879_b300 import _lib
    nmax, cut, n = 3, 2.0, 7
    pos = W.lattice_positions(n, 5)
    r = W.uniform_radii(n * 5, 0.08, 0.22, 77)
    b = math.radians(8.0)
    dirs = np.array([[0.0, 0.0], [b, 0.0]])
    pol = np.array([[1, 0, 0], [math.cos(b), 0, -math.sin(b)]], complex)
    pts = np.array([[1.0, 0.7, 2.0], [2.2, 1.1, 4.0], [0.3, 2.0, 9.0]])
    opts = _lib.make_opts(tol=1e-11, restart=80, max_iter=2000, cutoff=cut, taper=cut, precision=_lib.PREC_FP64)
    args = [pos, atoms(r), dirs, pol, pts]
    if space == "device":
        args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args]
    s, E, info, rc = ctx().tmat_forward(args[0], args[1], 1.0, 1.0, nmax, args[2], args[3], opts, args[4])
    assert rc == 0 and info.converged
    if space == "device":
        s, E = s.cpu().numpy(), E.cpu().numpy()
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pol)
    s2, _, _, rc2 = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    assert rc2 == 0 and rel_l2(s, s2) <= 1e-12
    for q in range(2):
        assert rel_l2(E[q], ctx().tmat_field(pos, 1.0, 1.0, nmax, s2[q], pts)) <= 1e-12
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    a0o = incident.planewave_incident(nmax, K0, pos, b, 0.0, incident.beta_hat(b, 0.0))
    with system.window(cut, cut):
        so = system.solve_dense(nmax, K0, pos, To, a0o, cut)
    assert rel_l2(E[1], field.scattered_field(nmax, K0, pos, so, pts)) <= 1e-9


def test_forward_call_argument_errors():
    from paper_2107_09879_b300 import _lib
    pos = W.lattice_positions(2, 2)
    opts = _lib.make_opts(tol=1e-8, precision=_lib.PREC_FP64)
    with pytest.raises(_lib.TMatError):
        ctx().tmat_forward(pos, atoms(np.full(4, 0.1)), 1.0, 1.0, 9, np.zeros((1, 2)), np.ones((1, 3), complex), opts,
                           np.ones((1, 3)))


def test_compressed_basis_solve_matches_the_complex64_basis_and_fp64():
    """Inner solves with a loose tolerance keep their final Krylov vectors in scaled fp16:
    the refined solution meets the same tolerance and agrees with the complex64-basis and
    the fp64 solves within the mixed path's bound."""
    from paper_2107_09879_b300 import _lib
    nmax, cut, n = 4, 4.0, 30
    pos = W.lattice_positions(n, n)
    r = W.uniform_radii(n * n, 0.08, 0.24, 91)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    b = math.radians(10.0)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0], [b, 0.0]]),
                                       np.array([[1, 0, 0], [math.cos(b), 0, -math.sin(b)]], complex))
    kw = dict(restart=200, max_iter=4000, cutoff=cut, taper=cut, path=_lib.PATH_LATTICE, lattice_nx=n, lattice_ny=n,
              lattice_pitch=0.5)
    o_mix = _lib.make_opts(tol=1e-7, precision=_lib.PREC_MIXED, inner_tol=0.2, **kw)
    s16, i16, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, o_mix)
    assert rc == 0 and i16.converged and max(i16.rel_residual[q] for q in range(2)) <= 1e-7
    ctx().set_compressed_basis(False)
    try:
        s32, i32, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, o_mix)
    finally:
        ctx().set_compressed_basis(True)
    assert rc == 0
    s64, _, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0,
                                     _lib.make_opts(tol=1e-10, precision=_lib.PREC_FP64, **kw))
    assert rc == 0
    assert rel_l2(s16, s64) <= 1e-6 and rel_l2(s32, s64) <= 1e-6
    assert i16.iterations <= 1.3 * i32.iterations + 10


def test_sampled_kernel_timing_counts_every_call():
    """tmat_ctx_set_timing(ctx, n): every launch of a timed kind is counted, one Arnoldi
    iteration in n of the complex64 inner solves carries the events (the dot pass is launched
    once per iteration), n = 1 times them all, and a negative n is rejected."""
    from paper_2107_09879_b300 import _lib
    nmax, cut, n = 4, 3.0, 24
    pos = W.lattice_positions(n, n)
    r = W.uniform_radii(n * n, 0.08, 0.24, 93)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), np.array([[1, 0, 0]], complex))
    opts = _lib.make_opts(tol=1e-7, restart=200, max_iter=4000, cutoff=cut, taper=cut, precision=_lib.PREC_MIXED,
                          inner_tol=0.2, path=_lib.PATH_LATTICE, lattice_nx=n, lattice_ny=n, lattice_pitch=0.5)
    c = _lib.Context(0)
    try:
        counts = {}
        for every in (1, 4):
            c.set_timing(every)
            s, info, _, rc = c.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
            assert rc == 0 and info.converged
            timed, ms = c.kernel_time("arnoldi_dots32")
            calls = c.kernel_calls("arnoldi_dots32")
            assert calls >= info.iterations >= 1 and ms > 0
            counts[every] = (timed, calls)
        assert counts[1][0] == counts[1][1]
        timed, calls = counts[4]
        assert abs(timed - math.ceil(calls / 4)) <= 1
        with pytest.raises(_lib.TMatError) as e:
            c.set_timing(-1)
        assert e.value.code == _lib.EINVAL
    finally:
        c.close()


def test_contexts_share_the_kernels_shared_memory_limits():
    """The dynamic shared-memory limit is an attribute of a kernel, not of a context: a context
    that launches the DCGS2 step with a shorter restart length (above 48 KB of shared memory,
    so it sets a limit too) must not lower the limit another context relies on (restart 1000
    needs ~134 KB)."""
    from paper_2107_09879_b300 import _lib
    nmax, cut, n = 3, 2.0, 12
    pos = W.lattice_positions(n, n)
    r = W.uniform_radii(n * n, 0.08, 0.24, 95)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), np.array([[1, 0, 0]], complex))
    kw = dict(tol=1e-7, max_iter=4000, cutoff=cut, taper=cut, precision=_lib.PREC_MIXED, inner_tol=1e-4,
              path=_lib.PATH_LATTICE, lattice_nx=n, lattice_ny=n, lattice_pitch=0.5)
    ca, cb = _lib.Context(0), _lib.Context(0)
    try:
        sa, ia, _, rc = ca.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, _lib.make_opts(restart=1000, **kw))
        assert rc == 0 and ia.converged
        _, ib, _, rc = cb.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, _lib.make_opts(restart=200, **kw))
        assert rc == 0 and ib.converged
        sa2, ia2, _, rc = ca.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, _lib.make_opts(restart=1000, **kw))
        assert rc == 0 and ia2.converged and rel_l2(sa2, sa) <= 1e-12
    finally:
        ca.close()
        cb.close()
