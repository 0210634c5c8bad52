"""GPU parity of the lattice (one block per lattice offset) path against the oracle."""
import math

import numpy as np
import pytest

from gpu_common import C64_APPLY_TOL, K0, atoms, ctx, rand_c, rel_l2
from oracle import incident, geometry, mie, system
from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(3, 13, 11, 1.6, 1), (4, 9, 7, 1.2, 2), (2, 6, 5, 0.0, 3),
                                                 (5, 5, 4, 1.1, 5), (6, 4, 3, 0.8, 2), (1, 17, 9, 2.0, 1)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_lattice_apply_vs_oracle(nmax, nx, ny, cutoff, R, op):
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 40 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 50 + nmax)
    nbr = geometry.neighbours(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(R)])
    y64 = ctx().tmat_apply_lattice(op, 0, nx, ny, 0.5, cutoff, K0, nmax, T, x)
    y32 = ctx().tmat_apply_lattice(op, 1, nx, ny, 0.5, cutoff, K0, nmax, T, x)
    assert rel_l2(y64, ref) <= 1e-12
    assert rel_l2(y32, ref) <= C64_APPLY_TOL


def test_lattice_matches_neighbour_path_bitwise_structure():
    """Same interaction set as the neighbour list on a lattice: both paths agree to rounding."""
    nx, ny, nmax, cutoff = 20, 17, 4, 3.0
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 3)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    x = rand_c((2, nx * ny, 48), 9)
    rp, col = ctx().tmat_neighbors(pos, cutoff)
    for op in range(3):
        a = ctx().tmat_apply(op, 0, pos, K0, nmax, T, rp, col, x)
        b = ctx().tmat_apply_lattice(op, 0, nx, ny, 0.5, cutoff, K0, nmax, T, x)
        assert rel_l2(b, a) <= 1e-13


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-9), (1, 1e-8, 1e-6)])
def test_lattice_solve_vs_oracle(precision, tol, bound):
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax, cutoff = 8, 7, 4, 1.6
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 12)
    T = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax)
    dirs = np.array([[0.0, 0.0], [math.radians(10), 0.0]])
    pols = np.array([[1, 0, 0], [math.cos(math.radians(10)), 0, -math.sin(math.radians(10))]], dtype=complex)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pols)
    opts = _lib.make_opts(tol=tol, cutoff=cutoff, precision=precision, path=2, lattice_nx=nx, lattice_ny=ny,
                          lattice_pitch=0.5)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    assert rc == 0 and info.converged
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    for q in range(2):
        a0o = incident.planewave_incident(nmax, K0, pos, dirs[q, 0], dirs[q, 1], pols[q])  # the oracle's own
        ref = system.solve_dense(nmax, K0, pos, To, a0o, cutoff)
        assert rel_l2(s[q], ref) <= bound


def test_lattice_adjoint_matches_neighbour_adjoint():
    from paper_2107_09879_b300 import _lib
    nx, ny, nmax, cutoff = 7, 6, 3, 1.3
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.1, 0.22, 17)
    T, dT = ctx().tmat_build(atoms(r), 1.0, 1.0, nmax, with_dr=True)
    A = np.array([[1, 0, 0]], dtype=complex)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), A)
    xf = np.array([1.5, 1.25, 4.0])
    grads = []
    for path in (1, 2):
        opts = _lib.make_opts(tol=1e-12, cutoff=cutoff, precision=0, path=path, lattice_nx=nx, lattice_ny=ny,
                              lattice_pitch=0.5)
        s, info, sol, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
        fom, v = ctx().tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, np.exp(1j * 2 * np.pi * 4.0) * A[0])
        g, mu, info = ctx().tmat_adjoint(sol, v, dT)
        grads.append(g)
    assert rel_l2(grads[1], grads[0]) <= 1e-10


def test_lattice_rejects_non_lattice_positions():
    from paper_2107_09879_b300 import _lib
    pos = W.lattice_positions(4, 4).copy()
    pos[5, 0] += 0.01
    T = ctx().tmat_build(atoms(np.full(16, 0.1)), 1.0, 1.0, 2)
    a0 = np.ones((1, 16, 16), complex)
    opts = _lib.make_opts(tol=1e-8, path=2, lattice_nx=4, lattice_ny=4, lattice_pitch=0.5)
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve(pos, 1.0, 1.0, 2, T, a0, opts)
    assert e.value.code == _lib.EINVAL


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(4, 23, 9, 2.0, 2), (3, 17, 13, 1.6, 1), (2, 9, 7, 1.2, 3),
                                                 (1, 11, 5, 1.0, 2), (4, 7, 6, 0.0, 5)])
@pytest.mark.parametrize("op", [0, 1, 2])
@pytest.mark.parametrize("variant,kind", [(1, "lattice_apply_tcv"), (2, "lattice_apply_tc")])
def test_tensor_core_apply_matches_cuda_cores_and_oracle(nmax, nx, ny, cutoff, R, op, variant, kind):
    """Both tcgen05 3xTF32 kernels (window view, gather) against the CUDA-core fp32 kernel
    and the oracle."""
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 60 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 70 + nmax)
    c = ctx()
    c.set_lattice_fft(False)
    try:
        c.set_tensor_cores(variant)
        c.set_timing(True)
        n0, _ = c.kernel_time(kind)
        ytc = c.tmat_apply_lattice(op, 1, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
        n_tc, _ = c.kernel_time(kind)
        n_tc -= n0
        c.set_tensor_cores(False)
        ycc = c.tmat_apply_lattice(op, 1, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    finally:
        c.set_tensor_cores(True)
        c.set_timing(False)
        c.set_lattice_fft(True)
    assert n_tc >= 1  # the tensor-core kernel really ran
    nbr = geometry.neighbours(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    with system.window(cutoff, cutoff):
        ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(R)])
    assert rel_l2(ytc, ref) <= C64_APPLY_TOL
    assert rel_l2(ytc, ycc) <= C64_APPLY_TOL


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(4, 23, 9, 2.0, 2), (3, 17, 13, 1.6, 1), (2, 9, 7, 1.2, 3),
                                                 (1, 11, 5, 1.0, 2), (4, 7, 6, 0.0, 5)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_fp64_tc_apply_matches_fp64(nmax, nx, ny, cutoff, R, op):
    """TMAT_PREC_FP64_TC (exact bf16-slice products on the tensor cores) against the fp64
    CUDA-core apply and the oracle; sources spanning six decades of magnitude."""
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 80 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 90 + nmax)
    x *= 10.0 ** (-6.0 * W.uniform_radii(nx * ny, 0.0, 1.0, 91))[None, :, None]
    c = ctx()
    c.set_timing(True)
    n0, _ = c.kernel_time("lattice_apply_oz")
    ytc = c.tmat_apply_lattice(op, 2, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    n1, _ = c.kernel_time("lattice_apply_oz")
    c.set_timing(False)
    assert n1 - n0 == 1
    y64 = c.tmat_apply_lattice(op, 0, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    nbr = geometry.neighbours(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    with system.window(cutoff, cutoff):
        ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(R)])
    assert rel_l2(y64, ref) <= 1e-12
    assert rel_l2(ytc, y64) <= 1e-11
    assert rel_l2(ytc, ref) <= 1e-11


def test_fp64_tc_solve_vs_oracle_and_neighbour_path_refused():
    from paper_2107_09879_b300 import _lib
    nmax, nx, ny, cutoff = 3, 9, 7, 1.5
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 95)
    at = atoms(r)
    T = ctx().tmat_build(at, 1.0, 1.0, nmax)
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0], [0.3, 0.0]]),
                                       np.array([[1, 0, 0], [math.cos(0.3), 0, -math.sin(0.3)]], dtype=complex))
    opts = _lib.make_opts(tol=1e-12, restart=80, max_iter=3000, cutoff=cutoff, taper=cutoff, precision=2, path=2,
                          lattice_nx=nx, lattice_ny=ny, lattice_pitch=0.5)
    s, info, _, rc = ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    assert rc == 0 and info.converged
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    a0o = [incident.planewave_incident(nmax, K0, pos, b, 0.0, np.array([math.cos(b), 0, -math.sin(b)], complex))
           for b in (0.0, 0.3)]  # the oracle's own incident coefficients
    with system.window(cutoff, cutoff):
        ref = np.array([system.solve_dense(nmax, K0, pos, To, a0o[q], cutoff) for q in range(2)])
    assert rel_l2(s, ref) <= 1e-9
    opts.path = 1
    with pytest.raises(_lib.TMatError) as e:
        ctx().tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    assert e.value.code == _lib.ENOTSUP


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(4, 23, 9, 2.0, 2), (3, 17, 13, 1.6, 1), (2, 9, 7, 0.0, 3),
                                                 (5, 11, 6, 1.4, 2), (6, 5, 4, 0.9, 1), (1, 31, 1, 3.0, 2),
                                                 (2, 1, 12, 2.0, 1)])
@pytest.mark.parametrize("op", [0, 1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_fft_apply_matches_direct_and_oracle(nmax, nx, ny, cutoff, R, op, precision):
    """The FFT-convolution lattice apply (default) against the direct block-Toeplitz kernels
    and the oracle: fp64 to 1e-12, complex64 to the complex64 tolerance; ragged and
    one-row lattices, every pair (cutoff 0), nmax 1..6, both window readings."""
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 120 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 130 + nmax)
    c = ctx()
    kind = "lattice_apply_fft64" if precision == 0 else "lattice_apply_fft32"
    c.set_timing(True)
    n0, _ = c.kernel_time(kind)
    yf = c.tmat_apply_lattice(op, precision, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    n1, _ = c.kernel_time(kind)
    c.set_timing(False)
    assert n1 - n0 == 1  # the FFT path ran
    c.set_lattice_fft(False)
    try:
        yd = c.tmat_apply_lattice(op, precision, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    finally:
        c.set_lattice_fft(True)
    nbr = geometry.neighbours(pos, cutoff)
    f = [system.apply_K, system.apply_KT, lambda nm, k, p, t, v, nb: system.apply_A(nm, k, p, v, nb)][op]
    with system.window(cutoff, cutoff):
        ref = np.array([f(nmax, K0, pos, T, x[q], nbr) for q in range(R)])
    bound = 1e-12 if precision == 0 else C64_APPLY_TOL
    assert rel_l2(yf, ref) <= bound
    assert rel_l2(yf, yd) <= bound


@pytest.mark.parametrize("nmax,nx,ny,cutoff,R", [(4, 37, 29, 3.0, 5), (3, 40, 3, 0.0, 2), (5, 13, 21, 2.2, 3),
                                                 (6, 7, 9, 1.1, 1), (1, 6, 50, 4.0, 4)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_fft_quad_product_matches_mirror_pair_product(nmax, nx, ny, cutoff, R, op):
    """The complex64 quad-mirror block product (one symmetric matrix per frequency quadruple,
    default) against the mirror-pair product (tmat_ctx_set_lattice_fft(ctx, 2)) and the
    oracle: odd RHS counts (a half-empty last RHS pass), partial ky tiles, every pair, one
    grid dimension much longer than the other, nmax 1..6."""
    from paper_2107_09879_b300 import _lib
    pos = W.lattice_positions(nx, ny)
    r = W.uniform_radii(nx * ny, 0.08, 0.24, 140 + nmax)
    T = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    x = rand_c((R, nx * ny, T.shape[1]), 150 + nmax)
    c = _lib.Context(0)
    yq = c.tmat_apply_lattice(op, 1, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    c.set_lattice_fft(2)
    yp = c.tmat_apply_lattice(op, 1, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    c.close()
    y64 = ctx().tmat_apply_lattice(op, 0, nx, ny, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    assert rel_l2(yq, y64) <= C64_APPLY_TOL
    assert rel_l2(yp, y64) <= C64_APPLY_TOL
    assert rel_l2(yq, yp) <= 2 * C64_APPLY_TOL


@pytest.mark.parametrize("nmax,n,cutoff,R", [(4, 130, 3.0, 2), (3, 125, 2.0, 3), (5, 129, 1.5, 1)])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_fft_256_grid_passes_match_fp64_and_direct(nmax, n, cutoff, R, op):
    """Lattices whose FFT grid is 256 x 256 take the four-step, transpose-free passes (x read
    and y written in place; P = 30, 48, 70: full and partial component blocks; odd R), in
    complex64 and, for the complex128 operator, in double-float: the complex128 FFT apply
    against the direct fp64 kernel to 1e-12, the complex64 one and the direct complex64
    kernel against it to the complex64 tolerance."""
    from paper_2107_09879_b300 import _lib
    r = W.uniform_radii(n * n, 0.08, 0.24, 160 + nmax)
    T = np.ascontiguousarray(np.array([mie.tmatrix_diag(nmax, K0, v, 2.0) for v in r]))
    x = rand_c((R, n * n, T.shape[1]), 170 + nmax)
    c = _lib.Context(0)
    y32 = c.tmat_apply_lattice(op, 1, n, n, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    y64 = c.tmat_apply_lattice(op, 0, n, n, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    c.set_lattice_fft(False)
    yd = c.tmat_apply_lattice(op, 1, n, n, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    yd64 = c.tmat_apply_lattice(op, 0, n, n, 0.5, cutoff, K0, nmax, T, x, taper=cutoff)
    c.close()
    assert rel_l2(y64, yd64) <= 1e-12
    assert rel_l2(y32, y64) <= C64_APPLY_TOL
    assert rel_l2(yd, y64) <= C64_APPLY_TOL
