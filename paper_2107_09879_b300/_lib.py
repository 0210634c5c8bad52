"""Thin ctypes binding of libtmat.so (include/tmat.h). Argument marshalling only:
every computation runs in the library's CUDA kernels.

Arrays may be numpy arrays (host memory; the library stages them) or torch
tensors on the GPU (used in place, on the context's stream). Complex arrays are
complex128 (layout-compatible with tmat_c128). There is no CPU fallback: if the
library is missing, importing this module raises.
"""
import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TMAT_LIB") or os.path.join(_HERE, "libtmat.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2107_09879_b300.build`")
lib = ct.CDLL(LIB_PATH)

OK, EINVAL, EOVERLAP, ENOMEM, ENOCONV, EBREAKDOWN, ECUDA, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_MIXED, PREC_FP64_TC = 0, 1, 2
PATH_AUTO, PATH_NEIGHBOUR, PATH_LATTICE = 0, 1, 2
OP_FORWARD, OP_ADJOINT, OP_COUPLE = 0, 1, 2
MAX_RHS = 16


class SolveOpts(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("restart", ct.c_int), ("max_iter", ct.c_int), ("cutoff", ct.c_double),
                ("precision", ct.c_int), ("inner_tol", ct.c_double), ("path", ct.c_int),
                ("lattice_nx", ct.c_int), ("lattice_ny", ct.c_int), ("lattice_pitch", ct.c_double),
                ("taper", ct.c_double), ("enclosing_radii", ct.c_void_p)]


class SolveInfo(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("refinements", ct.c_int), ("converged", ct.c_int), ("n_rhs", ct.c_int),
                ("rel_residual", ct.c_double * MAX_RHS), ("seconds", ct.c_double)]

    def as_dict(self):
        return dict(iterations=self.iterations, refinements=self.refinements, converged=bool(self.converged),
                    rel_residual=[self.rel_residual[i] for i in range(self.n_rhs)], seconds=self.seconds)


class SweepOpts(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("pitch", ct.c_double), ("x0", ct.c_double), ("y0", ct.c_double),
                ("z", ct.c_double), ("core_x", ct.c_int), ("core_y", ct.c_int), ("buffer", ct.c_int),
                ("z0", ct.c_double), ("n_beta", ct.c_int), ("n_alpha", ct.c_int), ("first", ct.c_int),
                ("count", ct.c_int)]


class SweepInfo(ct.Structure):
    _fields_ = [("subregions", ct.c_int), ("total_subregions", ct.c_int), ("unconverged", ct.c_int),
                ("iterations", ct.c_int), ("scatterer_solves", ct.c_int64), ("worst_rel_residual", ct.c_double),
                ("seconds", ct.c_double)]


class BatchProblem(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("wavelength", ct.c_double), ("T_diag", ct.c_void_p),
                ("a0", ct.c_void_p), ("s_out", ct.c_void_p)]


class Atom(ct.Structure):
    _fields_ = [("radius", ct.c_double), ("n_re", ct.c_double), ("n_im", ct.c_double)]


_vp, _i64, _i32, _d, _int = ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_double, ct.c_int
_SIGS = {
    "tmat_ctx_create": [_int, _vp, ct.POINTER(_vp)],
    "tmat_ctx_set_stream": [_vp, _vp],
    "tmat_ctx_destroy": [_vp],
    "tmat_last_error": [_vp],
    "tmat_ctx_launch_count": [_vp],
    "tmat_ctx_set_timing": [_vp, _int],
    "tmat_ctx_set_tensor_cores": [_vp, _int],
    "tmat_ctx_set_lattice_fft": [_vp, _int],
    "tmat_ctx_kernel_time": [_vp, ct.c_char_p, ct.POINTER(_i64), ct.POINTER(_d)],
    "tmat_ctx_kernel_bytes": [_vp, ct.c_char_p, ct.POINTER(_d)],
    "tmat_ctx_kernel_calls": [_vp, ct.c_char_p, ct.POINTER(_i64)],
    "tmat_neighbors": [_vp, _vp, _i64, _d, _vp, _vp, ct.POINTER(_i64)],
    "tmat_subregions": [_vp, _i64, _i64, _i64, _i64, _i64, _vp, _vp, _vp, _vp, ct.POINTER(_i64), ct.POINTER(_i64)],
    "tmat_build": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp],
    "tmat_incident_planewave": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _int, _vp],
    "tmat_incident_jinc": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _i64, _int, _d, _d, _int, _int, _int, _vp],
    "tmat_translation": [_vp, _int, _d, _vp, _i64, _vp],
    "tmat_apply": [_vp, _int, _int, _vp, _i64, _d, _int, _vp, _vp, _vp, _d, _d, _vp, _int, _vp],
    "tmat_apply_lattice": [_vp, _int, _int, _int, _int, _d, _d, _d, _d, _int, _vp, _vp, _int, _vp],
    "tmat_solve": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _int, ct.POINTER(SolveOpts), _vp, ct.POINTER(_vp),
                   ct.POINTER(SolveInfo)],
    "tmat_solution_free": [_vp],
    "tmat_sweep": [_vp, ct.POINTER(SweepOpts), _vp, _d, _d, _int, _vp, _int, ct.POINTER(SolveOpts), _vp, _i64, _vp,
                   ct.POINTER(SweepInfo)],
    "tmat_field": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _i64, _vp],
    "tmat_forward": [_vp, _vp, _i64, _vp, _d, _d, _int, _vp, _vp, _int, ct.POINTER(SolveOpts), _vp, _i64, _vp, _vp,
                     ct.POINTER(SolveInfo)],
    "tmat_farfield": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _i64, _vp],
    "tmat_point_fom": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _vp, ct.POINTER(_d), _vp],
    "tmat_field_noalloc": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _i64, _vp],
    "tmat_adjoint": [_vp, _vp, _vp, _vp, _vp, _vp, ct.POINTER(SolveInfo)],
    "tmat_position_gradient": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "tmat_measure_fma_peak": [_int, _int, ct.POINTER(_d)],
    "tmat_check_overlap": [_vp, _vp, _i64, _vp, _vp],
    "tmat_solve_batch": [_vp, _vp, _int, _d, _int, _d, _int, _int, ct.POINTER(SolveOpts), _vp],
    "tmat_ctx_memory": [_vp, ct.POINTER(_i64)],
    "tmat_ctx_set_field_precision": [_vp, _int],
    "tmat_ctx_set_compressed_basis": [_vp, _int],
    "tmat_build_cylinder": [_vp, _vp, _i64, _d, _d, _int, _int, _vp, _vp],
    "tmat_solve_tblocks": [_vp, _vp, _i64, _d, _d, _int, _vp, _vp, _i64, _vp, _int, ct.POINTER(SolveOpts), _vp,
                           ct.POINTER(_vp), ct.POINTER(SolveInfo)],
    "tmat_adjoint_tblocks": [_vp, _vp, _vp, _vp, _vp, _vp, ct.POINTER(SolveInfo)],
}
EXPORTED = []
for _name, _args in _SIGS.items():
    if hasattr(lib, _name):
        f = getattr(lib, _name)
        f.argtypes = _args
        f.restype = ct.c_int
        EXPORTED.append(_name)
lib.tmat_last_error.restype = ct.c_char_p
NOALLOC_FIELD_SLOTS = 65536
lib.tmat_ctx_launch_count.restype = ct.c_int64


class TMatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tmat error {code}: {msg}")
        self.code = code


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def ptr(a):
    """Raw pointer of a numpy array (C-contiguous) or torch tensor (contiguous)."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous(), "tensor must be contiguous"
        return ct.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return ct.c_void_p(a.ctypes.data)


def empty_like_space(ref, shape, dtype):
    """An output array in the same memory space as `ref` (numpy host or torch device)."""
    if _is_torch(ref):
        import torch
        tdt = {np.complex128: torch.complex128, np.float64: torch.float64, np.int64: torch.int64,
               np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


class Context:
    """A library context on one device and stream (default: the current torch
    stream when torch is present, else the legacy default stream)."""

    def __init__(self, device=0, stream=None):
        h = ct.c_void_p()
        self._check(lib.tmat_ctx_create(device, stream, ct.byref(h)), None)
        self.h = h

    def _check(self, rc, h=-1):
        if rc != OK:
            msg = lib.tmat_last_error(self.h if h == -1 else h)
            raise TMatError(rc, msg.decode() if msg else "")

    def check(self, rc):
        self._check(rc)

    def set_stream(self, stream):
        self.check(lib.tmat_ctx_set_stream(self.h, stream))

    def set_compressed_basis(self, on):
        """Loose inner solves (tolerance >= 1e-2) keep their final Krylov vectors in scaled fp16."""
        self.check(lib.tmat_ctx_set_compressed_basis(self.h, 1 if on else 0))

    def set_field_precision(self, precision):
        """PREC_FP64 (default) or PREC_MIXED: near fields in fp32 with fp64 phases."""
        self.check(lib.tmat_ctx_set_field_precision(self.h, precision))

    def memory(self):
        """Device scratch held by this context, bytes."""
        b = ct.c_int64()
        self.check(lib.tmat_ctx_memory(self.h, ct.byref(b)))
        return b.value

    def launches(self):
        return lib.tmat_ctx_launch_count(self.h)

    def set_tensor_cores(self, on):
        """0/False: CUDA cores; 1/True: tensor cores (window-view kernel where it fits); 2: gather kernel."""
        self.check(lib.tmat_ctx_set_tensor_cores(self.h, int(on)))

    def set_lattice_fft(self, on):
        """1/True: lattice operators by FFT convolution where the grid fits, quad-mirror complex64 block
        products (default); 2: FFT with the mirror-pair block products; 0/False: direct kernels."""
        self.check(lib.tmat_ctx_set_lattice_fft(self.h, on if isinstance(on, int) and not isinstance(on, bool)
                                                else (1 if on else 0)))

    def set_timing(self, on):
        """True / False, or n > 1: one Arnoldi iteration in n of the complex64 inner solves timed."""
        every = int(on) if not isinstance(on, bool) else (1 if on else 0)
        self.check(lib.tmat_ctx_set_timing(self.h, every))

    def kernel_calls(self, kind):
        n = ct.c_int64()
        self.check(lib.tmat_ctx_kernel_calls(self.h, kind.encode(), ct.byref(n)))
        return n.value

    def kernel_time(self, kind):
        n, ms = ct.c_int64(), ct.c_double()
        self.check(lib.tmat_ctx_kernel_time(self.h, kind.encode(), ct.byref(n), ct.byref(ms)))
        return n.value, ms.value

    def kernel_bytes(self, kind):
        b = ct.c_double()
        self.check(lib.tmat_ctx_kernel_bytes(self.h, kind.encode(), ct.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "h", None):
            lib.tmat_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- calls, named as in tmat.h ----------------------------------------
    def tmat_neighbors(self, pos, cutoff):
        N = pos.shape[0]
        row_ptr = empty_like_space(pos, (N + 1,), np.int64)
        nnz = ct.c_int64()
        self.check(lib.tmat_neighbors(self.h, ptr(pos), N, cutoff, ptr(row_ptr), None, ct.byref(nnz)))
        col = empty_like_space(pos, (max(nnz.value, 1),), np.int32)
        self.check(lib.tmat_neighbors(self.h, ptr(pos), N, cutoff, ptr(row_ptr), ptr(col), ct.byref(nnz)))
        return row_ptr, col[:nnz.value]

    def tmat_subregions(self, nx, ny, cx, cy, buf):
        nsub, tot = ct.c_int64(), ct.c_int64()
        nsub_n = -(-nx // cx) * -(-ny // cy)
        core_ptr = np.empty(nsub_n + 1, np.int64)
        sim_ptr = np.empty(nsub_n + 1, np.int64)
        self.check(lib.tmat_subregions(self.h, nx, ny, cx, cy, buf, ptr(core_ptr), None, ptr(sim_ptr), None,
                                       ct.byref(nsub), ct.byref(tot)))
        core_idx = np.empty(nx * ny, np.int64)
        sim_idx = np.empty(tot.value, np.int64)
        self.check(lib.tmat_subregions(self.h, nx, ny, cx, cy, buf, ptr(core_ptr), ptr(core_idx), ptr(sim_ptr),
                                       ptr(sim_idx), ct.byref(nsub), ct.byref(tot)))
        return core_ptr, core_idx, sim_ptr, sim_idx

    def tmat_build(self, atoms, wavelength, n_bg, nmax, with_dr=False):
        """atoms: (N, 3) float64 [radius, n_re, n_im] (numpy or torch)."""
        N = atoms.shape[0]
        P = 2 * nmax * (nmax + 2)
        T = empty_like_space(atoms, (N, P), np.complex128)
        dT = empty_like_space(atoms, (N, P), np.complex128) if with_dr else None
        self.check(lib.tmat_build(self.h, ptr(atoms), N, wavelength, n_bg, nmax, ptr(T), ptr(dT)))
        return (T, dT) if with_dr else T

    def tmat_incident_planewave(self, pos, wavelength, n_bg, nmax, dirs, pol):
        N = pos.shape[0]
        R = dirs.shape[0]
        P = 2 * nmax * (nmax + 2)
        a0 = empty_like_space(pos, (R, N, P), np.complex128)
        self.check(lib.tmat_incident_planewave(self.h, ptr(pos), N, wavelength, n_bg, nmax, ptr(dirs), ptr(pol), R,
                                               ptr(a0)))
        return a0

    def tmat_incident_jinc(self, pos, wavelength, n_bg, nmax, src_xy, src_A, z0, n_beta=0, n_alpha=0,
                           precision=PREC_FP64, src_pitch=0.0):
        """src_A: (R, S, 2) complex transverse amplitudes."""
        N = pos.shape[0]
        R, S = src_A.shape[0], src_A.shape[1]
        P = 2 * nmax * (nmax + 2)
        a0 = empty_like_space(pos, (R, N, P), np.complex128)
        self.check(lib.tmat_incident_jinc(self.h, ptr(pos), N, wavelength, n_bg, nmax, ptr(src_xy), ptr(src_A), S, R,
                                          z0, src_pitch, n_beta, n_alpha, precision, ptr(a0)))
        return a0

    def tmat_translation(self, nmax, k, disp):
        M = disp.shape[0]
        P = 2 * nmax * (nmax + 2)
        xi = empty_like_space(disp, (M, P, P), np.complex128)
        self.check(lib.tmat_translation(self.h, nmax, k, ptr(disp), M, ptr(xi)))
        return xi

    def tmat_apply(self, op, precision, pos, k, nmax, T, row_ptr, col, x, cutoff=0.0, taper=0.0):
        R, N, P = x.shape
        y = empty_like_space(x, (R, N, P), np.complex128)
        self.check(lib.tmat_apply(self.h, op, precision, ptr(pos), N, k, nmax, ptr(T), ptr(row_ptr), ptr(col),
                                  cutoff, taper, ptr(x), R, ptr(y)))
        return y

    def tmat_apply_lattice(self, op, precision, nx, ny, pitch, cutoff, k, nmax, T, x, taper=0.0):
        R, N, P = x.shape
        y = empty_like_space(x, (R, N, P), np.complex128)
        self.check(lib.tmat_apply_lattice(self.h, op, precision, nx, ny, pitch, cutoff, taper, k, nmax, ptr(T), ptr(x),
                                          R, ptr(y)))
        return y

    def tmat_solve(self, pos, wavelength, n_bg, nmax, T, a0, opts, keep=False, s_out=None):
        R, N, P = a0.shape
        s = s_out if s_out is not None else empty_like_space(a0, (R, N, P), np.complex128)
        info = SolveInfo()
        sol = ct.c_void_p()
        rc = lib.tmat_solve(self.h, ptr(pos), N, wavelength, n_bg, nmax, ptr(T), ptr(a0), R, ct.byref(opts), ptr(s),
                            ct.byref(sol) if keep else None, ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return s, info, (Solution(sol) if keep else None), rc

    def tmat_forward(self, pos, atoms, wavelength, n_bg, nmax, dirs, pol, opts, pts, want_s=True, s_out=None,
                     E_out=None):
        """Build + incident + solve + field of every incidence in one call; returns (s or None,
        E [R][M][3], info, rc). Outputs go to s_out / E_out when given (e.g. pinned host arrays),
        else to new arrays in the memory space of pos."""
        N, R, M = pos.shape[0], dirs.shape[0], pts.shape[0]
        P = 2 * nmax * (nmax + 2)
        s = s_out if s_out is not None else (empty_like_space(pos, (R, N, P), np.complex128) if want_s else None)
        E = E_out if E_out is not None else empty_like_space(pos, (R, M, 3), np.complex128)
        info = SolveInfo()
        rc = lib.tmat_forward(self.h, ptr(pos), N, ptr(atoms), wavelength, n_bg, nmax, ptr(dirs), ptr(pol), R,
                              ct.byref(opts), ptr(pts), M, ptr(s) if s is not None else None, ptr(E), ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return s, E, info, rc

    def tmat_sweep(self, sw, atoms, wavelength, n_bg, nmax, src_A, opts, pts, E=None):
        """src_A: (R, nx*ny, 2); E (R, M, 3) is accumulated into (zeros if None)."""
        R = src_A.shape[0]
        M = pts.shape[0]
        if E is None:
            E = np.zeros((R, M, 3), dtype=np.complex128) if not _is_torch(pts) else empty_like_space(pts, (R, M, 3), np.complex128).zero_()
        info = SweepInfo()
        rc = lib.tmat_sweep(self.h, ct.byref(sw), ptr(atoms), wavelength, n_bg, nmax, ptr(src_A), R, ct.byref(opts),
                            ptr(pts), M, ptr(E), ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return E, info, rc

    def tmat_solve_batch(self, problems, n_bg, nmax, pitch, opts, canvas=(0, 0)):
        """problems: list of dicts nx, ny, wavelength, T (nx*ny, P), a0 (nx*ny, P) complex128 (numpy
        or torch). Returns (list of s (nx*ny, P), list of SolveInfo, rc)."""
        n = len(problems)
        arr = (BatchProblem * n)()
        outs = []
        for i, p in enumerate(problems):
            s = empty_like_space(p["a0"], p["a0"].shape, np.complex128)
            outs.append(s)
            arr[i].nx, arr[i].ny, arr[i].wavelength = p["nx"], p["ny"], p["wavelength"]
            arr[i].T_diag, arr[i].a0, arr[i].s_out = ptr(p["T"]).value, ptr(p["a0"]).value, ptr(s).value
        infos = (SolveInfo * n)()
        rc = lib.tmat_solve_batch(self.h, arr, n, n_bg, nmax, pitch, canvas[0], canvas[1], ct.byref(opts), infos)
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return outs, list(infos), rc

    def tmat_check_overlap(self, pos, radii):
        """None when no two enclosing spheres intersect, else the first pair (i, j)."""
        pair = np.zeros(2, np.int64)
        rc = lib.tmat_check_overlap(self.h, ptr(pos), pos.shape[0], ptr(radii), ptr(pair))
        if rc == EOVERLAP:
            return int(pair[0]), int(pair[1])
        self.check(rc)
        return None

    def tmat_build_cylinder(self, cyl, wavelength, n_bg, nmax, n_quad=0, with_dr=False):
        """cyl: (n, 4) float64 [radius, height, n_re, n_im]; returns T (n, P, P) [and dT/dradius]."""
        n = cyl.shape[0]
        P = 2 * nmax * (nmax + 2)
        T = empty_like_space(cyl, (n, P, P), np.complex128)
        dT = empty_like_space(cyl, (n, P, P), np.complex128) if with_dr else None
        self.check(lib.tmat_build_cylinder(self.h, ptr(cyl), n, wavelength, n_bg, nmax, n_quad, ptr(T), ptr(dT)))
        return (T, dT) if with_dr else T

    def tmat_solve_tblocks(self, pos, wavelength, n_bg, nmax, T_blocks, a0, opts, types=None, keep=False):
        """T_blocks (n_types, P, P); types (N,) int32 or None (block i for scatterer i)."""
        R, N, P = a0.shape
        s = empty_like_space(a0, (R, N, P), np.complex128)
        info = SolveInfo()
        sol = ct.c_void_p()
        rc = lib.tmat_solve_tblocks(self.h, ptr(pos), N, wavelength, n_bg, nmax, ptr(T_blocks), ptr(types),
                                    T_blocks.shape[0], ptr(a0), R, ct.byref(opts), ptr(s),
                                    ct.byref(sol) if keep else None, ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return s, info, (Solution(sol) if keep else None), rc

    def tmat_adjoint_tblocks(self, sol, v, dT_blocks, want_mu=False):
        N = v.shape[0]
        grad = empty_like_space(v, (N,), np.float64)
        mu = empty_like_space(v, v.shape, np.complex128) if want_mu else None
        info = SolveInfo()
        rc = lib.tmat_adjoint_tblocks(self.h, sol.h, ptr(v), ptr(dT_blocks), ptr(grad), ptr(mu), ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return grad, mu, info

    def tmat_field(self, pos, wavelength, n_bg, nmax, s, pts):
        M = pts.shape[0]
        E = empty_like_space(pts, (M, 3), np.complex128)
        self.check(lib.tmat_field(self.h, ptr(pos), pos.shape[0], wavelength, n_bg, nmax, ptr(s), ptr(pts), M, ptr(E)))
        return E

    def tmat_farfield(self, pos, wavelength, n_bg, nmax, s, dirs):
        M = dirs.shape[0]
        F = empty_like_space(dirs, (M, 3), np.complex128)
        self.check(lib.tmat_farfield(self.h, ptr(pos), pos.shape[0], wavelength, n_bg, nmax, ptr(s), ptr(dirs), M,
                                     ptr(F)))
        return F

    def tmat_point_fom(self, pos, wavelength, n_bg, nmax, s, x_f, E_inc_f):
        N = pos.shape[0]
        P = 2 * nmax * (nmax + 2)
        v = empty_like_space(s, (N, P), np.complex128)
        fom = ct.c_double()
        self.check(lib.tmat_point_fom(self.h, ptr(pos), N, wavelength, n_bg, nmax, ptr(s), ptr(x_f), ptr(E_inc_f),
                                      ct.byref(fom), ptr(v)))
        return fom.value, v

    def tmat_adjoint(self, sol, v, dTdr, want_mu=False):
        N = v.shape[0]
        grad = empty_like_space(v, (N,), np.float64)
        mu = empty_like_space(v, v.shape, np.complex128) if want_mu else None
        info = SolveInfo()
        rc = lib.tmat_adjoint(self.h, sol.h, ptr(v), ptr(dTdr), ptr(grad), ptr(mu), ct.byref(info))
        if rc not in (OK, ENOCONV):
            self.check(rc)
        return grad, mu, info

    def tmat_position_gradient(self, sol, mu, x_f, E_f, da0_dx=None, da0_dy=None):
        """dFoM/d(x_i, y_i) as (N, 2) float64 for a lattice solution; mu from tmat_adjoint
        (want_mu=True), E_f the total field at the focal point x_f."""
        N = mu.shape[0]
        grad = empty_like_space(mu, (N, 2), np.float64)
        self.check(lib.tmat_position_gradient(self.h, sol.h, ptr(mu), ptr(da0_dx), ptr(da0_dy), ptr(x_f), ptr(E_f),
                                              ptr(grad)))
        return grad


def tmat_measure_fma_peak(device, precision):
    """Measured FMA rate of `device` in TFLOP/s (PREC_MIXED: fp32, PREC_FP64: fp64)."""
    v = ct.c_double()
    rc = lib.tmat_measure_fma_peak(device, precision, ct.byref(v))
    if rc != OK:
        raise TMatError(rc, "tmat_measure_fma_peak failed")
    return v.value


class Solution:
    """Owner of a tmat_solution* (freed on garbage collection)."""

    def __init__(self, h):
        self.h = h

    def free(self):
        if getattr(self, "h", None):
            lib.tmat_solution_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_sweep(**kw):
    o = SweepOpts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_opts(**kw):
    o = SolveOpts()
    for k, v in kw.items():
        if k == "enclosing_radii" and v is not None:
            o._radii = v  # keep the array alive as long as the options
            v = ptr(v)
        setattr(o, k, v)
    return o
