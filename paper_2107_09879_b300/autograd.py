"""Differentiable focal-point figure of merit over the sphere radii (torch.autograd).

`TMatSolve.apply(radii, problem)` returns FoM(r) = sum_c |E_inc,c(x_f) + E_sca,c(x_f)|^2,
the total-field intensity at one focal point (the adjoint section's objective with the
incident field included; the incident field does not depend on the radii, so the
gradient formula is unchanged).

forward:  tmat_build (T and dT/dr per sphere) -> tmat_solve (keeps the operator for the
          adjoint) -> tmat_point_fom (FoM and v = dFoM/ds, the Wirtinger derivative)
backward: tmat_adjoint solves (I - A^T T) mu = v and returns dFoM/dr_i =
          2 Re[mu_i^T T'_i e_i] with e_i = a0_i + (A s)_i; the incoming gradient scales it.

Every step runs in the native library; this module only marshals arguments. The
solve's Krylov basis is not kept: the backward pass runs a fresh adjoint solve on
the stored operator, so memory stays at one solve.
"""
import dataclasses

import numpy as np
import torch

from . import _lib


@dataclasses.dataclass
class FocalProblem:
    """Everything but the radii: positions (N, 3), sphere and background index, the
    incident coefficients a0 (1, N, P) and the incident field at the focal point."""

    ctx: "_lib.Context"
    pos: object
    nmax: int
    wavelength: float
    n_bg: float
    n_sphere: complex
    a0: object
    x_f: object
    E_inc_f: object
    opts: "_lib.SolveOpts"
    last_info: dict = None


def _atoms(radii, n_sphere):
    """(N, 3) float64 [radius, n_re, n_im] in the radii's memory space."""
    r = radii.detach().to(torch.float64)
    a = torch.empty((r.shape[0], 3), dtype=torch.float64, device=r.device)
    a[:, 0] = r
    a[:, 1] = float(np.real(n_sphere))
    a[:, 2] = float(np.imag(n_sphere))
    return a if a.is_cuda else a.numpy()


def _as_tensor(x, like):
    if isinstance(x, torch.Tensor):
        return x.to(device=like.device, dtype=like.dtype)
    return torch.from_numpy(np.asarray(x)).to(device=like.device, dtype=like.dtype)


class TMatSolve(torch.autograd.Function):
    """FoM(radii) with an adjoint backward; see the module docstring."""

    @staticmethod
    def forward(fctx, radii, problem):
        p = problem
        c = p.ctx
        atoms = _atoms(radii, p.n_sphere)
        T, dT = c.tmat_build(atoms, p.wavelength, p.n_bg, p.nmax, with_dr=True)
        s, info, sol, rc = c.tmat_solve(p.pos, p.wavelength, p.n_bg, p.nmax, T, p.a0, p.opts, keep=True)
        if rc != _lib.OK:
            sol.free()
            raise _lib.TMatError(rc, f"forward solve did not converge: {info}")
        p.last_info = info
        fom, v = c.tmat_point_fom(p.pos, p.wavelength, p.n_bg, p.nmax, s[0], p.x_f, p.E_inc_f)
        fctx.sol, fctx.v, fctx.dT, fctx.problem = sol, v, dT, p
        return torch.tensor(fom, dtype=torch.float64, device=radii.device)

    @staticmethod
    def backward(fctx, grad_out):
        p = fctx.problem
        # the solution stays alive until the graph is freed (backward may run again with
        # retain_graph); its destructor releases the device state
        grad, _, info = p.ctx.tmat_adjoint(fctx.sol, fctx.v, fctx.dT)
        g = _as_tensor(grad, grad_out)
        return grad_out * g, None


def focal_intensity(radii, problem):
    """FoM(radii) = sum_c |E_c(x_f)|^2, differentiable in the radii."""
    return TMatSolve.apply(radii, problem)
