"""torch.autograd.Function over the radii: forward = solve + focal FoM, backward = adjoint
solve. Checked against the oracle gradient, torch.autograd.gradcheck and, on the 50 x 50
adjoint workload, central finite differences of fp64 GPU solves (h = 1e-5 wavelengths)."""
import numpy as np
import pytest
import torch

from gpu_common import K0, ctx, rel_l2
from oracle import adjoint, incident, mie
from paper_2107_09879_b300 import _lib
from paper_2107_09879_b300 import workloads as W
from paper_2107_09879_b300.autograd import FocalProblem, focal_intensity

pytestmark = pytest.mark.gpu


def _problem(pos, nmax, xf, opts, device=None):
    A = np.array([1.0, 0.0, 0.0], dtype=complex)
    Einc = incident.planewave_field(K0, 0.0, 0.0, A, xf[None])[0]
    a0 = ctx().tmat_incident_planewave(pos, 1.0, 1.0, nmax, np.array([[0.0, 0.0]]), A[None])
    if device is not None:
        pos = torch.from_numpy(pos).to(device)
        a0 = torch.from_numpy(a0).to(device)
    return FocalProblem(ctx=ctx(), pos=pos, nmax=nmax, wavelength=1.0, n_bg=1.0, n_sphere=2.0, a0=a0, x_f=xf,
                        E_inc_f=Einc, opts=opts)


@pytest.mark.parametrize("device", [None, "cuda"])
def test_autograd_matches_oracle_gradient(device):
    nmax, cutoff = 3, 0.8
    pos = W.lattice_positions(3, 2)
    r = W.uniform_radii(6, 0.1, 0.22, 7)
    xf = np.array([0.5, 0.25, 3.0])
    opts = _lib.make_opts(tol=1e-12, restart=60, max_iter=2000, cutoff=cutoff, precision=_lib.PREC_FP64)
    prob = _problem(pos, nmax, xf, opts, device)
    rt = torch.tensor(r, dtype=torch.float64, device=device or "cpu", requires_grad=True)
    fom = focal_intensity(rt, prob)
    fom.backward()
    To = np.array([mie.tmatrix_diag(nmax, K0, x, 2.0) for x in r])
    dTo = np.array([mie.tmatrix_diag_dr(nmax, K0, x, 2.0) for x in r])
    from oracle import system
    a0 = incident.planewave_incident(nmax, K0, pos, 0.0, 0.0, np.array([1.0, 0.0, 0.0], dtype=complex))[None]
    so = system.solve_dense(nmax, K0, pos, To, a0[0], cutoff)
    Einc = prob.E_inc_f
    assert abs(fom.item() - adjoint.fom(nmax, K0, pos, so, xf, Einc)) <= 1e-9 * fom.item()
    vo = adjoint.adjoint_source(nmax, K0, pos, so, xf, Einc)
    go, _ = adjoint.radius_gradient(nmax, K0, pos, To, dTo, a0[0], so, vo, cutoff=cutoff)
    assert rel_l2(rt.grad.cpu().numpy(), go) <= 1e-9


def test_autograd_gradcheck():
    nmax, cutoff = 2, 1.2
    pos = W.lattice_positions(3, 3)
    r = W.uniform_radii(9, 0.1, 0.22, 11)
    xf = np.array([0.5, 0.5, 2.0])
    opts = _lib.make_opts(tol=1e-13, restart=60, max_iter=2000, cutoff=cutoff, precision=_lib.PREC_FP64)
    prob = _problem(pos, nmax, xf, opts)
    rt = torch.tensor(r, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: focal_intensity(x, prob), (rt,), eps=1e-6, atol=1e-6, rtol=1e-4)


def test_adjoint_workload_50x50_vs_central_differences():
    """50 x 50 spheres, nmax 4, cutoff 10 (raised-cosine window over [0, cutoff]), focal point
    20 wavelengths above the centre: the mixed-precision adjoint gradient of all 2,500 radii
    against the fp64 adjoint gradient, and both against central differences (h = 1e-5) of fp64
    solves at 8 seeded radii."""
    w = W.lattice_50x50_adjoint()
    nmax, cut = w["nmax"], w["cutoff"]
    lat = dict(path=_lib.PATH_LATTICE, lattice_nx=50, lattice_ny=50, lattice_pitch=0.5, taper=cut, cutoff=cut)
    o64 = _lib.make_opts(tol=1e-11, restart=300, max_iter=4000, precision=_lib.PREC_FP64, **lat)
    omx = _lib.make_opts(tol=1e-7, restart=300, max_iter=4000, precision=_lib.PREC_MIXED, inner_tol=1e-4, **lat)
    grads = {}
    for name, opts in (("fp64", o64), ("mixed", omx)):
        prob = _problem(w["pos"], nmax, w["focus"], opts, "cuda")
        rt = torch.tensor(w["radius"], dtype=torch.float64, device="cuda", requires_grad=True)
        fom = focal_intensity(rt, prob)
        fom.backward()
        grads[name] = rt.grad.cpu().numpy()
        assert prob.last_info.converged
    g = grads["fp64"]
    assert rel_l2(grads["mixed"], g) <= 1e-4
    prob = _problem(w["pos"], nmax, w["focus"], o64, "cuda")
    idx = np.sort(np.random.default_rng(2107_09879).choice(2500, 8, replace=False))
    h = 1e-5
    gmax = np.max(np.abs(g))
    for i in idx:
        f = []
        for sgn in (1, -1):
            rr = torch.tensor(w["radius"], dtype=torch.float64, device="cuda")
            rr[i] += sgn * h
            with torch.no_grad():
                f.append(focal_intensity(rr, prob).item())
        fd = (f[0] - f[1]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-4 * gmax, (i, g[i], fd)
        assert abs(grads["mixed"][i] - fd) <= 1e-4 * gmax, (i, grads["mixed"][i], fd)
