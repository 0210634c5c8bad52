"""Served stream with continuous batching: each result is the same alone and in the mix (the
mixed path's tolerance), requests share batched launches, admission respects the memory
budget, and a sample of small requests matches the oracle."""
import math

import numpy as np
import pytest

from paper_2107_09879_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_results_same_alone_and_in_the_mix():
    from paper_2107_09879_b300 import serve
    reqs = W.served_stream(10, seed=W.BASE_SEED + 3, rate_per_s=1000.0, k_lo=6, k_hi=14)
    srv = serve.Server(slots=2, mem_budget=16 << 30, max_batch=4)
    mixed = srv.run(reqs, keep_solutions=True)
    srv.close()
    assert all("E" in r and r["rc"] == 0 for r in mixed), mixed
    assert max(r["batch"] for r in mixed) >= 2  # some requests shared launches
    # batches overlapped on the GPU: some request was admitted before another one finished
    assert any(a["admit"] < b["finish"] and b["admit"] < a["finish"] for a in mixed for b in mixed
               if a["slot"] != b["slot"])
    for req in reqs[:5]:
        alone = serve.Server(slots=1, mem_budget=16 << 30, max_batch=1)
        rec = alone.run([dict(req, arrival=0.0)], keep_solutions=True)[0]
        alone.close()
        mix = mixed[req["rid"]]
        assert _rel(mix["s"], rec["s"]) <= 1e-6
        assert _rel(mix["E"], rec["E"]) <= 1e-6


def test_admission_respects_memory_budget():
    """A budget that fits one request at a time serialises the stream into batches of one."""
    from paper_2107_09879_b300 import serve
    reqs = W.served_stream(5, seed=W.BASE_SEED + 4, rate_per_s=1000.0, k_lo=8, k_hi=8)
    for r in reqs:
        r["nmax"] = 4  # equal estimates
    est = [serve.request_bytes(r["side"], r["nmax"]) for r in reqs]
    budget = max(est)
    assert 2 * min(est) > budget  # so no two requests fit together
    srv = serve.Server(slots=4, mem_budget=budget, max_batch=8)
    recs = srv.run(reqs)
    srv.close()
    assert all("E" in r for r in recs)
    assert srv.mem_high <= budget and all(b == 1 for b in srv.batches)
    spans = sorted((r["admit"], r["finish"]) for r in recs)
    assert all(spans[i][1] <= spans[i + 1][0] + 1e-3 for i in range(len(spans) - 1))  # one at a time
    assert srv.ctx_mem_high > 0


def test_served_results_match_the_oracle():
    """Small requests (3 x 3 cores with a 1-site ring, nmax 2, fp64-checked): the served field at
    the detector and the coefficients against the oracle's jinc sources, dense solve and field."""
    from oracle import field, incident, mie, system
    from paper_2107_09879_b300 import serve
    reqs = W.served_stream(3, seed=W.BASE_SEED + 7, rate_per_s=1000.0, k_lo=3, k_hi=3, buf=1)
    for r in reqs:
        r["nmax"] = 2
    srv = serve.Server(slots=1, mem_budget=16 << 30, max_batch=4, cutoff=1.2, tol=1e-9)
    recs = srv.run(reqs, keep_solutions=True)
    srv.close()
    for req, rec in zip(reqs, recs):
        side, k, b, w = req["side"], req["k"], req["buf"], req["wavelength"]
        kk = 2 * math.pi / w
        pos = W.lattice_positions(side, side)
        cy, cx = np.divmod(np.arange(k * k), k)
        src = np.stack([(cx + b) * 0.5, (cy + b) * 0.5], axis=1)
        A = np.zeros((k * k, 2), complex)
        A[:, 0] = np.exp(1j * kk * srv.z0)
        ext = max(np.hypot(*(p[:2] - q)) for p in pos for q in src) + abs(srv.z0)
        rule = incident.jinc_rule(*incident.jinc_rule_size(kk, ext))
        a0 = incident.jinc_group_coeffs(2, kk, pos, src, A, srv.z0, rule, pitch=0.5)
        To = np.array([mie.tmatrix_diag(2, kk, x, 2.0) for x in req["radii"]])
        with system.window(1.2, 1.2):
            so = system.solve_dense(2, kk, pos, To, a0, 1.2)
        c = (side - 1) * 0.25
        Eo = field.scattered_field(2, kk, pos, so, np.array([[c, c, srv.det_h]]))
        assert _rel(rec["s"], so) <= 1e-6
        assert _rel(rec["E"], Eo) <= 1e-6


def test_sweep_through_the_request_loop_matches_tmat_sweep_and_oracle():
    """A small large-area sweep served as sub-region requests (batched, shifted to the origin)
    against tmat_sweep (absolute coordinates) and the oracle's sweep definition."""
    from oracle import incident, sweep
    from paper_2107_09879_b300 import _lib, serve
    from gpu_common import K0, atoms, ctx
    nx, ny, core, buf, nmax, cut, z0 = 14, 11, 5, 2, 2, 1.2, -1.0
    r = W.smooth_radius_map(nx, ny, W.BASE_SEED + 9)
    pos = W.lattice_positions(nx, ny)
    src = np.zeros((2, nx * ny, 2), complex)
    for q, deg in enumerate((0.0, 8.0)):
        th = math.radians(deg)
        src[q, :, 0] = math.cos(th) * np.exp(1j * K0 * (math.sin(th) * pos[:, 0] + math.cos(th) * z0))
    pts = np.array([[1.0, 2.0, 3.0], [4.5, 2.5, 2.0], [6.0, 4.0, 5.0]])
    reqs = serve.sweep_requests(nx, ny, core, buf, 0.5, r, 2.0, src, z0, pts, nmax)
    srv = serve.Server(slots=2, mem_budget=16 << 30, max_batch=4, cutoff=cut, tol=1e-9, restart=100)
    recs = srv.run(reqs)
    srv.close()
    assert all("E" in x and x["rc"] == 0 for x in recs)
    E = serve.sweep_field(recs, 2, len(pts))
    opts = _lib.make_opts(tol=1e-9, restart=100, max_iter=3000, cutoff=cut, taper=cut, precision=_lib.PREC_MIXED)
    sw = _lib.make_sweep(nx=nx, ny=ny, pitch=0.5, core_x=core, core_y=core, buffer=buf, z0=z0)
    Ed, info, rc = ctx().tmat_sweep(sw, atoms(r), 1.0, 1.0, nmax, src, opts, pts)
    assert rc == 0 and _rel(E, Ed) <= 1e-6
    xy = pos[:, :2]
    rule_for = lambda p, s: incident.jinc_rule(*incident.jinc_rule_size(
        K0, max(np.hypot(*(a[:2] - b)) for a in p for b in s) + abs(z0)))
    Eo = sweep.sweep_fields(nmax, K0, nx, ny, 0.5, 0.0, r, 2.0, src[0], z0, (core, core), buf, pts, rule_for,
                            cutoff=cut, taper=cut)
    assert _rel(E[0], Eo) <= 1e-6
