"""Benchmark of the T-matrix hot path on one workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = the whole hot path over one synthetic input: Mie T-matrices of every
sphere, plane-wave incident coefficients for the two incidences, the coupled
solve (GMRES on the block-Toeplitz lattice operator, complex64 apply with fp64
iterative refinement to 1e-6), and the scattered field at a line of detector
points. Workload: 200 x 200 spheres on a 0.5-wavelength lattice, radii
U[0.08, 0.24], index 2.0, nmax = 4 (P = 48), cutoff 8 wavelengths, plane waves
at 0 and 10 degrees. `value` counts solves (one solve = both incidences) per
second with inputs resident in HBM; `e2e` repeats the step through the C ABI
with pinned host buffers (host<->device copies inside the timed region).

Multi-GPU: the solve does not shard; N processes run N independent replicas
(weak scaling), one per GPU, launched by torchrun.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_09879_b300 import workloads as W  # noqa: E402

PITCH = 0.5
METRIC = "solves/s + p50/p99 latency; T-matvec GFLOP/s, mixed vs FP64 at 1e-6 rel err"
UNIT = "solves/s"
TOL = 1e-7  # refinement stops at ||r|| / ||b|| <= 1e-7, so the solution error is <= 1e-6
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
HBM_PEAK_GBS = 6451.5  # measured copy bandwidth of the B300s (MEASURED_PEAKS.json)


def workload(size=200):
    """The 200 x 200 workload; `size` < 200 takes its lower-left size x size corner (smaller
    cases of the same structure, for profiler captures)."""
    w = dict(W.lattice_200x200())
    nx = ny = size
    if size != 200:
        keep = [iy * 200 + ix for iy in range(size) for ix in range(size)]
        w["pos"] = w["pos"][keep]
        w["radius"] = w["radius"][keep]
    a = np.zeros((nx * ny, 3))
    a[:, 0] = w["radius"]
    a[:, 1] = w["n_sphere"]
    dirs = np.array([[math.radians(d), 0.0] for d in w["angles_deg"]])
    pols = np.array([[math.cos(d[0]), 0.0, -math.sin(d[0])] for d in dirs], dtype=complex)  # p-pol (beta-hat)
    pts = np.array([[x, 49.75, 20.0] for x in np.linspace(40.0, 60.0, 64)])
    return dict(w=w, nx=nx, ny=ny, pos=w["pos"], atoms=a, dirs=dirs, pols=pols, pts=pts)


def pairs_within(nx, ny, cutoff_sites):
    """Directed pairs of an nx x ny lattice with offsets inside the cutoff."""
    c2 = cutoff_sites * cutoff_sites
    tot = 0
    for dy in range(-cutoff_sites, cutoff_sites + 1):
        for dx in range(-cutoff_sites, cutoff_sites + 1):
            if (dx or dy) and dx * dx + dy * dy <= c2:
                tot += max(0, nx - abs(dx)) * max(0, ny - abs(dy))
    return tot


class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) / algorithmic bytes of one ncu capture of each HBM-bound kernel as
# it stands, scaled to the timed launches by their algorithmic bytes (traffic grows with the
# bytes a launch must move): profiles/arnoldi_dcgs2_100x100_nmax4.md (dot and update passes),
# profiles/lattice_fft_200x200_nmax4.md (block product). Set an entry to None when its kernel
# changes.
TRAFFIC_RATIO = {"arnoldi_dots32": (490.18e6 + 4.41e6) / (62 * 2 * 480000 * 8),
                 "arnoldi_update32": (468.52e6 + 13.44e6) / (63 * 2 * 480000 * 8),
                 "lattice_fft_mul32": (390.22e6 + 40.69e6) / 405.01e6}
# DRAM bytes per launch of the direct-path kernels (profiles/lattice_tc2_200x200_nmax4.md) and
# of the block product (profiles/lattice_fft_200x200_nmax4.md)
MEASURED_TRAFFIC = {"lattice_tc2_kernel<4,0>": 238.0e6 + 23.0e6,
                    "fft_mul_kernel<float,24,0,2>": 390.22e6 + 40.69e6}


def roofline(kern_name, achieved, launches, avg_ms, flop_per_launch):
    extra = {}
    if "tcgen05" in kern_name:
        # TF32 dense peak of measured: bf16 burst 1736 TFLOP/s x nominal TF32/BF16 ratio 1.1/2.25.
        # 3xTF32 executes 3 tensor GEMMs per algorithmic product, so frac <= 1/3 by construction.
        peak = 1736.0 * 1.1 / 2.25
        note = "TF32 dense: measured bf16 burst 1736 x nominal 1.1/2.25 (of measured)"
        bound = "tensor"
        extra = {"tensor_flop_per_algorithmic_flop": 3,
                 "tensor_pipe_frac": (3 * achieved / peak) if achieved else None}
    else:
        peak, note = FP32_PEAK_TFLOPS, "FP32 FMA issue rate: 148 SMs x 128 lanes x 2 flop x 2.032 GHz (derived)"
        bound = "alu"
    traffic = next((v for k, v in MEASURED_TRAFFIC.items() if kern_name.startswith(k)), None)
    out = {"kernel": kern_name, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": (achieved / peak) if achieved else None, "traffic": traffic, "launches": launches,
           "avg_launch_ms": avg_ms, "flop_per_launch": flop_per_launch, "peak_note": note}
    out.update(extra)
    return out


def roofline_hbm(hbm, step_total_ms):
    """The dominant kernel (largest summed time in the timed region) of the HBM-bound ones
    the library counts algorithmic bytes for: achieved = its bytes / its time."""
    kind, v = max(hbm.items(), key=lambda kv: kv[1]["total_ms"])
    achieved = v["bytes"] / (v["total_ms"] * 1e-3) / 1e9
    ratio = TRAFFIC_RATIO.get(kind)
    return {"kernel": v["kernel"], "bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
            "frac": achieved / HBM_PEAK_GBS,
            "traffic": (ratio * v["bytes"] / v["launches"]) if ratio else None,
            "launches": v["launches"], "avg_launch_ms": v["total_ms"] / v["launches"],
            "bytes_per_launch": v["bytes"] / v["launches"], "share_of_timed_region": v["total_ms"] / step_total_ms,
            "peak_note": "STREAM-style copy bandwidth of MEASURED_PEAKS.json (of measured)"}


def cpu_baseline(wl, matvecs_per_solve, budget_s=12.0):
    """The oracle (plain fp64 numpy, test infrastructure) on a bounded sample:
    rows of one operator application for both incidences, extrapolated to the
    full matvec and to the solve's number of operator applications."""
    from oracle import geometry, mie, system
    pos, nmax, cutoff = wl["pos"], wl["w"]["nmax"], wl["w"]["cutoff"]
    k = 2 * math.pi
    N = len(pos)
    rng = np.random.default_rng(0)
    x = (rng.normal(size=(2, N, 48)) + 1j * rng.normal(size=(2, N, 48))) * 0.1
    centre = [(100 + dy) * 200 + 100 + dx for dy in range(-8, 8) for dx in range(-8, 8)]
    # neighbour rows of the sampled targets only (the oracle's definition, restricted)
    t0 = time.perf_counter()
    rows_done = 0
    for i in centre:
        d = pos - pos[i]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        d2 = d2 + d[:, 2] * d[:, 2]
        js = np.nonzero(d2 <= cutoff * cutoff)[0]
        js = js[js != i].astype(np.int32)
        rp = np.zeros(N + 1, dtype=np.int64)
        rp[i + 1:] = len(js)
        Ti = np.zeros((N, 48), complex)
        Ti[i] = mie.tmatrix_diag(nmax, k, wl["w"]["radius"][i], 2.0)
        for q in range(2):
            system.apply_K_rows(nmax, k, pos, Ti, x[q], (rp, js), [i])
        rows_done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    per_matvec = dt / rows_done * N
    per_solve = per_matvec * matvecs_per_solve
    return {"value": 1.0 / per_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{rows_done} interior target rows of one operator application (both incidences, "
                      f"{dt:.1f} s), extrapolated x{N / rows_done:.0f} to one application and "
                      f"x{matvecs_per_solve} applications per solve (the GPU run's count)"}


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, t_max_ms):
    """Solves per second of the whole job: every rank solves `steps` independent
    problems (replicas, weak scaling) within the slowest rank's time."""
    return world * steps / (t_max_ms / 1e3)


def _wall(fn, sync):
    sync()
    t0 = time.perf_counter()
    r = fn()
    sync()
    return time.perf_counter() - t0, r


def bench_dense_fp64(ctx, torch, steps=20):
    """8 x 8 spheres, nmax 3, every pair coupled, fp64 GMRES to 1e-10: on the lattice path
    (every offset of the 8 x 8 lattice; FFT convolution) and on the neighbour-list path."""
    from paper_2107_09879_b300 import _lib
    w = W.dense_8x8()
    a = np.zeros((64, 3))
    a[:, 0], a[:, 1] = w["radius"], w["n_sphere"]
    pos = torch.from_numpy(w["pos"]).cuda()
    atoms = torch.from_numpy(a).cuda()
    dirs = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    pol = torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.complex128, device="cuda")
    out = {"workload": "dense_8x8_nmax3_fp64_tol1e-10",
           "note": "one solve = Mie build + incident + GMRES; launched eagerly (no graph capture)"}
    for path, extra in (("lattice", dict(path=_lib.PATH_LATTICE, lattice_nx=8, lattice_ny=8, lattice_pitch=PITCH)),
                        ("neighbour", dict(path=_lib.PATH_NEIGHBOUR))):
        opts = _lib.make_opts(tol=w["tol"], restart=100, max_iter=2000, cutoff=0.0, precision=_lib.PREC_FP64, **extra)
        info = []

        def one():
            T = ctx.tmat_build(atoms, 1.0, 1.0, w["nmax"])
            a0 = ctx.tmat_incident_planewave(pos, 1.0, 1.0, w["nmax"], dirs, pol)
            s, inf, _, rc = ctx.tmat_solve(pos, 1.0, 1.0, w["nmax"], T, a0, opts)
            info.append(inf)
            return rc
        for _ in range(3):
            one()
        dt, _ = _wall(lambda: [one() for _ in range(steps)], torch.cuda.synchronize)
        out[path] = {"solves_per_s": steps / dt, "ms_per_solve": dt / steps * 1e3, "iterations": info[-1].iterations,
                     "rel_residual": info[-1].rel_residual[0]}
    out["solves_per_s"] = out["lattice"]["solves_per_s"]
    return out


def bench_adjoint(ctx, torch, steps=3):
    """50 x 50 spheres, nmax 4, cutoff 10 (raised-cosine window), focal |E|^2 at 20 wavelengths:
    forward solve + FoM + adjoint solve + gradient of all 2,500 radii, mixed precision to 1e-7."""
    from paper_2107_09879_b300 import _lib
    w = W.lattice_50x50_adjoint()
    nmax, cut = w["nmax"], w["cutoff"]
    a = np.zeros((2500, 3))
    a[:, 0], a[:, 1] = w["radius"], w["n_sphere"]
    pos = torch.from_numpy(w["pos"]).cuda()
    atoms = torch.from_numpy(a).cuda()
    dirs = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    pol = torch.tensor([[1.0, 0.0, 0.0]], dtype=torch.complex128, device="cuda")
    xf = w["focus"]
    E_inc = np.array([np.exp(1j * 2 * math.pi * xf[2]), 0.0, 0.0])  # x-polarised plane wave along +z
    opts = _lib.make_opts(tol=1e-7, restart=300, max_iter=4000, cutoff=cut, taper=cut, precision=_lib.PREC_MIXED,
                          inner_tol=1e-4, path=_lib.PATH_LATTICE, lattice_nx=50, lattice_ny=50, lattice_pitch=PITCH)
    rec = []

    def one():
        T, dT = ctx.tmat_build(atoms, 1.0, 1.0, nmax, with_dr=True)
        a0 = ctx.tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pol)
        s, fi, sol, rc = ctx.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
        fom, v = ctx.tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, E_inc)
        g, _, ai = ctx.tmat_adjoint(sol, v, dT)
        sol.free()
        rec.append((fi.iterations, ai.iterations, fi.rel_residual[0], ai.rel_residual[0]))
        return g
    one()
    dt, g = _wall(lambda: [one() for _ in range(steps)][-1], torch.cuda.synchronize)
    fi, ai, fr, ar = rec[-1]
    # position gradient dFoM/d(x_i, y_i) from the same adjoint solution (normal incidence:
    # the incident coefficients do not change with in-plane positions)
    T, dT = ctx.tmat_build(atoms, 1.0, 1.0, nmax, with_dr=True)
    a0 = ctx.tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pol)
    s, fi2, sol, rc = ctx.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts, keep=True)
    fom, v = ctx.tmat_point_fom(pos, 1.0, 1.0, nmax, s[0], xf, E_inc)
    _, mu, _ = ctx.tmat_adjoint(sol, v, dT, want_mu=True)
    Ef = np.ascontiguousarray(E_inc + ctx.tmat_field(pos, 1.0, 1.0, nmax, s[0],
                                                     torch.from_numpy(np.asarray(xf)[None]).cuda()).cpu().numpy()[0])
    xf_a = np.ascontiguousarray(np.asarray(xf, dtype=np.float64))
    ctx.tmat_position_gradient(sol, mu, xf_a, Ef)
    dtp, gp = _wall(lambda: [ctx.tmat_position_gradient(sol, mu, xf_a, Ef) for _ in range(steps)][-1],
                    torch.cuda.synchronize)
    sol.free()
    return {"workload": "lattice_50x50_nmax4_cutoff10_adjoint_mixed", "gradients_per_s": steps / dt,
            "ms_per_gradient": dt / steps * 1e3, "forward_iterations": fi, "adjoint_iterations": ai,
            "forward_rel_residual": fr, "adjoint_rel_residual": ar, "grad_norm": float(torch.linalg.vector_norm(g)),
            "position_gradient_ms": dtp / steps * 1e3,
            "position_grad_norm": float(torch.linalg.vector_norm(gp)) if hasattr(gp, "shape") else None,
            "note": "one gradient = Mie build with dT/dr + incident + forward solve + focal FoM + adjoint solve; "
                    "position_gradient_ms: dFoM/d(x_i, y_i) of all 2,500 spheres from the kept adjoint "
                    "solution (derivative blocks, their fp64 spectra, four fp64 FFT applies, explicit field term)"}


def bench_served(args, torch):
    """Served stream of sub-region requests (k x k jinc core + 4-pitch ring, k ~ U{10..60},
    nmax ~ U{3,4,5}, wavelength ~ U[0.9, 1.1]): Poisson arrivals at 1.5x and 0.5x of the
    measured single-stream service rate."""
    from paper_2107_09879_b300 import serve
    calib = W.served_stream(8, seed=W.BASE_SEED + 3, rate_per_s=0.0)
    srv = serve.Server(slots=1, mem_budget=64 << 30)
    srv.run(calib[:2])  # warm-up
    t0 = time.perf_counter()
    srv.run(calib)
    mu = len(calib) / (time.perf_counter() - t0)
    srv.close()
    out = {"workload": "served_subregions_k10-60_ring4_nmax3-5_mixed", "single_stream_solves_per_s": mu}
    for name, factor, n in (("rate_1.5x", 1.5, args.served_requests), ("rate_0.5x", 0.5, max(8, args.served_requests // 4))):
        reqs = W.served_stream(n, seed=W.BASE_SEED + 3, rate_per_s=factor * mu)
        srv = serve.Server(slots=4, mem_budget=64 << 30)
        t0 = time.perf_counter()
        recs = srv.run(reqs)
        wall = time.perf_counter() - t0
        srv.close()
        summ = serve.summarize(recs, wall)
        summ["arrival_rate_per_s"] = factor * mu
        summ["mem_high_water_bytes_est"] = srv.mem_high
        out[name] = summ
    return out


def bench_sweep(ctx, torch, inner_tol=0.1):
    """1200 x 1200 spheres (smooth radius map), nmax 3, cutoff 6, 60 x 60 cores + 8-pitch rings,
    4 incidences as RHS, mixed: four sampled sub-regions (corner, edge, two interior),
    extrapolated to the 400-sub-region sweep."""
    from paper_2107_09879_b300 import _lib
    n = 1200
    r = W.smooth_radius_map(n, n, W.BASE_SEED + 5)
    atoms = np.zeros((n * n, 3))
    atoms[:, 0], atoms[:, 1] = r, 2.0
    pos = W.lattice_positions(n, n)
    z0 = -1.0
    src = np.zeros((4, n * n, 2), complex)
    for q, deg in enumerate((0.0, 5.0, 10.0, 15.0)):
        th = math.radians(deg)
        src[q, :, 0] = math.cos(th) * np.exp(1j * 2 * math.pi * (math.sin(th) * pos[:, 0] + math.cos(th) * z0))
    pts = np.array([[x, 300.0, 20.0] for x in np.linspace(0.0, 600.0, 64)])
    opts = _lib.make_opts(tol=1e-7, restart=300, max_iter=4000, cutoff=6.0, taper=6.0, precision=_lib.PREC_MIXED,
                          inner_tol=inner_tol)
    d_atoms = torch.from_numpy(atoms).cuda()
    d_src = torch.from_numpy(src).cuda()
    d_pts = torch.from_numpy(pts).cuda()
    E = torch.zeros((4, 64, 3), dtype=torch.complex128, device="cuda")
    samples = {"corner": 0, "edge": 10, "interior_a": 210, "interior_b": 114}
    kw = dict(nx=n, ny=n, pitch=PITCH, core_x=60, core_y=60, buffer=8, z0=z0)
    # warm-up on the corner job
    ctx.tmat_sweep(_lib.make_sweep(first=0, count=1, **kw), d_atoms, 1.0, 1.0, 3, d_src, opts, d_pts, E=E)
    per = {}
    infos = {}
    for name, first in samples.items():
        dt, res = _wall(lambda: ctx.tmat_sweep(_lib.make_sweep(first=first, count=1, **kw), d_atoms, 1.0, 1.0, 3,
                                               d_src, opts, d_pts, E=E), torch.cuda.synchronize)
        per[name] = dt
        infos[name] = res[1]
    mean = statistics.mean(per.values())
    return {"workload": "sweep_1200x1200_nmax3_cutoff6_core60_ring8_4rhs_mixed",
            "seconds_per_subregion": per, "subregions_per_s": 1.0 / mean,
            "extrapolated_sweep_s": 400 * mean,
            "iterations": {k: v.iterations for k, v in infos.items()},
            "worst_rel_residual": max(v.worst_rel_residual for v in infos.values()),
            "note": "sampled sub-regions (corner, edge, 2 interior) timed; full sweep extrapolated x400 from their mean"}


def bench_padding(ctx, torch):
    """Padding (buffer-ring) convergence of the sub-region decomposition, the synthetic
    analog of the paper's padding study: an 80 x 80 array (nmax 3, smooth radius map, cutoff 6
    with a raised-cosine window, jinc sources sampling a normally incident x-polarised plane
    wave at z0 = -1) solved whole and as 16 sub-regions of 20 x 20 with rings of 0..16 pitches;
    error of the summed field on a detector line 10 wavelengths above the array, and of the
    intensity at its brightest point, against the whole-array solve (fp64 throughout)."""
    from paper_2107_09879_b300 import _lib
    n, nmax, z0, cut = 80, 3, -1.0, 6.0
    r = W.smooth_radius_map(n, n, W.BASE_SEED + 6)
    at = np.zeros((n * n, 3))
    at[:, 0], at[:, 1] = r, 2.0
    pos = W.lattice_positions(n, n)
    src = np.zeros((1, n * n, 2), complex)
    src[0, :, 0] = np.exp(1j * 2 * math.pi * z0)
    pts = np.array([[x, 19.75, 10.0] for x in np.linspace(5.0, 35.0, 32)])
    opts = _lib.make_opts(tol=1e-11, restart=200, max_iter=4000, cutoff=cut, taper=cut, precision=_lib.PREC_FP64,
                          path=_lib.PATH_LATTICE, lattice_nx=n, lattice_ny=n, lattice_pitch=PITCH)
    T = ctx.tmat_build(at, 1.0, 1.0, nmax)
    a0 = ctx.tmat_incident_jinc(pos, 1.0, 1.0, nmax, np.ascontiguousarray(pos[:, :2]), src, z0, precision=0,
                                src_pitch=PITCH)
    s, info, _, rc = ctx.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
    full = ctx.tmat_field(pos, 1.0, 1.0, nmax, s[0], pts)
    I_full = np.sum(np.abs(full) ** 2, axis=1)
    peak = int(np.argmax(I_full))
    sopts = _lib.make_opts(tol=1e-11, restart=200, max_iter=4000, cutoff=cut, taper=cut, precision=_lib.PREC_FP64)
    rows = []
    for buf in (0, 2, 4, 8, 16):
        sw = _lib.make_sweep(nx=n, ny=n, pitch=PITCH, core_x=20, core_y=20, buffer=buf, z0=z0)
        t0 = time.perf_counter()
        E, sinfo, src_rc = ctx.tmat_sweep(sw, at, 1.0, 1.0, nmax, src, sopts, pts)
        dt = time.perf_counter() - t0
        E = E[0]
        I = np.sum(np.abs(E) ** 2, axis=1)
        rows.append({"buffer_pitches": buf, "buffer_wavelengths": buf * PITCH,
                     "rel_field_error": float(np.linalg.norm(E - full) / np.linalg.norm(full)),
                     "peak_intensity_rel_error": float(abs(I[peak] - I_full[peak]) / I_full[peak]),
                     "seconds": dt})
    return {"workload": "padding_80x80_nmax3_cutoff6_core20_fp64", "whole_array_iterations": info.iterations,
            "rows": rows,
            "note": "16 sub-regions of 20 x 20; field on 32 detector points at height 10; the whole-array "
                    "solve (lattice path, fp64) is the reference"}


def fp64_plain_estimate(ctx, torch, step_inputs, opts_kw, krylov_iters, iters=6):
    """The plain complex128 GPU solve of the same workload, bounded: `iters` fp64 GMRES
    iterations timed, scaled to the mixed run's Krylov count (an estimate, labelled so)."""
    from paper_2107_09879_b300 import _lib
    pos, atoms, dirs, pols = step_inputs
    kw = dict(opts_kw)
    kw.update(precision=_lib.PREC_FP64, max_iter=iters)
    opts = _lib.make_opts(**kw)
    T = ctx.tmat_build(atoms, 1.0, 1.0, 4)
    a0 = ctx.tmat_incident_planewave(pos, 1.0, 1.0, 4, dirs, pols)
    ctx.tmat_solve(pos, 1.0, 1.0, 4, T, a0, opts)  # warm-up (allocates the fp64 basis)
    dt, res = _wall(lambda: ctx.tmat_solve(pos, 1.0, 1.0, 4, T, a0, opts), torch.cuda.synchronize)
    it = res[1].iterations
    per_it = dt / (it + 1)  # the cycle ends with one true-residual application
    est = per_it * (krylov_iters + 1)
    return {"ms_per_iteration": per_it * 1e3, "timed_iterations": it, "est_seconds_per_solve": est,
            "est_solves_per_s": 1.0 / est,
            "note": f"estimate: fp64 iteration time x {krylov_iters} iterations (the mixed run's Krylov count); "
                    "the fp64 solve to the same tolerance needs at least that many"}


def run_ours(args, rank, world):
    import torch
    from paper_2107_09879_b300 import _lib
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    ctx = _lib.Context(dev, None)
    ctx.set_tensor_cores(0 if args.cuda_cores else args.tc_variant)
    ctx.set_lattice_fft(not args.direct)
    wl = workload(args.size)
    w = wl["w"]
    nmax, cutoff = w["nmax"], w["cutoff"]
    N, R, P = len(wl["pos"]), 2, 48
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_pos, d_atoms, d_dirs, d_pols, d_pts = map(tt, (wl["pos"], wl["atoms"], wl["dirs"], wl["pols"], wl["pts"]))
    opts_kw = dict(tol=TOL, restart=300, max_iter=4000, cutoff=cutoff, taper=cutoff, precision=_lib.PREC_MIXED,
                   inner_tol=args.inner_tol, path=_lib.PATH_LATTICE, lattice_nx=wl["nx"], lattice_ny=wl["ny"],
                   lattice_pitch=PITCH)
    opts = _lib.make_opts(**opts_kw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    infos = []

    def step(pos, atoms, dirs, pols, pts, host=False):
        T = ctx.tmat_build(atoms, 1.0, 1.0, nmax)
        a0 = ctx.tmat_incident_planewave(pos, 1.0, 1.0, nmax, dirs, pols)
        s, info, _, rc = ctx.tmat_solve(pos, 1.0, 1.0, nmax, T, a0, opts)
        if rc != 0:
            raise RuntimeError(f"solve did not converge: {info.as_dict()}")
        E = ctx.tmat_field(pos, 1.0, 1.0, nmax, s[0], pts)
        infos.append(info)
        return s, E

    dev_in = (d_pos, d_atoms, d_dirs, d_pols, d_pts)
    for _ in range(args.warmup):
        step(*dev_in)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx.set_timing(True)
    launches0 = ctx.launches()
    infos.clear()
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()  # 256 MB write: evict L2 between steps
        evs[k][0].record(stream)
        step(*dev_in)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per_step = sorted(a.elapsed_time(b) for a, b in evs)
    total_ms = sum(per_step)
    gpu_launches = ctx.launches() - launches0
    apply_kinds = [("lattice_apply_fft32", "FFT convolution, complex64 (lattice_fft.cu)"),
                   ("lattice_apply_tcv", "lattice_tc2_kernel<4,0> (tcgen05 3xTF32, window view)"),
                   ("lattice_apply_tc", "lattice_tc_kernel<4,2,0> (tcgen05 3xTF32, gather)"),
                   ("lattice_apply_fp32", "lattice_apply_kernel<float,4,2,0> (CUDA cores)")]
    n32, ms32, kern_name = 0, 0.0, None
    for kind, name in apply_kinds:
        n32, ms32 = ctx.kernel_time(kind)
        kern_name = name
        if n32:
            break
    hbm_kinds = {"arnoldi_dots32": "dots32_kernel<true> (Arnoldi dot pass, two targets)",
                 "arnoldi_update32": "dcgs2_update_kernel (Arnoldi update pass, two outputs)",
                 "lattice_fft_mul32": "fft_mul_kernel<float,24,0,2> (block products, mirror pairs (kx, +-ky))"}
    hbm = {}
    for kind, name in hbm_kinds.items():
        nk, msk = ctx.kernel_time(kind)
        if nk:
            hbm[kind] = {"kernel": name, "launches": nk, "total_ms": msk, "bytes": ctx.kernel_bytes(kind)}
    res_kinds = [("lattice_apply_fft64", "FFT convolution, complex128 (lattice_fft.cu)"),
                 ("lattice_apply_oz", "lattice_oz_kernel<4,0> (tcgen05 bf16 slices, exact group sums, fp64-class)"),
                 ("lattice_apply_fp64", "lattice_apply_kernel<double,4,2,0> (FP64 CUDA cores)")]
    n64, ms64, res_kernel = 0, 0.0, None
    for kind, name in res_kinds:
        n64, ms64 = ctx.kernel_time(kind)
        res_kernel = name
        if n64:
            break

    ctx.set_timing(False)
    it = [i.iterations for i in infos]
    ref = [i.refinements for i in infos]
    # e2e: same step through the C ABI with pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_in = tuple(map(pin, (wl["pos"], wl["atoms"], wl["dirs"], wl["pols"], wl["pts"])))
    step(*h_in, host=True)
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s, E = step(*h_in, host=True)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(a.nbytes for a in h_in)
    d2h = R * N * P * 16 + E.nbytes
    # max over ranks
    t_local = max_over_ranks(total_ms, world, "cuda")
    value = replica_throughput(world, args.steps, t_local)
    pairs = pairs_within(wl["nx"], wl["ny"], int(round(cutoff / PITCH)))
    flop_per_launch = 8.0 * (P * P / 2) * pairs * R  # nonzero complex MACs x 8 flop, both RHS per launch
    avg32 = ms32 / max(n32, 1)
    achieved = flop_per_launch / (avg32 * 1e-3) / 1e12 if n32 else None
    matvecs = int(round(statistics.mean(it))) + int(round(statistics.mean(ref)))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 apply / f64 refinement", "data": "synthetic",
        "config": {"workload": f"lattice_{wl['nx']}x{wl['ny']}_nmax4_cutoff8_2rhs_mixed", "spheres": N, "nmax": nmax, "P": P,
                   "rhs": R, "cutoff_wavelengths": cutoff, "coupling_window": "raised cosine over [0, cutoff] (taper = cutoff)", "tol": TOL, "restart": 300, "path": "lattice (block per offset)",
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before every step"},
        "p50_ms": per_step[len(per_step) // 2], "p99_ms": per_step[min(len(per_step) - 1, int(0.99 * len(per_step)))],
        "gmres_iterations_per_solve": statistics.mean(it), "refinements_per_solve": statistics.mean(ref),
        "tmatvec_gflops": (flop_per_launch / (avg32 * 1e-3) / 1e9) if n32 else None,
        "roofline": (roofline_hbm(hbm, total_ms) if hbm else
                     roofline(kern_name, achieved, n32, avg32, flop_per_launch)),
        "hbm_kernels": {k: dict(v, achieved_gbs=v["bytes"] / (v["total_ms"] * 1e-3) / 1e9,
                                frac=v["bytes"] / (v["total_ms"] * 1e-3) / 1e9 / HBM_PEAK_GBS) for k, v in hbm.items()},
        "operator_apply": {"path": kern_name, "launches": n32, "avg_ms": avg32,
                           "direct_sum_equivalent_tflops": achieved},
        "fp64_residual_kernel": res_kernel, "fp64_residual_launches": n64,
        "fp64_residual_avg_ms": (ms64 / n64) if n64 else None,
        "e2e": {"value": world * 1e3 / statistics.median(e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
    }
    if not args.no_extras:
        out["fp64_plain"] = fp64_plain_estimate(ctx, torch, dev_in[:4], opts_kw, matvecs - int(round(statistics.mean(ref))))
        out["dense_8x8_fp64"] = bench_dense_fp64(ctx, torch)
        out["adjoint_50x50"] = bench_adjoint(ctx, torch)
        out["served"] = bench_served(args, torch)
        out["sweep_1200x1200"] = bench_sweep(ctx, torch)
        try:
            out["padding_study"] = bench_padding(ctx, torch)
        except Exception as exc:  # a study, not the headline: report it rather than lose the line
            out["padding_study"] = {"error": repr(exc)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, matvecs)
    return out


def run_kernel_only(args):
    """The dominant kernel alone, in the launch configuration the solve uses
    (complex64 lattice apply, both incidences per launch): for ncu captures and
    kernel tuning. Holds well under 1 GB on the device."""
    import torch
    from paper_2107_09879_b300 import _lib
    ctx = _lib.Context(0, None)
    ctx.set_tensor_cores(0 if args.cuda_cores else args.tc_variant)
    ctx.set_lattice_fft(not args.direct)
    wl = workload()
    w = wl["w"]
    N, P, R = len(wl["pos"]), 48, 2
    T = ctx.tmat_build(torch.from_numpy(wl["atoms"]).cuda(), 1.0, 1.0, w["nmax"])
    g = torch.Generator(device="cpu").manual_seed(0)
    x = (torch.randn(R, N, P, dtype=torch.complex128, generator=g) * 0.1).cuda()
    ctx.set_timing(True)
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            ctx.set_timing(True)
        y = ctx.tmat_apply_lattice(_lib.OP_FORWARD, args.kernel_precision, 200, 200, PITCH, w["cutoff"], 2 * math.pi,
                                   w["nmax"], T, x, taper=w["cutoff"])
    kind = {0: "lattice_apply_fp64", 1: "lattice_apply_fp32", 2: "lattice_apply_oz"}[args.kernel_precision]
    n, ms = ctx.kernel_time(kind)
    for alt in ({0: "lattice_apply_fft64", 1: "lattice_apply_fft32"}.get(args.kernel_precision, "none"),
                "lattice_apply_tcv", "lattice_apply_tc"):
        if n == 0:
            kind = alt
            n, ms = ctx.kernel_time(kind)
    pairs = pairs_within(200, 200, int(round(w["cutoff"] / PITCH)))
    flop = 8.0 * (P * P / 2) * pairs * R
    return {"kernel": kind, "launches": n, "avg_ms": ms / max(n, 1), "tflops": flop / (ms / max(n, 1) * 1e-3) / 1e12,
            "flop_per_launch": flop, "y_norm": float(torch.linalg.vector_norm(y).item())}


def run_jinc_only(args):
    """Incident coefficients of one jinc group in the 1200 x 1200 sweep's sub-region shape
    (76 x 76 spheres = 60 x 60 core + 8-pitch ring, sources on the core, nmax 3, 4 RHS,
    source plane z0 = -1), complex64 and fp64 paths: per-kernel CUDA-event times and the
    relative difference of the two results (for kernel tuning and ncu captures)."""
    import torch
    from paper_2107_09879_b300 import _lib
    ctx = _lib.Context(0, None)
    side, core, ring, nmax, R = 76, 60, 8, 3, 4
    pos = W.lattice_positions(side, side)
    src = W.lattice_positions(core, core)[:, :2] + ring * PITCH
    A = np.zeros((R, core * core, 2), complex)
    for q, deg in enumerate((0.0, 5.0, 10.0, 15.0)):
        th = math.radians(deg)
        A[q, :, 0] = math.cos(th) * np.exp(1j * 2 * math.pi * (math.sin(th) * src[:, 0] - math.cos(th)))
    out, res = {}, {}
    kinds = ("jinc_nodes", "jinc_phase32", "jinc_gemm32", "jinc_accum64")
    for prec in (1, 0):
        for k in range(args.warmup + args.steps):
            if k == args.warmup:
                ctx.set_timing(True)
            a = ctx.tmat_incident_jinc(pos, 1.0, 1.0, nmax, src, A, -1.0, precision=prec, src_pitch=PITCH)
        torch.cuda.synchronize()
        t = {kk: ctx.kernel_time(kk) for kk in kinds}
        ctx.set_timing(False)
        res[prec] = a
        out["complex64" if prec == 1 else "fp64"] = {kk: v[1] / max(args.steps, 1) for kk, v in t.items() if v[0]}
    out["workload"] = "jinc_group_76x76_core60_nmax3_4rhs"
    out["unit"] = "ms per call"
    out["rel_l2_c64_vs_fp64"] = float(np.linalg.norm(res[1] - res[0]) / np.linalg.norm(res[0]))
    return out


def run_reference(args, rank, world):
    """The reference arm: the oracle (plain fp64 CPU), timed on the host cores."""
    if rank != 0:
        return None
    wl = workload()
    per = []
    base = None
    for k in range(args.warmup + args.steps):
        base = cpu_baseline(wl, matvecs_per_solve=args.ref_matvecs, budget_s=3.0)
        if k >= args.warmup:
            per.append(1.0 / base["value"])
    value = 1.0 / statistics.mean(per)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(per) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lattice_200x200_nmax4_cutoff8_2rhs_mixed", "spheres": 40000},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (fp64 plain estimate, 8x8 fp64, adjoint, served stream, sweep)")
    ap.add_argument("--served-requests", type=int, default=48, help="requests in the 1.5x-rate served stream")
    ap.add_argument("--ref-matvecs", type=int, default=276, help="operator applications per solve for the oracle arm")
    ap.add_argument("--kernel-only", action="store_true", help="time the dominant kernel alone (for ncu captures)")
    ap.add_argument("--kernel-precision", type=int, default=1, help="1: complex64 apply, 0: complex128 apply, 2: fp64-class tensor-core apply")
    ap.add_argument("--cuda-cores", action="store_true", help="complex64 apply on CUDA cores instead of tcgen05")
    ap.add_argument("--size", type=int, default=200,
                    help="lattice side (200: the benchmark; smaller: its corner, for profiler captures)")
    ap.add_argument("--direct", action="store_true",
                    help="lattice operator by the direct block-Toeplitz kernels instead of FFT convolution")
    ap.add_argument("--tc-variant", type=int, default=1, choices=[1, 2],
                    help="tensor-core lattice kernel: 1 window view (default), 2 gather")
    ap.add_argument("--jinc-only", action="store_true",
                    help="time one jinc group of the sweep's sub-region shape (complex64 and fp64 paths)")
    ap.add_argument("--inner-tol", type=float, default=0.2,
                    help="relative tolerance of each complex64 inner solve of the refinement (0.2: short inner "
                         "solves; the Krylov count stays ~260 while the orthogonalisation work shrinks with "
                         "the square of the inner length)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.kernel_only:
        print(json.dumps(run_kernel_only(args)))
        return
    if args.jinc_only:
        print(json.dumps(run_jinc_only(args)))
        return
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        out = run_reference(args, rank, world)
        print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
