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
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock


def workload():
    w = W.lattice_200x200()
    nx = ny = 200
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
    out = {"kernel": kern_name, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": (achieved / peak) if achieved else None, "traffic": None, "launches": launches,
           "avg_launch_ms": avg_ms, "flop_per_launch": flop_per_launch, "peak_note": note}
    out.update(extra)
    return out


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


def run_ours(args, rank, world):
    import torch
    from paper_2107_09879_b300 import _lib
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    ctx = _lib.Context(dev, None)
    ctx.set_tensor_cores(0 if args.cuda_cores else args.tc_variant)
    wl = workload()
    w = wl["w"]
    nmax, cutoff = w["nmax"], w["cutoff"]
    N, R, P = len(wl["pos"]), 2, 48
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_pos, d_atoms, d_dirs, d_pols, d_pts = map(tt, (wl["pos"], wl["atoms"], wl["dirs"], wl["pols"], wl["pts"]))
    opts = _lib.make_opts(tol=1e-6, restart=300, max_iter=4000, cutoff=cutoff, taper=cutoff, precision=_lib.PREC_MIXED,
                          inner_tol=1e-4, path=_lib.PATH_LATTICE, lattice_nx=wl["nx"], lattice_ny=wl["ny"],
                          lattice_pitch=PITCH)
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
    n32, ms32 = ctx.kernel_time("lattice_apply_tcv")
    kern_name = "lattice_tc2_kernel<4,0> (tcgen05 3xTF32, window view)"
    if n32 == 0:
        n32, ms32 = ctx.kernel_time("lattice_apply_tc")
        kern_name = "lattice_tc_kernel<4,2,0> (tcgen05 3xTF32, gather)"
    if n32 == 0:
        n32, ms32 = ctx.kernel_time("lattice_apply_fp32")
        kern_name = "lattice_apply_kernel<float,4,2,0> (CUDA cores)"
    n64, ms64 = ctx.kernel_time("lattice_apply_fp64")
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
    t_local = total_ms
    if world > 1:
        t = torch.tensor([t_local], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_local = float(t.item())
    value = world * args.steps / (t_local / 1e3)
    pairs = pairs_within(200, 200, int(round(cutoff / PITCH)))
    flop_per_launch = 8.0 * (P * P / 2) * pairs * R  # nonzero complex MACs x 8 flop, both RHS per launch
    avg32 = ms32 / max(n32, 1)
    achieved = flop_per_launch / (avg32 * 1e-3) / 1e12 if n32 else None
    matvecs = int(round(statistics.mean(it))) + int(round(statistics.mean(ref)))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 apply / f64 refinement", "data": "synthetic",
        "config": {"workload": "lattice_200x200_nmax4_cutoff8_2rhs_mixed", "spheres": N, "nmax": nmax, "P": P,
                   "rhs": R, "cutoff_wavelengths": cutoff, "coupling_window": "raised cosine over [0, cutoff] (taper = cutoff)", "tol": 1e-6, "restart": 300, "path": "lattice (block per offset)",
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before every step"},
        "p50_ms": per_step[len(per_step) // 2], "p99_ms": per_step[min(len(per_step) - 1, int(0.99 * len(per_step)))],
        "gmres_iterations_per_solve": statistics.mean(it), "refinements_per_solve": statistics.mean(ref),
        "tmatvec_gflops": (flop_per_launch / (avg32 * 1e-3) / 1e9) if n32 else None,
        "roofline": roofline(kern_name, achieved, n32, avg32, flop_per_launch),
        "fp64_residual_launches": n64, "fp64_residual_avg_ms": (ms64 / n64) if n64 else None,
        "e2e": {"value": world * 1e3 / statistics.median(e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
    }
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
    kind = "lattice_apply_fp32" if args.kernel_precision == _lib.PREC_MIXED else "lattice_apply_fp64"
    n, ms = ctx.kernel_time(kind)
    for alt in ("lattice_apply_tcv", "lattice_apply_tc"):
        if args.kernel_precision == _lib.PREC_MIXED and n == 0:
            kind = alt
            n, ms = ctx.kernel_time(kind)
    pairs = pairs_within(200, 200, int(round(w["cutoff"] / PITCH)))
    flop = 8.0 * (P * P / 2) * pairs * R
    return {"kernel": kind, "launches": n, "avg_ms": ms / max(n, 1), "tflops": flop / (ms / max(n, 1) * 1e-3) / 1e12,
            "flop_per_launch": flop, "y_norm": float(torch.linalg.vector_norm(y).item())}


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
    ap.add_argument("--ref-matvecs", type=int, default=276, help="operator applications per solve for the oracle arm")
    ap.add_argument("--kernel-only", action="store_true", help="time the dominant kernel alone (for ncu captures)")
    ap.add_argument("--kernel-precision", type=int, default=1, help="1: complex64 apply, 0: complex128 apply")
    ap.add_argument("--cuda-cores", action="store_true", help="complex64 apply on CUDA cores instead of tcgen05")
    ap.add_argument("--tc-variant", type=int, default=1, choices=[1, 2],
                    help="tensor-core lattice kernel: 1 window view (default), 2 gather")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.kernel_only:
        print(json.dumps(run_kernel_only(args)))
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
