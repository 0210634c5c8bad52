"""Request loop for sub-region solves on one GPU (the paper's sub-region jobs,
main text "Low-overhead multi-GPU simulation strategy", run as a served stream).

A request is one sub-region: a k x k core of jinc sources (App. II) sampling a
normally incident x-polarised plane wave, the core plus a padding ring of
spheres, its own wavelength and nmax. The loop admits requests in arrival order
when a slot is free and the request's device-memory estimate fits the budget;
every slot owns a library context bound to its own CUDA stream, so admitted
requests run concurrently and their kernels overlap on the device. Each request
is solved by the same deterministic kernels whatever else runs, so its result
does not depend on the mix.

Everything numeric runs in the native library (libtmat.so) through `_lib`.
"""
import collections
import concurrent.futures as cf
import math
import threading
import time

import numpy as np

from . import _lib


def request_bytes(side, nmax, R=1, restart=60, cutoff_sites=16):
    """Device-memory estimate of one request (Krylov basis, vectors, blocks, the FFT
    operator's block spectra and work grids, tables)."""
    N = side * side
    P = 2 * nmax * (nmax + 2)
    L = P // 2
    krylov = (restart + 1) * R * N * P * 8
    vectors = 14 * R * N * P * 16
    blocks = 800 * 2 * L ** 2 * (16 + 8 + 2 * 8)
    M = 1
    while M < side + cutoff_sites:
        M *= 2
    spectra = 2 * L * L * M * M * (16 * 3 + 8)  # complex128 spectra + 2 staging grids, complex64 spectra
    work = R * P * M * M * (16 * 3 + 8 * 3)
    jinc = 8192 * R * P * 16
    return krylov + vectors + blocks + spectra + work + jinc + (8 << 20)


class Server:
    def __init__(self, slots=4, mem_budget=8 << 30, device=0, tol=1e-7, cutoff=8.0, restart=60, z0=-1.0,
                 detector_height=5.0, inner_tol=1e-4):
        import torch
        self.slots = slots
        self.mem_budget = mem_budget
        self.tol, self.cutoff, self.restart, self.z0, self.det_h = tol, cutoff, restart, z0, detector_height
        self.inner_tol = inner_tol
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.ctxs = [_lib.Context(device, ct_stream(s)) for s in self.streams]
        self.pool = [cf.ThreadPoolExecutor(max_workers=1) for _ in range(slots)]
        self.lock = threading.Condition()
        self.free = collections.deque(range(slots))
        self.mem_in_use = 0
        self.mem_high = 0

    def close(self):
        for p in self.pool:
            p.shutdown(wait=True)
        for c in self.ctxs:
            c.close()

    # ---- one request, on its slot's context -------------------------------------
    def _solve(self, slot, req):
        ctx = self.ctxs[slot]
        side, k, b, nmax, w = req["side"], req["k"], req["buf"], req["nmax"], req["wavelength"]
        pitch = 0.5
        n = side * side
        iy, ix = np.divmod(np.arange(n), side)
        pos = np.zeros((n, 3))
        pos[:, 0] = ix * pitch
        pos[:, 1] = iy * pitch
        atoms = np.stack([req["radii"], np.full(n, 2.0), np.zeros(n)], axis=1)
        cy, cx = np.divmod(np.arange(k * k), k)
        src = np.stack([(cx + b) * pitch, (cy + b) * pitch], axis=1)
        kk = 2 * math.pi / w
        A = np.zeros((1, k * k, 2), complex)
        A[0, :, 0] = np.exp(1j * kk * self.z0)  # normally incident x-polarised plane wave at z = z0
        T = ctx.tmat_build(atoms, w, 1.0, nmax)
        a0 = ctx.tmat_incident_jinc(pos, w, 1.0, nmax, src, A, self.z0, precision=_lib.PREC_MIXED, src_pitch=pitch)
        opts = _lib.make_opts(tol=self.tol, restart=self.restart, max_iter=3000, cutoff=self.cutoff,
                              taper=self.cutoff, precision=_lib.PREC_MIXED, inner_tol=self.inner_tol, path=_lib.PATH_LATTICE,
                              lattice_nx=side, lattice_ny=side, lattice_pitch=pitch)
        s, info, _, rc = ctx.tmat_solve(pos, w, 1.0, nmax, T, a0, opts)
        c = (side - 1) * pitch / 2
        det = np.array([[c, c, self.det_h]])
        E = ctx.tmat_field(pos, w, 1.0, nmax, s[0], det)
        return s, E, info, rc

    # ---- the loop ----------------------------------------------------------------
    def run(self, requests, keep_solutions=False):
        """Release each request at its arrival time (seconds after the start), admit
        by slot and memory, and return per-request records."""
        t0 = time.perf_counter()
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
        ready = collections.deque()
        records = {}
        running = 0

        def done(slot, req, est, fut):
            nonlocal running
            t = time.perf_counter() - t0
            with self.lock:
                rec = records[req["rid"]]
                rec["finish"] = t
                try:
                    s, E, info, rc = fut.result()
                    rec.update(E=E, iterations=info.iterations, refinements=info.refinements,
                               residual=max(info.rel_residual[:1]), rc=rc)
                    if keep_solutions:
                        rec["s"] = s
                except Exception as e:  # recorded, not raised: one failed job does not stop the loop
                    rec["error"] = repr(e)
                self.mem_in_use -= est
                self.free.append(slot)
                running -= 1
                self.lock.notify_all()

        with self.lock:
            while pending or ready or running:
                now = time.perf_counter() - t0
                while pending and pending[0]["arrival"] <= now:
                    ready.append(pending.popleft())
                while ready and self.free:
                    req = ready[0]
                    est = request_bytes(req["side"], req["nmax"], restart=self.restart)
                    if self.mem_in_use + est > self.mem_budget and running > 0:
                        break  # wait for memory to free up
                    ready.popleft()
                    slot = self.free.popleft()
                    self.mem_in_use += est
                    self.mem_high = max(self.mem_high, self.mem_in_use)
                    running += 1
                    records[req["rid"]] = dict(rid=req["rid"], arrival=req["arrival"], admit=now, slot=slot,
                                               side=req["side"], nmax=req["nmax"], wavelength=req["wavelength"])
                    fut = self.pool[slot].submit(self._solve, slot, req)
                    fut.add_done_callback(lambda f, s=slot, r=req, e=est: done(s, r, e, f))
                wait = 0.05
                if pending:
                    wait = max(0.0, min(wait, pending[0]["arrival"] - (time.perf_counter() - t0)))
                if pending or ready or running:
                    self.lock.wait(timeout=wait)
        return [records[k] for k in sorted(records)]


def ct_stream(torch_stream):
    return torch_stream.cuda_stream


def summarize(records, wall_s):
    lat = sorted(r["finish"] - r["arrival"] for r in records if "finish" in r)
    q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
    return {"requests": len(records), "completed": sum(1 for r in records if "E" in r),
            "errors": sum(1 for r in records if "error" in r),
            "solves_per_s": len(lat) / wall_s if wall_s > 0 else None,
            "p50_latency_s": q(0.50), "p99_latency_s": q(0.99), "wall_s": wall_s}
