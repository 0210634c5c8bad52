"""Request loop for sub-region solves on one GPU (the paper's sub-region jobs, main text
"Low-overhead multi-GPU simulation strategy", run as a served stream).

A request is one sub-region: a k x k core of jinc sources (App. II) sampling a normally
incident x-polarised plane wave, the core plus a padding ring of spheres, its own
wavelength and nmax.

Continuous batching: whenever a slot is free the loop forms a batch from the requests that
have arrived (oldest first; up to `max_batch` requests of the same nmax and canvas class),
admits it if its device memory fits, and solves it with one tmat_solve_batch call on the
slot's own library context and CUDA stream: the requests of a batch share every kernel
launch (FFT applies with their own block spectra, Arnoldi and Givens passes), their Krylov
bases stay resident on the device through all refinement steps, and batches on different
slots overlap on the GPU. Requests that arrive while batches run wait only for the next free
slot. A request's canvas (the lattice its problem is placed on) depends only on its own size
class, so its result does not depend on what it was batched with (to rounding in fp64,
within the solve tolerance in mixed precision).

Admission is by device memory: a batch's estimate (request_bytes) must fit both the
configured budget and the free memory the driver reports (cudaMemGetInfo through torch),
and the contexts' own scratch (tmat_ctx_memory, what the library really holds) is sampled
after every batch and reported beside the estimate.

Everything numeric runs in the native library (libtmat.so) through `_lib`.
"""
import collections
import concurrent.futures as cf
import math
import threading
import time

import numpy as np

from . import _lib

CANVAS_CLASSES = (24, 32, 48, 68)  # canvas side of a request: the smallest class >= its side


def canvas_of(side):
    for c in CANVAS_CLASSES:
        if side <= c:
            return c
    return side


def request_bytes(side, nmax, R=1, restart=60, cutoff_sites=16):
    """Device-memory estimate of one request on its canvas (Krylov basis, vectors, blocks,
    the FFT operator's block spectra and work grids, jinc staging)."""
    c = canvas_of(side)
    N = c * c
    P = 2 * nmax * (nmax + 2)
    L = P // 2
    krylov = (restart + 1) * R * N * P * 8
    vectors = 14 * R * N * P * 16
    blocks = 800 * 2 * L ** 2 * (16 + 8 + 2 * 8)
    M = 1
    while M < c + cutoff_sites:
        M *= 2
    spectra = 2 * L * L * M * M * (16 * 2 + 8 * 2)  # complex128 + complex64 spectra, batch copies
    work = R * P * M * M * (16 * 3 + 8 * 3)
    jinc = 8192 * R * P * 16
    return krylov + vectors + blocks + spectra + work + jinc + (8 << 20)


def _canvas(req):
    """Canvas side of a request: its size class (sub-region sweeps: their own side)."""
    if "sweep" in req:
        return max(req["w"], req["h"])
    return canvas_of(req["side"])


def sweep_requests(nx, ny, core, buf, pitch, radius, n_sphere, src_A, z0, pts, nmax):
    """One request per sub-region of an nx x ny sweep (cores of core x core sites, rings of buf
    sites, clipped at the edge): src_A (R, nx * ny, 2) transverse amplitudes of the jinc source
    at every site, detectors pts (M, 3) in the sweep's coordinates. All arrive at t = 0."""
    g = dict(nx=nx, ny=ny, pitch=pitch, radius=np.asarray(radius), n_sphere=n_sphere, src_A=np.asarray(src_A),
             z0=z0, pts=np.asarray(pts, dtype=np.float64))
    out = []
    nax, nay = -(-nx // core), -(-ny // core)
    for a in range(nax * nay):
        ax, ay = a % nax, a // nax
        cx0, cy0 = ax * core, ay * core
        cx1, cy1 = min(nx, cx0 + core), min(ny, cy0 + core)
        px0, py0 = max(0, cx0 - buf), max(0, cy0 - buf)
        px1, py1 = min(nx, cx1 + buf), min(ny, cy1 + buf)
        out.append(dict(rid=a, arrival=0.0, nmax=nmax, sweep=g, cx0=cx0, cy0=cy0, cw=cx1 - cx0, ch=cy1 - cy0,
                        px0=px0, py0=py0, w=px1 - px0, h=py1 - py0, side=max(px1 - px0, py1 - py0),
                        wavelength=1.0))
    return out


def sweep_field(records, R, M):
    """The decomposed field of the whole array: the sub-regions' fields added in sub-region
    order (deterministic), fp64 on the host."""
    E = np.zeros((R, M, 3), dtype=np.complex128)
    for rec in sorted(records, key=lambda r: r["rid"]):
        E += rec["E"]
    return E


def ct_stream(torch_stream):
    return torch_stream.cuda_stream


def _device_free_bytes(device):
    import torch
    free, _ = torch.cuda.mem_get_info(device)
    return free


class Server:
    def __init__(self, slots=4, mem_budget=8 << 30, device=0, tol=1e-7, cutoff=8.0, restart=60, z0=-1.0,
                 detector_height=5.0, inner_tol=1e-4, max_batch=8, reserve_bytes=2 << 30):
        import torch
        self.slots, self.mem_budget, self.device = slots, mem_budget, device
        self.tol, self.cutoff, self.restart, self.z0, self.det_h = tol, cutoff, restart, z0, detector_height
        self.inner_tol, self.max_batch, self.reserve = inner_tol, max_batch, reserve_bytes
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.ctxs = [_lib.Context(device, ct_stream(s)) for s in self.streams]
        self.pool = [cf.ThreadPoolExecutor(max_workers=1) for _ in range(slots)]
        self.lock = threading.Condition()
        self.free = collections.deque(range(slots))
        self.mem_in_use = 0
        self.mem_high = 0           # largest sum of the estimates of the batches in flight
        self.ctx_mem_high = 0       # largest measured scratch held by the contexts
        self.batches = []           # sizes of the batches run
        self.slot_mem = [0] * slots  # scratch each slot's context held after its last batch

    def close(self):
        for p in self.pool:
            p.shutdown(wait=True)
        for c in self.ctxs:
            c.close()

    # ---- one batch, on its slot's context ------------------------------------------
    def _problem(self, ctx, req):
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
        A = np.zeros((1, k * k, 2), complex)
        A[0, :, 0] = np.exp(1j * (2 * math.pi / w) * self.z0)  # x-polarised plane wave at normal incidence, z = z0
        T = ctx.tmat_build(atoms, w, 1.0, nmax)
        a0 = ctx.tmat_incident_jinc(pos, w, 1.0, nmax, src, A, self.z0, precision=_lib.PREC_MIXED, src_pitch=pitch)
        return dict(nx=side, ny=side, wavelength=w, T=T, a0=np.ascontiguousarray(a0[0]), pos=pos)

    def _sweep_problems(self, ctx, req):
        """A sub-region of a large-area sweep (main text, Fig. 3): its spheres (core + ring) on
        a lattice at the origin, the jinc sources of its core shifted by the same offset (the
        problem is translation invariant), one problem per incidence."""
        g = req["sweep"]
        pitch, nx = g["pitch"], g["nx"]
        px0, py0, w, h = req["px0"], req["py0"], req["w"], req["h"]
        iy, ix = np.divmod(np.arange(w * h), w)
        pos = np.zeros((w * h, 3))
        pos[:, 0], pos[:, 1] = ix * pitch, iy * pitch
        sites = (py0 + iy) * nx + px0 + ix
        atoms = np.stack([g["radius"][sites], np.full(w * h, g["n_sphere"]), np.zeros(w * h)], axis=1)
        cy, cx = np.divmod(np.arange(req["cw"] * req["ch"]), req["cw"])
        csites = (req["cy0"] + cy) * nx + req["cx0"] + cx
        src = np.stack([(req["cx0"] - px0 + cx) * pitch, (req["cy0"] - py0 + cy) * pitch], axis=1)
        A = np.ascontiguousarray(g["src_A"][:, csites, :])
        T = ctx.tmat_build(atoms, 1.0, 1.0, req["nmax"])
        a0 = ctx.tmat_incident_jinc(pos, 1.0, 1.0, req["nmax"], src, A, g["z0"], precision=_lib.PREC_MIXED,
                                    src_pitch=pitch)
        return [dict(nx=w, ny=h, wavelength=1.0, T=T, a0=np.ascontiguousarray(a0[r]), pos=pos)
                for r in range(A.shape[0])]

    def _solve_batch(self, slot, reqs):
        ctx = self.ctxs[slot]
        nmax = reqs[0]["nmax"]
        canvas = max(_canvas(r) for r in reqs)
        per_req = [self._sweep_problems(ctx, r) if "sweep" in r else [self._problem(ctx, r)] for r in reqs]
        probs = [p for pr in per_req for p in pr]
        opts = _lib.make_opts(tol=self.tol, restart=self.restart, max_iter=3000, cutoff=self.cutoff,
                              taper=self.cutoff, precision=_lib.PREC_MIXED, inner_tol=self.inner_tol)
        outs, infos, rc = ctx.tmat_solve_batch(probs, 1.0, nmax, 0.5, opts, canvas=(canvas, canvas))
        res, q = [], 0
        for req, pr in zip(reqs, per_req):
            if "sweep" in req:  # field of every incidence at the sweep's detectors (shifted)
                shift = np.array([req["px0"] * req["sweep"]["pitch"], req["py0"] * req["sweep"]["pitch"], 0.0])
                pts = np.ascontiguousarray(req["sweep"]["pts"] - shift)
                E = np.stack([ctx.tmat_field(p["pos"], 1.0, 1.0, nmax, outs[q + i], pts) for i, p in enumerate(pr)])
                s = None
            else:
                p = pr[0]
                c = (p["nx"] - 1) * 0.5 / 2
                s = outs[q]
                E = ctx.tmat_field(p["pos"], p["wavelength"], 1.0, nmax, s, np.array([[c, c, self.det_h]]))
            res.append((s, E, infos[q]))
            q += len(pr)
        return res, rc, ctx.memory()

    # ---- batch formation -----------------------------------------------------------
    def _problems_of(self, r):
        return r["sweep"]["src_A"].shape[0] if "sweep" in r else 1

    def _take_batch(self, ready):
        """The oldest ready request and up to max_batch - 1 more of the same nmax and canvas
        class, as many as the memory budget left over by the running batches allows (at least
        the oldest one)."""
        head = ready[0]
        key = (head["nmax"], _canvas(head))
        room = min(self.mem_budget - self.mem_in_use, _device_free_bytes(self.device) - self.reserve)
        batch, est, nprob = [], 0, 0
        for r in ready:
            if (r["nmax"], _canvas(r)) != key:
                continue
            e = request_bytes(_canvas(r), r["nmax"], R=self._problems_of(r), restart=self.restart)
            k = self._problems_of(r)
            if batch and (est + e > room or len(batch) >= self.max_batch or nprob + k > _lib.MAX_RHS):
                break
            batch.append(r)
            est += e
            nprob += k
        return batch, est

    # ---- the loop ------------------------------------------------------------------
    def run(self, requests, keep_solutions=False):
        """Release each request at its arrival time (seconds after the start), batch and admit
        by slot and device memory, and return per-request records."""
        t0 = time.perf_counter()
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
        ready = []
        records = {}
        running = 0

        def done(slot, reqs, est, fut):
            nonlocal running
            t = time.perf_counter() - t0
            with self.lock:
                try:
                    res, rc, ctx_mem = fut.result()
                    # each context is read only by its own slot's thread (contexts are not
                    # thread-safe): the slot reports its scratch with the batch's results
                    self.slot_mem[slot] = ctx_mem
                    self.ctx_mem_high = max(self.ctx_mem_high, sum(self.slot_mem))
                    for req, (s, E, info) in zip(reqs, res):
                        rec = records[req["rid"]]
                        rec.update(finish=t, E=E, iterations=info.iterations, refinements=info.refinements,
                                   residual=info.rel_residual[0], rc=0 if info.converged else _lib.ENOCONV)
                        if keep_solutions:
                            rec["s"] = s
                except Exception as e:  # recorded, not raised: one failed batch does not stop the loop
                    for req in reqs:
                        records[req["rid"]].update(finish=t, error=repr(e))
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
                    batch, est = self._take_batch(ready)
                    fits = (self.mem_in_use + est <= self.mem_budget and
                            est + self.reserve <= _device_free_bytes(self.device))
                    if not fits and running > 0:
                        break  # wait for memory to free up
                    for r in batch:
                        ready.remove(r)
                    slot = self.free.popleft()
                    self.mem_in_use += est
                    self.mem_high = max(self.mem_high, self.mem_in_use)
                    self.batches.append(len(batch))
                    running += 1
                    for r in batch:
                        records[r["rid"]] = dict(rid=r["rid"], arrival=r["arrival"], admit=now, slot=slot,
                                                 side=r["side"], nmax=r["nmax"], wavelength=r["wavelength"],
                                                 batch=len(batch))
                    fut = self.pool[slot].submit(self._solve_batch, slot, batch)
                    fut.add_done_callback(lambda f, s=slot, b=batch, e=est: done(s, b, e, f))
                wait = 0.02
                if pending:
                    wait = max(0.0, min(wait, pending[0]["arrival"] - (time.perf_counter() - t0)))
                if pending or ready or running:
                    self.lock.wait(timeout=wait)
        return [records[k] for k in sorted(records)]


def summarize(records, wall_s):
    lat = sorted(r["finish"] - r["arrival"] for r in records if "finish" in r)
    q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
    return {"requests": len(records), "completed": sum(1 for r in records if "E" in r),
            "errors": sum(1 for r in records if "error" in r),
            "solves_per_s": len(lat) / wall_s if wall_s > 0 else None,
            "p50_latency_s": q(0.50), "p99_latency_s": q(0.99), "wall_s": wall_s,
            "mean_batch": (sum(r.get("batch", 1) for r in records) / len(records)) if records else None}
