"""Integer geometry of the method.

* Interaction neighbour lists: all sources j != i with |x_i - x_j| <= cutoff
  (inclusive). The paper couples every pair (App. I-D); the cutoff is a
  parameter of this implementation (cutoff <= 0 means every pair). The test is
  done in fp64 exactly as written: d2 = dx*dx + dy*dy + dz*dz (left to right,
  each product rounded), compared with cutoff*cutoff.
* Sub-region index sets (main text, "Low-overhead multi-GPU simulation
  strategy"; Fig. 3 caption): on an nx x ny lattice (site index iy*nx + ix),
  sub-region (ax, ay) has core sites ix in [ax*cx, (ax+1)*cx), iy likewise
  (clipped to the lattice), and its simulated set is the core plus a padding
  ring of `buf` sites on every side, clipped to the lattice.
"""
import numpy as np


def neighbours(pos, cutoff):
    """CSR (row_ptr int64 (N+1,), col int32) of sources per target, ascending."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    rows = []
    c2 = float(cutoff) * float(cutoff)
    for i in range(N):
        dx = pos[i, 0] - pos[:, 0]
        dy = pos[i, 1] - pos[:, 1]
        dz = pos[i, 2] - pos[:, 2]
        d2 = dx * dx + dy * dy
        d2 = d2 + dz * dz
        if cutoff > 0:
            ok = d2 <= c2
        else:
            ok = np.ones(N, dtype=bool)
        ok[i] = False
        rows.append(np.nonzero(ok)[0].astype(np.int32))
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows) if N else np.zeros(0, dtype=np.int32)
    return row_ptr, col.astype(np.int32)


def subregion_sets(nx, ny, cx, cy, buf):
    """List over sub-regions (row-major in (ay, ax)) of (core_idx, sim_idx),
    both int64 ascending site indices."""
    out = []
    nax = -(-nx // cx)
    nay = -(-ny // cy)
    for ay in range(nay):
        for ax in range(nax):
            x0, x1 = ax * cx, min((ax + 1) * cx, nx)
            y0, y1 = ay * cy, min((ay + 1) * cy, ny)
            core = [iy * nx + ix for iy in range(y0, y1) for ix in range(x0, x1)]
            px0, px1 = max(0, x0 - buf), min(nx, x1 + buf)
            py0, py1 = max(0, y0 - buf), min(ny, y1 + buf)
            sim = [iy * nx + ix for iy in range(py0, py1) for ix in range(px0, px1)]
            out.append((np.array(core, dtype=np.int64), np.array(sim, dtype=np.int64)))
    return out


def first_overlap(pos, radii):
    """The enclosing-sphere condition of App. I-C (the method assumes no two enclosing
    spheres intersect): the first pair (i < j, smallest i, then j) with
    d2 < (r_i + r_j)^2, d2 = dx*dx + dy*dy + dz*dz evaluated left to right, or None.
    Brute force over all pairs."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    for i in range(n):
        for j in range(i + 1, n):
            d = pos[i] - pos[j]
            d2 = float(d[0]) * float(d[0]) + float(d[1]) * float(d[1])
            d2 = d2 + float(d[2]) * float(d[2])
            s = float(radii[i]) + float(radii[j])
            if d2 < s * s:
                return i, j
    return None
