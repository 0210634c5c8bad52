"""Seeded synthetic inputs shaped like the paper's metasurfaces.

This module holds no arithmetic of the method: it only draws positions, radii,
indices and request streams. Both the CUDA path and the CPU oracle are fed from
here. Random numbers come from splitmix64 (Steele, Lea & Flood 2014):
    x += 0x9E3779B97F4A7C15; z = x; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; return z ^ (z >> 31)
and a uniform double is u = (z >> 11) * 2^-53.

Lattice conventions: wavelength 1 (scaled units), sites (ix * pitch, iy * pitch, 0)
in row-major order (site index iy * nx + ix); radii are drawn in that order.
"""
import math

import numpy as np

MASK = (1 << 64) - 1
BASE_SEED = 210709879


class SplitMix64:
    def __init__(self, seed):
        self.state = seed & MASK

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self):
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def uniforms(self, n):
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)


def lattice_positions(nx, ny, pitch=0.5, origin=(0.0, 0.0)):
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.zeros((nx * ny, 3), dtype=np.float64)
    pos[:, 0] = origin[0] + ix.reshape(-1) * pitch
    pos[:, 1] = origin[1] + iy.reshape(-1) * pitch
    return pos


def uniform_radii(n, lo, hi, seed):
    g = SplitMix64(seed)
    return lo + (hi - lo) * g.uniforms(n)


# ----------------------------------------------------------------------------
# Named workloads (sizes of the sphere-array configurations).
# ----------------------------------------------------------------------------

def dense_8x8():
    """8x8 lattice, 64 identical spheres r = 0.2, index 2.0, pitch 0.5,
    nmax = 3, every pair coupled, normal-incidence x-polarised plane wave."""
    pos = lattice_positions(8, 8)
    return dict(name="dense_8x8_nmax3", pos=pos, radius=np.full(64, 0.2), n_sphere=2.0,
                nmax=3, cutoff=0.0, angles_deg=[0.0], wavelength=1.0, tol=1e-10)


def lattice_200x200(seed_offset=2):
    """200x200 lattice (40,000 spheres), radii U[0.08, 0.24], index 2.0,
    nmax = 4, cutoff 8 wavelengths, plane waves at 0 and 10 degrees."""
    pos = lattice_positions(200, 200)
    r = uniform_radii(40000, 0.08, 0.24, BASE_SEED + seed_offset)
    return dict(name="lattice_200x200_nmax4_c8", pos=pos, radius=r, n_sphere=2.0,
                nmax=4, cutoff=8.0, angles_deg=[0.0, 10.0], wavelength=1.0, tol=1e-6)


def lattice_50x50_adjoint(seed_offset=4):
    """50x50 lattice (2,500 spheres), radii U[0.1, 0.22], index 2.0, nmax = 4,
    cutoff 10 wavelengths, focal point 20 wavelengths above the centre."""
    pos = lattice_positions(50, 50)
    r = uniform_radii(2500, 0.1, 0.22, BASE_SEED + seed_offset)
    return dict(name="lattice_50x50_nmax4_c10_adjoint", pos=pos, radius=r, n_sphere=2.0,
                nmax=4, cutoff=10.0, angles_deg=[0.0], wavelength=1.0,
                focus=np.array([12.25, 12.25, 20.0]))


def small_lattice(nx, ny, nmax, cutoff, seed, lo=0.08, hi=0.24, pitch=0.5):
    pos = lattice_positions(nx, ny, pitch)
    r = uniform_radii(nx * ny, lo, hi, seed)
    return dict(name=f"lattice_{nx}x{ny}_nmax{nmax}", pos=pos, radius=r, n_sphere=2.0,
                nmax=nmax, cutoff=cutoff, angles_deg=[0.0], wavelength=1.0)


def random_positions(n, box, min_sep, seed):
    """n points in [0, box]^2 x {0} with pairwise separation >= min_sep
    (dart throwing with a splitmix64 stream)."""
    g = SplitMix64(seed)
    pts = []
    tries = 0
    while len(pts) < n and tries < 100000:
        tries += 1
        p = np.array([g.uniform() * box, g.uniform() * box, 0.0])
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def jittered_lattice(nx, ny, jitter, seed, pitch=0.5):
    """A disordered array: the nx x ny lattice sites, each displaced in x and y by
    U[-jitter, jitter] (splitmix64 stream, x then y per site), z = 0."""
    g = SplitMix64(seed)
    pos = lattice_positions(nx, ny, pitch)
    u = g.uniforms(2 * nx * ny).reshape(nx * ny, 2)
    pos[:, :2] += jitter * (2.0 * u - 1.0)
    return pos


def smooth_radius_map(nx, ny, seed, pitch=0.5):
    """Seeded smoothly varying radius map in [0.08, 0.24] plus U[-0.01, 0.01]
    noise: r = 0.16 + 0.065 sin(2 pi x/97 + p1) cos(2 pi y/131 + p2) + noise."""
    g = SplitMix64(seed)
    p1 = 2 * math.pi * g.uniform()
    p2 = 2 * math.pi * g.uniform()
    noise = g.uniforms(nx * ny)
    r = np.empty(nx * ny)
    for iy in range(ny):
        for ix in range(nx):
            x, y = ix * pitch, iy * pitch
            v = 0.16 + 0.065 * math.sin(2 * math.pi * x / 97 + p1) * math.cos(2 * math.pi * y / 131 + p2)
            v += -0.01 + 0.02 * noise[iy * nx + ix]
            r[iy * nx + ix] = min(0.24, max(0.08, v))
    return r


def served_stream(n_requests, seed, rate_per_s, k_lo=10, k_hi=60, buf=4):
    """Request stream of sub-region solves: core k x k with k ~ U{k_lo..k_hi}, a
    `buf`-site padding ring, radii ~ U[0.08, 0.24] over the (k + 2 buf)^2 patch,
    wavelength ~ U[0.9, 1.1], nmax ~ U{3, 4, 5}, Poisson arrivals at `rate_per_s`
    (exponential gaps). Returns a list of dicts, ordered by arrival time."""
    g = SplitMix64(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        k = k_lo + min(k_hi - k_lo, int(g.uniform() * (k_hi - k_lo + 1)))
        side = k + 2 * buf
        radii = 0.08 + 0.16 * g.uniforms(side * side)
        wavelength = 0.9 + 0.2 * g.uniform()
        nmax = 3 + min(2, int(g.uniform() * 3))
        gap = -math.log(max(1e-300, 1.0 - g.uniform())) / rate_per_s if rate_per_s > 0 else 0.0
        t += gap
        out.append(dict(rid=rid, k=k, buf=buf, side=side, radii=radii, wavelength=wavelength, nmax=nmax, arrival=t))
    return out
