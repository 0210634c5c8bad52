"""Sub-region decomposition of a large-area simulation (main text: "Low-overhead
multi-GPU simulation strategy"; Fig. 3): the incident field is represented by
one jinc source per lambda/2 grid point (App. II); the sources are grouped by
sub-region core; each group is simulated with the scatterers of its core plus a
padding ring, and the scattered fields of all groups are added.

Plain definition: for every sub-region (oracle.geometry.subregion_sets order),
  a0  = jinc-group coefficients of the core's sources about the padded set,
  s   = solution of (I - T A) s = T a0 on the padded set (dense LU),
  E  += sum_{i in padded set} s_i^T Phi(k(x - x_i)) at the detectors.
"""
import numpy as np

from . import field, geometry, incident, mie, system


def sweep_fields(nmax, k0, nx, ny, pitch, z, radius, n_sphere, src_A, z0, core, buf, pts, rule_for, cutoff=0.0,
                 taper=0.0):
    """src_A: (nx*ny, 2) transverse amplitudes of the source at each site.
    rule_for(sim_pos, src_xy) -> jinc rule for one sub-region. Returns E (M, 3)."""
    pos_all = np.zeros((nx * ny, 3))
    iy, ix = np.divmod(np.arange(nx * ny), nx)
    pos_all[:, 0] = ix * pitch
    pos_all[:, 1] = iy * pitch
    pos_all[:, 2] = z
    E = np.zeros((len(pts), 3), dtype=np.complex128)
    for core_idx, sim_idx in geometry.subregion_sets(nx, ny, core[0], core[1], buf):
        pos = pos_all[sim_idx]
        src_xy = pos_all[core_idx, :2]
        rule = rule_for(pos, src_xy)
        a0 = incident.jinc_group_coeffs(nmax, k0, pos, src_xy, src_A[core_idx], z0, rule, pitch=pitch)
        T = np.array([mie.tmatrix_diag(nmax, k0, radius[i], n_sphere) for i in sim_idx])
        with system.window(cutoff, taper):
            s = system.solve_dense(nmax, k0, pos, T, a0, cutoff)
        E += field.scattered_field(nmax, k0, pos, s, pts)
    return E
