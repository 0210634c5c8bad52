// Sub-region sweep (main text, "Low-overhead multi-GPU simulation strategy";
// Fig. 3): the incident field is sampled by one jinc source per lattice site
// (App. II); the sources of each sub-region core drive an independent solve over
// the core plus a padding ring, and the scattered fields of all sub-regions are
// added at the detectors in sub-region order (deterministic).
#include <chrono>
#include <cmath>
#include <vector>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

// gather a rectangle [px0, px0+w) x [py0, py0+h) of the lattice: positions, atoms, and
// (for the core) source positions and amplitudes
__global__ void sweep_gather_kernel(int nx, double pitch, double x0, double y0, double z, int px0, int py0, int w,
                                    int h, const tmat_atom* __restrict__ atoms, double* __restrict__ pos,
                                    tmat_atom* __restrict__ sub_atoms) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w * h) return;
  int ix = px0 + t % w, iy = py0 + t / w;
  pos[3 * t] = x0 + ix * pitch;
  pos[3 * t + 1] = y0 + iy * pitch;
  pos[3 * t + 2] = z;
  sub_atoms[t] = atoms[(int64_t)iy * nx + ix];
}

// every site's position and sphere radius (for the overlap check)
__global__ void sweep_sites_kernel(int nx, int nsites, double pitch, double x0, double y0, double z,
                                   const tmat_atom* __restrict__ atoms, double* __restrict__ pos,
                                   double* __restrict__ rad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsites) return;
  pos[3 * t] = x0 + (t % nx) * pitch;
  pos[3 * t + 1] = y0 + (t / nx) * pitch;
  pos[3 * t + 2] = z;
  rad[t] = atoms[t].radius;
}

__global__ void sweep_sources_kernel(int nx, int nsites, double pitch, double x0, double y0, int cx0, int cy0, int w,
                                     int h, int R, const double2* __restrict__ src_A, double* __restrict__ sxy,
                                     double2* __restrict__ sA) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w * h) return;
  int ix = cx0 + t % w, iy = cy0 + t / w;
  int64_t site = (int64_t)iy * nx + ix;
  sxy[2 * t] = x0 + ix * pitch;
  sxy[2 * t + 1] = y0 + iy * pitch;
  for (int r = 0; r < R; ++r) {
    sA[((int64_t)r * w * h + t) * 2] = src_A[((int64_t)r * nsites + site) * 2];
    sA[((int64_t)r * w * h + t) * 2 + 1] = src_A[((int64_t)r * nsites + site) * 2 + 1];
  }
}

__global__ void add_kernel(double2* __restrict__ acc, const double2* __restrict__ v, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) acc[t] = cadd(acc[t], v[t]);
}

int field_dev(tmat_ctx* ctx, const double* pos, int64_t N, double k, int nmax, const double2* s, const double* pts,
              int64_t M, bool far, double2* E);  // field.cu

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_sweep(tmat_ctx* ctx, const tmat_sweep_opts* sw, const tmat_atom* atoms, double wavelength,
                          double n_bg, int nmax, const tmat_c128* src_A, int R, const tmat_solve_opts* opts,
                          const double* pts, int64_t M, tmat_c128* E_out, tmat_sweep_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (!sw || !opts || !atoms || !src_A || R < 1 || R > 4 || M < 0 || (M > 0 && (!pts || !E_out)) || sw->nx <= 0 ||
      sw->ny <= 0 || sw->core_x <= 0 || sw->core_y <= 0 || sw->buffer < 0 || !(sw->pitch > 0) || !(wavelength > 0) ||
      !(n_bg > 0))
    return set_error(ctx, TMAT_EINVAL, "tmat_sweep: bad arguments (R must be 1..4)");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int nx = sw->nx, ny = sw->ny, nsites = nx * ny;
  const int P = num_coeffs(nmax);
  const double k = 2.0 * M_PI * n_bg / wavelength;
  Staged sa, ssrc, spts, sE;
  TM_TRY(stage_in(ctx, "sw_atoms", atoms, sizeof(tmat_atom) * nsites, &sa));
  TM_TRY(stage_in(ctx, "sw_srcA", src_A, sizeof(double2) * 2 * (size_t)R * nsites, &ssrc));
  TM_TRY(stage_in(ctx, "sw_pts", pts, sizeof(double) * 3 * M, &spts));
  // E_out accumulates: bring the caller's values in, add, copy back
  TM_TRY(stage_in(ctx, "sw_E", E_out, sizeof(double2) * 3 * (size_t)R * M, &sE));
  const int nax = (nx + sw->core_x - 1) / sw->core_x, nay = (ny + sw->core_y - 1) / sw->core_y;
  const int nsub = nax * nay;
  const int first = sw->first > 0 ? sw->first : 0;
  const int last = sw->count > 0 ? std::min(nsub, first + sw->count) : nsub;
  const int maxw = std::min(nx, sw->core_x + 2 * sw->buffer), maxh = std::min(ny, sw->core_y + 2 * sw->buffer);
  const int64_t maxn = (int64_t)maxw * maxh;
  double *pos, *sxy;
  tmat_atom* sat;
  double2 *T, *a0, *s, *Ea, *sA;
  // the sub-region buffers live in context scratch under their own names
  TM_TRY(scratch(ctx, "sw_pos", sizeof(double) * 3 * maxn, (void**)&pos));
  TM_TRY(scratch(ctx, "sw_subatoms", sizeof(tmat_atom) * maxn, (void**)&sat));
  TM_TRY(scratch(ctx, "sw_T", sizeof(double2) * maxn * P, (void**)&T));
  TM_TRY(scratch(ctx, "sw_a0", sizeof(double2) * (size_t)R * maxn * P, (void**)&a0));
  TM_TRY(scratch(ctx, "sw_s", sizeof(double2) * (size_t)R * maxn * P, (void**)&s));
  TM_TRY(scratch(ctx, "sw_Ea", sizeof(double2) * 3 * (size_t)std::max<int64_t>(M, 1), (void**)&Ea));
  TM_TRY(scratch(ctx, "sw_sxy", sizeof(double) * 2 * (size_t)sw->core_x * sw->core_y, (void**)&sxy));
  TM_TRY(scratch(ctx, "sw_sA", sizeof(double2) * 2 * (size_t)R * sw->core_x * sw->core_y, (void**)&sA));
  {
    // the spheres of the whole array must not intersect (App. I-C); checked once per call
    double *pall, *rall;
    TM_TRY(scratch(ctx, "sw_pos_all", sizeof(double) * 3 * (size_t)nsites, (void**)&pall));
    TM_TRY(scratch(ctx, "sw_rad_all", sizeof(double) * (size_t)nsites, (void**)&rall));
    sweep_sites_kernel<<<(unsigned)cdiv(nsites, 256), 256, 0, ctx->stream>>>(
        nx, nsites, sw->pitch, sw->x0, sw->y0, sw->z, (const tmat_atom*)sa.dev, pall, rall);
    TM_LAUNCHED(ctx);
    TM_TRY(check_overlap(ctx, pall, rall, nsites, nullptr));
  }
  tmat_sweep_info inf = tmat_sweep_info();
  for (int a = first; a < last; ++a) {
    const int ax = a % nax, ay = a / nax;
    const int cx0 = ax * sw->core_x, cx1 = std::min(nx, cx0 + sw->core_x);
    const int cy0 = ay * sw->core_y, cy1 = std::min(ny, cy0 + sw->core_y);
    const int px0 = std::max(0, cx0 - sw->buffer), px1 = std::min(nx, cx1 + sw->buffer);
    const int py0 = std::max(0, cy0 - sw->buffer), py1 = std::min(ny, cy1 + sw->buffer);
    const int w = px1 - px0, h = py1 - py0, cw = cx1 - cx0, ch = cy1 - cy0;
    const int64_t n = (int64_t)w * h;
    sweep_gather_kernel<<<(unsigned)cdiv(n, 128), 128, 0, ctx->stream>>>(nx, sw->pitch, sw->x0, sw->y0, sw->z, px0,
                                                                         py0, w, h, (const tmat_atom*)sa.dev, pos, sat);
    TM_LAUNCHED(ctx);
    sweep_sources_kernel<<<(unsigned)cdiv((int64_t)cw * ch, 128), 128, 0, ctx->stream>>>(
        nx, nsites, sw->pitch, sw->x0, sw->y0, cx0, cy0, cw, ch, R, (const double2*)ssrc.dev, sxy, sA);
    TM_LAUNCHED(ctx);
    TM_TRY(tmat_build(ctx, sat, n, wavelength, n_bg, nmax, (tmat_c128*)T, nullptr));
    TM_TRY(tmat_incident_jinc(ctx, pos, n, wavelength, n_bg, nmax, sxy, (const tmat_c128*)sA, (int64_t)cw * ch, R,
                              sw->z0, sw->pitch, sw->n_beta, sw->n_alpha,
                              opts->precision == TMAT_PREC_MIXED ? TMAT_PREC_MIXED : TMAT_PREC_FP64, (tmat_c128*)a0));
    tmat_solve_opts o = *opts;
    o.enclosing_radii = nullptr;  // checked for the whole array above
    o.path = TMAT_PATH_LATTICE;
    o.lattice_nx = w;
    o.lattice_ny = h;
    o.lattice_pitch = sw->pitch;
    tmat_solve_info si;
    int rc = tmat_solve(ctx, pos, n, wavelength, n_bg, nmax, (const tmat_c128*)T, (const tmat_c128*)a0, R, &o,
                        (tmat_c128*)s, nullptr, &si);
    if (rc != TMAT_OK && rc != TMAT_ENOCONV) return rc;
    inf.iterations += si.iterations;
    if (!si.converged) inf.unconverged++;
    for (int r = 0; r < R; ++r) inf.worst_rel_residual = std::max(inf.worst_rel_residual, si.rel_residual[r]);
    for (int r = 0; r < R && M > 0; ++r) {
      TM_TRY(field_dev(ctx, pos, n, k, nmax, s + (size_t)r * n * P, (const double*)spts.dev, M, false, Ea));
      add_kernel<<<(unsigned)cdiv(3 * M, 256), 256, 0, ctx->stream>>>((double2*)sE.dev + (size_t)r * 3 * M, Ea, 3 * M);
      TM_LAUNCHED(ctx);
    }
    inf.subregions++;
    inf.scatterer_solves += n;
  }
  if (sE.host) {
    TM_CUDA(ctx, cudaMemcpyAsync(E_out, sE.dev, sizeof(double2) * 3 * (size_t)R * M, cudaMemcpyDeviceToHost, ctx->stream));
  }
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  inf.total_subregions = nsub;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (info) *info = inf;
  return inf.unconverged ? set_error(ctx, TMAT_ENOCONV, "tmat_sweep: %d sub-regions did not converge", inf.unconverged)
                         : TMAT_OK;
}
