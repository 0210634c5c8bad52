// tmat_solve_batch: several independent lattice problems (sub-region jobs of the main text,
// each with its own lattice size, wavelength, T and incident coefficients) solved together
// with shared kernel launches. Every problem is placed at the origin of a common canvas
// lattice with T = 0 and a0 = 0 on the canvas sites it does not own; the operator
// y = x - T A x then keeps a vector supported on the problem's sites there (T = 0 zeroes the
// rest), so GMRES on the canvas is GMRES on the problem, and the problems become the
// right-hand sides of one batched operator: every launch (FFT passes, block products with
// each problem's own spectra, Arnoldi passes, Givens steps) covers all of them, and a
// problem that has converged drops out of the Arnoldi work (per-RHS activity masks).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "dev.cuh"
#include "solver.h"

namespace tmat {

// dst[canvas site][u] = src[site][u] for the problem's sites (ix < nx, iy < ny), 0 elsewhere
template <typename R>
__global__ void canvas_scatter_kernel(const C<R>* __restrict__ src, int nx, int ny, int S, int64_t Nc, int P,
                                      C<R>* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Nc * P; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t site = e / P;
    const int u = (int)(e % P);
    const int ix = (int)(site % S), iy = (int)(site / S);
    dst[e] = (ix < nx && iy < ny) ? src[((int64_t)iy * nx + ix) * P + u] : mk<R>((R)0, (R)0);
  }
}

// dst[site][u] = src[canvas site][u] for the problem's sites
__global__ void canvas_gather_kernel(const double2* __restrict__ src, int nx, int ny, int S, int P,
                                     double2* __restrict__ dst) {
  const int64_t n = (int64_t)nx * ny * P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t site = e / P;
    const int u = (int)(e % P);
    const int ix = (int)(site % nx), iy = (int)(site / nx);
    dst[e] = src[((int64_t)iy * S + ix) * P + u];
  }
}

__global__ void canvas_positions_kernel(int S, int64_t Nc, double pitch, double* __restrict__ pos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Nc; i += (int64_t)gridDim.x * blockDim.x) {
    pos[3 * i] = (double)(i % S) * pitch;
    pos[3 * i + 1] = (double)(i / S) * pitch;
    pos[3 * i + 2] = 0.0;
  }
}

// b[r][i][u] = T[r][i][u] a[r][i][u] (every RHS its own T)
__global__ void tdiag_batch_mul_kernel(const double2* __restrict__ T, const double2* __restrict__ a,
                                       double2* __restrict__ b, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = cmul(T[t], a[t]);
}

static unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(cdiv(n, 256), 16384); }

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_solve_batch(tmat_ctx* ctx, const tmat_batch_problem* probs, int n, double n_bg, int nmax,
                                double pitch, int canvas_nx, int canvas_ny, const tmat_solve_opts* opts,
                                tmat_solve_info* infos) {
  if (!ctx) return TMAT_EINVAL;
  if (n < 1 || n > TMAT_MAX_RHS || !probs || !opts || !(n_bg > 0) || !(pitch > 0) || canvas_nx < 0 || canvas_ny < 0)
    return set_error(ctx, TMAT_EINVAL, "tmat_solve_batch: bad arguments (1..%d problems)", TMAT_MAX_RHS);
  if (opts->precision != TMAT_PREC_FP64 && opts->precision != TMAT_PREC_MIXED)
    return set_error(ctx, TMAT_EINVAL, "tmat_solve_batch: precision must be TMAT_PREC_FP64 or TMAT_PREC_MIXED");
  if (!(opts->taper >= 0) || (opts->taper > 0 && !(opts->taper <= opts->cutoff)))
    return set_error(ctx, TMAT_EINVAL, "tmat_solve_batch: taper must be in [0, cutoff]");
  int Sx = canvas_nx, Sy = canvas_ny;
  for (int r = 0; r < n; ++r) {
    const tmat_batch_problem& p = probs[r];
    if (p.nx <= 0 || p.ny <= 0 || !(p.wavelength > 0) || !p.T_diag || !p.a0 || !p.s_out)
      return set_error(ctx, TMAT_EINVAL, "tmat_solve_batch: problem %d has bad arguments", r);
    if (canvas_nx == 0) Sx = std::max(Sx, p.nx);
    if (canvas_ny == 0) Sy = std::max(Sy, p.ny);
    if (p.nx > Sx || p.ny > Sy) return set_error(ctx, TMAT_EINVAL, "tmat_solve_batch: problem %d exceeds the canvas", r);
  }
  Tables* t;
  TM_TRY(get_tables(ctx, nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  auto t_start = std::chrono::steady_clock::now();
  const int P = t->P;
  const int64_t Nc = (int64_t)Sx * Sy;
  const bool mixed = opts->precision == TMAT_PREC_MIXED;
  if (infos)
    for (int r = 0; r < n; ++r) {
      infos[r] = tmat_solve_info();
      infos[r].n_rhs = 1;
    }
  // canvas positions (the lattice of every problem starts at the canvas origin)
  double* dpos;
  TM_TRY(scratch(ctx, "bt_pos", sizeof(double) * 3 * Nc, (void**)&dpos));
  canvas_positions_kernel<<<grid_for(Nc), 256, 0, ctx->stream>>>(Sx, Nc, pitch, dpos);
  TM_LAUNCHED(ctx);
  // per problem: T and a0 on the canvas (internal layout), its operator's block spectra
  double2 *T64, *a0c, *b, *x, *tmp;
  float2* T32 = nullptr;
  TM_TRY(scratch(ctx, "bt_T64", sizeof(double2) * n * Nc * P, (void**)&T64));
  if (mixed) TM_TRY(scratch(ctx, "bt_T32", sizeof(float2) * n * Nc * P, (void**)&T32));
  TM_TRY(scratch(ctx, "bt_a0", sizeof(double2) * n * Nc * P, (void**)&a0c));
  TM_TRY(scratch(ctx, "bt_b", sizeof(double2) * n * Nc * P, (void**)&b));
  TM_TRY(scratch(ctx, "bt_x", sizeof(double2) * n * Nc * P, (void**)&x));
  int64_t maxn = 0;
  for (int r = 0; r < n; ++r) maxn = std::max<int64_t>(maxn, (int64_t)probs[r].nx * probs[r].ny);
  TM_TRY(scratch(ctx, "bt_tmp", sizeof(double2) * maxn * P, (void**)&tmp));
  OpPair first;
  void *B64 = nullptr, *B32 = nullptr, *C32 = nullptr;
  int64_t s64 = 0, s32 = 0, sc32 = 0;
  for (int r = 0; r < n; ++r) {
    const tmat_batch_problem& p = probs[r];
    const int64_t np_ = (int64_t)p.nx * p.ny;
    Staged sT, sa;
    TM_TRY(stage_in(ctx, "bt_stT", p.T_diag, sizeof(double2) * np_ * P, &sT));
    TM_TRY(to_internal(ctx, t, (const double2*)sT.dev, tmp, false, np_));
    canvas_scatter_kernel<double><<<grid_for(Nc * P), 256, 0, ctx->stream>>>(tmp, p.nx, p.ny, Sx, Nc, P,
                                                                             T64 + (int64_t)r * Nc * P);
    TM_LAUNCHED(ctx);
    if (mixed) {
      TM_TRY(to_internal(ctx, t, (const double2*)sT.dev, tmp, true, np_));
      canvas_scatter_kernel<float><<<grid_for(Nc * P), 256, 0, ctx->stream>>>((const float2*)tmp, p.nx, p.ny, Sx, Nc,
                                                                             P, T32 + (int64_t)r * Nc * P);
      TM_LAUNCHED(ctx);
    }
    TM_TRY(stage_in(ctx, "bt_sta", p.a0, sizeof(double2) * np_ * P, &sa));
    TM_TRY(to_internal(ctx, t, (const double2*)sa.dev, tmp, false, np_));
    canvas_scatter_kernel<double><<<grid_for(Nc * P), 256, 0, ctx->stream>>>(tmp, p.nx, p.ny, Sx, Nc, P,
                                                                             a0c + (int64_t)r * Nc * P);
    TM_LAUNCHED(ctx);
    // this problem's operator (wave number of its wavelength), then its spectra into the batch
    OpPair ops;
    const double k = 2.0 * M_PI * n_bg / p.wavelength;
    TM_TRY(make_lattice_ops(ctx, t, dpos, Nc, k, Sx, Sy, pitch, opts->cutoff, opts->taper,
                            T64 + (int64_t)r * Nc * P, mixed ? T32 + (int64_t)r * Nc * P : nullptr, mixed, &ops, 0));
    if (!ops.lat64.use_fft || (mixed && !ops.lat32.use_fft))
      return set_error(ctx, TMAT_ENOTSUP, "tmat_solve_batch: the canvas does not fit the FFT lattice operator");
    const int64_t F = (int64_t)ops.lat64.fft_Mx * ops.lat64.fft_My;
    if (r == 0) {
      first = ops;
      s64 = 2 * (int64_t)t->L * t->L * F;
      TM_TRY(scratch(ctx, "bt_B64", sizeof(double2) * n * s64, &B64));
      if (mixed) {
        s32 = s64;
        TM_TRY(scratch(ctx, "bt_B32", sizeof(float2) * n * s32, &B32));
        if (ops.lat32.fft_C) {
          const int hx = ops.lat32.fft_Mx / 2 + 1, hy = ops.lat32.fft_My / 2 + 1;
          sc32 = (int64_t)hx * hy * 2 * (((t->L * t->L + 7) / 16) * 16 + 8);
          TM_TRY(scratch(ctx, "bt_C32", sizeof(float2) * n * sc32, &C32));
        }
      }
    }
    TM_CUDA(ctx, cudaMemcpyAsync((double2*)B64 + r * s64, ops.lat64.fft_Bhat, sizeof(double2) * s64,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
    if (mixed) {
      TM_CUDA(ctx, cudaMemcpyAsync((float2*)B32 + r * s32, ops.lat32.fft_Bhat, sizeof(float2) * s32,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
      if (C32)
        TM_CUDA(ctx, cudaMemcpyAsync((float2*)C32 + r * sc32, ops.lat32.fft_C, sizeof(float2) * sc32,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  // the batched operators: problem r is RHS r
  OpPair bops;
  bops.lat64 = first.lat64;
  bops.lat64.T = T64;
  bops.lat64.t_stride = Nc * P;
  bops.lat64.fft_Bhat = B64;
  bops.lat64.fft_bstride = s64;
  bops.lat64.fft_C = nullptr;  // per-problem spectra: the mirror-pair product
  bops.A64.kind = 1;
  bops.A64.lat = &bops.lat64;
  if (mixed) {
    bops.lat32 = first.lat32;
    bops.lat32.T = T32;
    bops.lat32.t_stride = Nc * P;
    bops.lat32.fft_Bhat = B32;
    bops.lat32.fft_bstride = s32;
    bops.lat32.fft_C = C32;
    bops.lat32.fft_cstride = sc32;
    bops.A32.kind = 1;
    bops.A32.lat = &bops.lat32;
    bops.have32 = true;
  }
  tdiag_batch_mul_kernel<<<grid_for((int64_t)n * Nc * P), 256, 0, ctx->stream>>>(T64, a0c, b, (int64_t)n * Nc * P);
  TM_LAUNCHED(ctx);
  SolveParams sp;
  sp.precision = opts->precision;
  sp.tol = opts->tol > 0 ? opts->tol : 1e-6;
  sp.restart = opts->restart > 0 ? opts->restart : 40;
  sp.max_iter = opts->max_iter > 0 ? opts->max_iter : 2000;
  sp.inner_tol = opts->inner_tol > 0 ? opts->inner_tol : 1e-4;
  SolveStats st;
  TM_TRY(solve_system(ctx, bops.A64, mixed ? &bops.A32 : nullptr, TMAT_OP_FORWARD, b, x, n, sp, &st));
  if (mixed && bops.lat32.fft_C) {
    int* pin = (int*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, bops.lat32.fft_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pin[0]) return set_error(ctx, TMAT_ECUDA, "tmat_solve_batch: %d tiles gave up on a bounded wait", pin[0]);
  }
  bool all = true;
  for (int r = 0; r < n; ++r) {
    const tmat_batch_problem& p = probs[r];
    const int64_t np_ = (int64_t)p.nx * p.ny;
    canvas_gather_kernel<<<grid_for(np_ * P), 256, 0, ctx->stream>>>(x + (int64_t)r * Nc * P, p.nx, p.ny, Sx, P, tmp);
    TM_LAUNCHED(ctx);
    Staged ss;
    TM_TRY(stage_out(ctx, "bt_sts", p.s_out, sizeof(double2) * np_ * P, &ss));
    TM_TRY(from_internal(ctx, t, tmp, false, (double2*)ss.dev, np_));
    TM_TRY(finish_out(ctx, &ss));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // tmp and the staging buffer are reused
    const bool ok = st.rel_res[r] <= sp.tol;
    all = all && ok;
    if (infos) {
      infos[r].iterations = st.iterations;
      infos[r].refinements = st.refinements;
      infos[r].converged = ok ? 1 : 0;
      infos[r].rel_residual[0] = st.rel_res[r];
      infos[r].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
  }
  if (!all) return set_error(ctx, TMAT_ENOCONV, "tmat_solve_batch: not every problem converged");
  return TMAT_OK;
}
