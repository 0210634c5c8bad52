// tmat_solve / tmat_adjoint: the collective-scattering solve of App. I-C/I-D
// (K s = T a0 with K = I - T A) and the adjoint radius gradient of App. IV.
#include <chrono>
#include <cmath>

#include "dev.cuh"
#include "solver.h"

struct tmat_solution {
  int device = 0;
  int64_t N = 0;
  int nmax = 0;
  double k = 0;
  tmat::SolveParams params;
  int path = TMAT_PATH_NEIGHBOUR;
  double cutoff = 0;
  double taper = 0;
  int lattice_nx = 0, lattice_ny = 0;
  double lattice_pitch = 0;
  // owned device copies (internal layout where coefficients)
  double* pos = nullptr;
  double2* T64 = nullptr;
  float2* T32 = nullptr;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double2* a0 = nullptr;  // RHS 0
  double2* s = nullptr;   // RHS 0
};

namespace tmat {

bool Operator::fp32() const { return kind == 0 ? nbr.fp32 : lattice_fp32(*lat); }
int64_t Operator::N() const { return kind == 0 ? nbr.N : lattice_N(*lat); }
int Operator::nmax() const { return kind == 0 ? nbr.nmax : lattice_nmax(*lat); }

int op_apply(tmat_ctx* ctx, const Operator& A, int mode, const void* x, void* y, int R) {
  if (A.kind == 0) return nbr_apply(ctx, A.nbr, mode, x, y, R);
  return lattice_apply(ctx, *A.lat, mode, x, y, R);
}

// b[r][i][u] = T[i][u] a[r][i][u]   (internal layout, complex128)
__global__ void tdiag_mul_kernel(const double2* __restrict__ T, const double2* __restrict__ a, double2* __restrict__ b,
                                 int64_t NP, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = cmul(T[t % NP], a[t]);
}

// grad[i] = 2 Re sum_u mu[i][u] dT[i][u] e[i][u]; e = a0 + (A s)
__global__ void grad_kernel(const double2* __restrict__ mu, const double2* __restrict__ dT, const double2* __restrict__ a0,
                            const double2* __restrict__ As, int64_t N, int P, double* __restrict__ grad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0;
  for (int u = 0; u < P; ++u) {
    int64_t o = i * P + u;
    double2 e = make_double2(a0[o].x + As[o].x, a0[o].y + As[o].y);
    double2 t = cmul(cmul(mu[o], dT[o]), e);
    acc += t.x;
  }
  grad[i] = 2.0 * acc;
}

template <typename T>
static int dmalloc_copy(tmat_ctx* ctx, T** dst, const void* src, size_t bytes) {
  TM_CUDA(ctx, cudaMalloc((void**)dst, bytes ? bytes : 16));
  if (bytes && src) TM_CUDA(ctx, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return TMAT_OK;
}

static void free_solution(tmat_solution* s) {
  if (!s) return;
  cudaFree(s->pos);
  cudaFree(s->T64);
  cudaFree(s->T32);
  cudaFree(s->row_ptr);
  cudaFree(s->col);
  cudaFree(s->a0);
  cudaFree(s->s);
  delete s;
}


static int make_nbr_ops(const Tables* t, const double* d_pos, int64_t N, double k, int nmax, const int64_t* rp,
                        const int32_t* col, double cutoff, double taper, const double2* T64, const float2* T32,
                        bool mixed, OpPair* ops) {
  NbrOp a;
  a.cutoff = cutoff;
  a.taper = taper;
  a.pos = d_pos;
  a.N = N;
  a.k = k;
  a.nmax = nmax;
  a.fp32 = false;
  a.T = T64;
  a.row_ptr = rp;
  a.col = col;
  a.tab = t;
  ops->A64.kind = 0;
  ops->A64.nbr = a;
  if (mixed) {
    a.fp32 = true;
    a.T = T32;
    ops->A32.kind = 0;
    ops->A32.nbr = a;
    ops->have32 = true;
  }
  return TMAT_OK;
}

// The tensor-core kernel counts CTAs that gave up on a bounded wait.
static int check_tc_errors(tmat_ctx* ctx, const OpPair& ops) {
  const int* counters[2] = {
      (ops.have32 && ops.A32.kind == 1 && ops.lat32.use_tc) ? ops.lat32.tc_err : nullptr,
      ops.have_oz ? ops.lat64oz.oz_err : nullptr};
  for (const int* c : counters) {
    if (!c) continue;
    int* pin = (int*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, c, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pin[0]) return set_error(ctx, TMAT_ECUDA, "tensor-core apply: %d tiles gave up on a bounded wait", pin[0]);
  }
  return TMAT_OK;
}

// The solve's operators: the iterated one (A64 or, for TMAT_PREC_FP64_TC, R64), the
// complex64 one and the refinement residual's.
static int solve_with(tmat_ctx* ctx, const OpPair& ops, int precision, int mode, const double2* b, double2* x, int R,
                      const SolveParams& sp, SolveStats* st) {
  if (precision == TMAT_PREC_FP64_TC) {
    if (!ops.have_oz)
      return set_error(ctx, TMAT_ENOTSUP,
                       "TMAT_PREC_FP64_TC needs the lattice path, tensor cores enabled, nmax <= 4 and a cutoff window that fits");
    return solve_system(ctx, ops.R64, nullptr, mode, b, x, R, sp, st);
  }
  return solve_system(ctx, ops.A64, ops.have32 ? &ops.A32 : nullptr, mode, b, x, R, sp, st,
                      ops.have_oz ? &ops.R64 : nullptr);
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_solution_free(tmat_solution* sol) {
  free_solution(sol);
  return TMAT_OK;
}

extern "C" int tmat_solve(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                          const tmat_c128* T_diag, const tmat_c128* a0, int R, const tmat_solve_opts* opts,
                          tmat_c128* s_out, tmat_solution** keep, tmat_solve_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (keep) *keep = nullptr;
  if (N < 0 || R < 1 || R > TMAT_MAX_RHS || !opts || !(wavelength > 0) || !(n_bg > 0) ||
      (N > 0 && (!pos || !T_diag || !a0 || !s_out)))
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: bad arguments (R must be 1..%d)", TMAT_MAX_RHS);
  if (!(opts->taper >= 0) || (opts->taper > 0 && !(opts->taper <= opts->cutoff)))
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: taper must be in [0, cutoff]");
  if (opts->precision != TMAT_PREC_FP64 && opts->precision != TMAT_PREC_MIXED && opts->precision != TMAT_PREC_FP64_TC)
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: unknown precision %d", opts->precision);
  Tables* t;
  TM_TRY(get_tables(ctx, nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = t->P;
  const double k = 2.0 * M_PI * n_bg / wavelength;
  SolveParams sp;
  sp.precision = opts->precision;
  sp.tol = opts->tol > 0 ? opts->tol : 1e-6;
  sp.restart = opts->restart > 0 ? opts->restart : 40;
  sp.max_iter = opts->max_iter > 0 ? opts->max_iter : 2000;
  sp.inner_tol = opts->inner_tol > 0 ? opts->inner_tol : 1e-4;
  int path = opts->path;
  if (path == TMAT_PATH_AUTO) path = opts->lattice_nx > 0 ? TMAT_PATH_LATTICE : TMAT_PATH_NEIGHBOUR;
  if (path != TMAT_PATH_NEIGHBOUR && path != TMAT_PATH_LATTICE)
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: unknown path %d", opts->path);
  if (info) {
    *info = tmat_solve_info();
    info->n_rhs = R;
  }
  if (N == 0) {
    if (info) info->converged = 1;
    return TMAT_OK;
  }
  Staged spos, sT, sa, ss;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &spos));
  int ok;
  TM_TRY(check_coplanar(ctx, (const double*)spos.dev, N, &ok));
  if (!ok) return set_error(ctx, TMAT_EINVAL, "tmat_solve: positions must be coplanar (equal z) and finite");
  TM_TRY(stage_in(ctx, "st_T", T_diag, sizeof(double2) * N * P, &sT));
  TM_TRY(stage_in(ctx, "st_a0", a0, sizeof(double2) * R * N * P, &sa));
  TM_TRY(stage_out(ctx, "st_s", s_out, sizeof(double2) * R * N * P, &ss));
  const bool mixed = sp.precision == TMAT_PREC_MIXED;
  void *T64, *T32 = nullptr;
  TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, false, "sv_T64", &T64));
  if (mixed) TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, true, "sv_T32", &T32));
  OpPair ops;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  int64_t nnz = 0;
  if (path == TMAT_PATH_NEIGHBOUR) {
    TM_TRY(scratch(ctx, "sv_rowptr", sizeof(int64_t) * (N + 1), (void**)&rp));
    TM_TRY(build_neighbors(ctx, (const double*)spos.dev, N, opts->cutoff, rp, nullptr, &nnz));
    TM_TRY(scratch(ctx, "sv_col", sizeof(int32_t) * (nnz + 1), (void**)&col));
    TM_TRY(build_neighbors(ctx, (const double*)spos.dev, N, opts->cutoff, rp, col, &nnz));
    TM_TRY(make_nbr_ops(t, (const double*)spos.dev, N, k, nmax, rp, col, opts->cutoff, opts->taper,
                        (const double2*)T64, (const float2*)T32, mixed, &ops));
  } else {
    TM_TRY(make_lattice_ops(ctx, t, (const double*)spos.dev, N, k, opts->lattice_nx, opts->lattice_ny,
                            opts->lattice_pitch, opts->cutoff, opts->taper, (const double2*)T64, (const float2*)T32, mixed, &ops,
                            sp.precision == TMAT_PREC_FP64_TC ? 2 : (mixed ? 1 : 0)));
  }
  // b = T a0 (internal layout)
  double2 *a0i, *b, *x;
  TM_TRY(scratch(ctx, "sv_a0", sizeof(double2) * R * N * P, (void**)&a0i));
  TM_TRY(scratch(ctx, "sv_b", sizeof(double2) * R * N * P, (void**)&b));
  TM_TRY(scratch(ctx, "sv_x", sizeof(double2) * R * N * P, (void**)&x));
  TM_TRY(to_internal(ctx, t, (const double2*)sa.dev, a0i, false, (int64_t)R * N));
  tdiag_mul_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)R * N * P, 256), 65535), 256, 0, ctx->stream>>>(
      (const double2*)T64, a0i, b, N * P, (int64_t)R * N * P);
  TM_LAUNCHED(ctx);
  SolveStats st;
  TM_TRY(solve_with(ctx, ops, sp.precision, TMAT_OP_FORWARD, b, x, R, sp, &st));
  TM_TRY(check_tc_errors(ctx, ops));
  TM_TRY(from_internal(ctx, t, x, false, (double2*)ss.dev, (int64_t)R * N));
  TM_TRY(finish_out(ctx, &ss));
  if (keep) {
    tmat_solution* so = new tmat_solution();
    so->device = ctx->device;
    so->N = N;
    so->nmax = nmax;
    so->k = k;
    so->params = sp;
    so->path = path;
    so->cutoff = opts->cutoff;
    so->taper = opts->taper;
    so->lattice_nx = opts->lattice_nx;
    so->lattice_ny = opts->lattice_ny;
    so->lattice_pitch = opts->lattice_pitch;
    int rc = TMAT_OK;
    do {
      if ((rc = dmalloc_copy(ctx, &so->pos, spos.dev, sizeof(double) * 3 * N))) break;
      if ((rc = dmalloc_copy(ctx, &so->T64, T64, sizeof(double2) * N * P))) break;
      if (mixed && (rc = dmalloc_copy(ctx, &so->T32, T32, sizeof(float2) * N * P))) break;
      if (path == TMAT_PATH_NEIGHBOUR) {
        if ((rc = dmalloc_copy(ctx, &so->row_ptr, rp, sizeof(int64_t) * (N + 1)))) break;
        if ((rc = dmalloc_copy(ctx, &so->col, col, sizeof(int32_t) * (nnz + 1)))) break;
      }
      if ((rc = dmalloc_copy(ctx, &so->a0, a0i, sizeof(double2) * N * P))) break;
      if ((rc = dmalloc_copy(ctx, &so->s, x, sizeof(double2) * N * P))) break;
    } while (0);
    if (rc) {
      free_solution(so);
      return rc;
    }
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *keep = so;
  }
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (info) {
    info->iterations = st.iterations;
    info->refinements = st.refinements;
    info->converged = st.converged ? 1 : 0;
    for (int r = 0; r < R; ++r) info->rel_residual[r] = st.rel_res[r];
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  if (!st.converged) return set_error(ctx, TMAT_ENOCONV, "tmat_solve: not converged after %d iterations", st.iterations);
  return TMAT_OK;
}

extern "C" int tmat_adjoint(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* v, const tmat_c128* dTdr,
                            double* grad_out, tmat_c128* mu_out, tmat_solve_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (!sol || !v || !dTdr || !grad_out) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint: bad arguments");
  if (sol->device != ctx->device) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint: solution is on another device");
  Tables* t;
  TM_TRY(get_tables(ctx, sol->nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t N = sol->N;
  const int P = t->P;
  if (info) {
    *info = tmat_solve_info();
    info->n_rhs = 1;
  }
  Staged sv, sd, sg, sm;
  TM_TRY(stage_in(ctx, "st_v", v, sizeof(double2) * N * P, &sv));
  TM_TRY(stage_in(ctx, "st_dT", dTdr, sizeof(double2) * N * P, &sd));
  TM_TRY(stage_out(ctx, "st_grad", grad_out, sizeof(double) * N, &sg));
  TM_TRY(stage_out(ctx, "st_mu", mu_out, sizeof(double2) * N * P, &sm));
  const bool mixed = sol->params.precision == TMAT_PREC_MIXED;
  OpPair ops;
  if (sol->path == TMAT_PATH_NEIGHBOUR) {
    TM_TRY(make_nbr_ops(t, sol->pos, N, sol->k, sol->nmax, sol->row_ptr, sol->col, sol->cutoff, sol->taper, sol->T64,
                        sol->T32, mixed, &ops));
  } else {
    TM_TRY(make_lattice_ops(ctx, t, sol->pos, N, sol->k, sol->lattice_nx, sol->lattice_ny, sol->lattice_pitch,
                            sol->cutoff, sol->taper, sol->T64, sol->T32, mixed, &ops,
                            sol->params.precision == TMAT_PREC_FP64_TC ? 2 : (mixed ? 1 : 0)));
  }
  double2 *vi, *mu, *dTi, *As;
  TM_TRY(scratch(ctx, "adj_v", sizeof(double2) * N * P, (void**)&vi));
  TM_TRY(scratch(ctx, "adj_mu", sizeof(double2) * N * P, (void**)&mu));
  TM_TRY(scratch(ctx, "adj_dT", sizeof(double2) * N * P, (void**)&dTi));
  TM_TRY(scratch(ctx, "adj_As", sizeof(double2) * N * P, (void**)&As));
  TM_TRY(to_internal(ctx, t, (const double2*)sv.dev, vi, false, N));
  TM_TRY(to_internal(ctx, t, (const double2*)sd.dev, dTi, false, N));
  SolveStats st;
  TM_TRY(solve_with(ctx, ops, sol->params.precision, TMAT_OP_ADJOINT, vi, mu, 1, sol->params, &st));
  // e = a0 + A s with an fp64-accurate operator
  TM_TRY(op_apply(ctx, ops.have_oz ? ops.R64 : ops.A64, TMAT_OP_COUPLE, sol->s, As, 1));
  TM_TRY(check_tc_errors(ctx, ops));
  grad_kernel<<<(unsigned)cdiv(N, 128), 128, 0, ctx->stream>>>(mu, dTi, sol->a0, As, N, P, (double*)sg.dev);
  TM_LAUNCHED(ctx);
  if (mu_out) TM_TRY(from_internal(ctx, t, mu, false, (double2*)sm.dev, N));
  TM_TRY(finish_out(ctx, &sg));
  TM_TRY(finish_out(ctx, &sm));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (info) {
    info->iterations = st.iterations;
    info->refinements = st.refinements;
    info->converged = st.converged ? 1 : 0;
    info->rel_residual[0] = st.rel_res[0];
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  if (!st.converged) return set_error(ctx, TMAT_ENOCONV, "tmat_adjoint: not converged after %d iterations", st.iterations);
  return TMAT_OK;
}
