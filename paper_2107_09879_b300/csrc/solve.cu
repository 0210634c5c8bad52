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
  bool threed = false;    // positions not coplanar (neighbour path with full 3-D blocks)
  double2* a0 = nullptr;  // RHS 0
  double2* s = nullptr;   // RHS 0
  // T-block solutions (tmat_solve_tblocks): blocks in internal order, both storages
  bool tblocks = false;
  int64_t n_types = 0;
  double2 *tb64c = nullptr, *tb64r = nullptr;
  float2 *tb32c = nullptr, *tb32r = nullptr;
  int32_t* ttype = nullptr;  // null: scatterer i uses block i
};

namespace tmat {

bool Operator::fp32() const { return kind == 0 ? nbr.fp32 : lattice_fp32(*lat); }
int64_t Operator::N() const { return kind == 0 ? nbr.N : lattice_N(*lat); }
int Operator::nmax() const { return kind == 0 ? nbr.nmax : lattice_nmax(*lat); }

static int op_apply_inner(tmat_ctx* ctx, const Operator& A, int mode, const void* x, void* y, int R) {
  if (A.kind == 0) return nbr_apply(ctx, A.nbr, mode, x, y, R);
  return lattice_apply(ctx, *A.lat, mode, x, y, R);
}

// y = x - t + w (the transposed T-block operator from t = T^T x and w = t - A^T t)
template <typename R>
__global__ void tb_combine_kernel(const C<R>* __restrict__ x, const C<R>* __restrict__ t, const C<R>* __restrict__ w,
                                  C<R>* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cadd(csub(x[i], t[i]), w[i]);
}

int op_apply(tmat_ctx* ctx, const Operator& A, int mode, const void* x, void* y, int R) {
  if (!A.tbc || mode == TMAT_OP_COUPLE) return op_apply_inner(ctx, A, mode, x, y, R);
  const bool f32 = A.fp32();
  const int64_t N = A.N();
  const int P = num_coeffs(A.nmax());
  const size_t bytes = (f32 ? sizeof(float2) : sizeof(double2)) * (size_t)R * N * P;
  void *z, *w;
  TM_TRY(scratch(ctx, f32 ? "tb_z32" : "tb_z64", bytes, &z));
  if (mode == TMAT_OP_FORWARD) {
    TM_TRY(op_apply_inner(ctx, A, TMAT_OP_COUPLE, x, z, R));
    return tblock_mul(ctx, A.tbc, A.ttype, z, x, y, N, P, R, f32);
  }
  TM_TRY(scratch(ctx, f32 ? "tb_w32" : "tb_w64", bytes, &w));
  TM_TRY(tblock_mul(ctx, A.tbr, A.ttype, x, nullptr, z, N, P, R, f32));  // t = T^T x
  TM_TRY(op_apply_inner(ctx, A, TMAT_OP_ADJOINT, z, w, R));             // w = t - A^T t (inner T = 1)
  const int64_t n = (int64_t)R * N * P;
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(n, 256), 8192);
  if (f32) tb_combine_kernel<float><<<g, 256, 0, ctx->stream>>>((const float2*)x, (const float2*)z, (const float2*)w, (float2*)y, n);
  else tb_combine_kernel<double><<<g, 256, 0, ctx->stream>>>((const double2*)x, (const double2*)z, (const double2*)w, (double2*)y, n);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

// out[r][i][a] = sum_c Tm[(type_i P + c) P + a] in[r][i][c] (minus that from xsub when given);
// one thread per (scatterer, a), the scatterer's input read by broadcast
template <typename R>
__global__ void tblock_mul_kernel(const C<R>* __restrict__ Tm, const int32_t* __restrict__ type, const C<R>* __restrict__ in,
                                  const C<R>* __restrict__ xsub, C<R>* __restrict__ out, int64_t N, int P, int R_, int SB) {
  const int loc = threadIdx.x / P, a = threadIdx.x % P;
  const int64_t i = (int64_t)blockIdx.x * SB + loc;
  if (loc >= SB || i >= N) return;
  const C<R>* Tt = Tm + (int64_t)(type ? type[i] : i) * P * P + a;
  for (int r = 0; r < R_; ++r) {
    const C<R>* v = in + ((int64_t)r * N + i) * P;
    C<R> acc = mk<R>((R)0, (R)0);
    for (int c = 0; c < P; ++c) cfma(acc, Tt[(int64_t)c * P], v[c]);
    const int64_t o = ((int64_t)r * N + i) * P + a;
    out[o] = xsub ? csub(xsub[o], acc) : acc;
  }
}

int tblock_mul(tmat_ctx* ctx, const void* Tm, const int32_t* type, const void* in, const void* xsub, void* out,
               int64_t N, int P, int R, bool fp32) {
  if (N == 0) return TMAT_OK;
  const int SB = std::max(1, 256 / P);
  const unsigned g = (unsigned)cdiv(N, SB);
  if (fp32)
    tblock_mul_kernel<float><<<g, SB * P, 0, ctx->stream>>>((const float2*)Tm, type, (const float2*)in,
                                                            (const float2*)xsub, (float2*)out, N, P, R, SB);
  else
    tblock_mul_kernel<double><<<g, SB * P, 0, ctx->stream>>>((const double2*)Tm, type, (const double2*)in,
                                                             (const double2*)xsub, (double2*)out, N, P, R, SB);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
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
  cudaFree(s->tb64c);
  cudaFree(s->tb64r);
  cudaFree(s->tb32c);
  cudaFree(s->tb32r);
  cudaFree(s->ttype);
  delete s;
}


static int make_nbr_ops(const Tables* t, const double* d_pos, int64_t N, double k, int nmax, const int64_t* rp,
                        const int32_t* col, double cutoff, double taper, const double2* T64, const float2* T32,
                        bool mixed, OpPair* ops, bool threed = false) {
  NbrOp a;
  a.cutoff = cutoff;
  a.taper = taper;
  a.threed = threed;
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
  const int* counters[3] = {
      (ops.have32 && ops.A32.kind == 1 && ops.lat32.use_tc) ? ops.lat32.tc_err : nullptr,
      ops.have_oz ? ops.lat64oz.oz_err : nullptr,
      (ops.have32 && ops.A32.kind == 1 && ops.lat32.use_fft && ops.lat32.fft_C) ? ops.lat32.fft_err : nullptr};
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

namespace tmat {
// T-blocks of a tmat_solve_tblocks call (API order, host or device)
struct TBlockArgs {
  const tmat_c128* blocks = nullptr;
  const int32_t* type = nullptr;
  int64_t n_types = 0;
};
}  // namespace tmat

// kept by the solution object of a T-block solve
struct TBlockDev {
  double2 *c64 = nullptr, *r64 = nullptr;
  float2 *c32 = nullptr, *r32 = nullptr;
  const int32_t* type = nullptr;
};

template <typename R>
__global__ void unit_kernel(C<R>* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mk<R>((R)1, (R)0);
}

// an all-ones diagonal T (internal layout) for operators whose blocks are applied around them
static int unit_T(tmat_ctx* ctx, int64_t n, bool fp32, const char* name, void** out) {
  TM_TRY(scratch(ctx, name, (fp32 ? sizeof(float2) : sizeof(double2)) * n, out));
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(n, 256), 8192);
  if (fp32) unit_kernel<float><<<g, 256, 0, ctx->stream>>>((float2*)*out, n);
  else unit_kernel<double><<<g, 256, 0, ctx->stream>>>((double2*)*out, n);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

static void attach_tblocks(OpPair* ops, const TBlockDev& d) {
  ops->A64.tbc = d.c64;
  ops->A64.tbr = d.r64;
  ops->A64.ttype = d.type;
  if (ops->have32) {
    ops->A32.tbc = d.c32;
    ops->A32.tbr = d.r32;
    ops->A32.ttype = d.type;
  }
}

// blocks in internal order: c[(ty P + c) P + a] = T[a][c], r[(ty P + c) P + a] = T[c][a]
// (internal indices; T flat is [ty][perm[a]][perm[c]])
template <typename R>
__global__ void tblock_internal_kernel(const double2* __restrict__ Tf, const int* __restrict__ perm, int64_t n, int P,
                                       C<R>* __restrict__ oc, C<R>* __restrict__ orw) {
  const int64_t PP = (int64_t)P * P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * PP; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ty = e / PP;
    const int c = (int)((e % PP) / P), a = (int)(e % P);
    const double2 tac = Tf[ty * PP + (int64_t)perm[a] * P + perm[c]];
    const double2 tca = Tf[ty * PP + (int64_t)perm[c] * P + perm[a]];
    oc[e] = mk<R>((R)tac.x, (R)tac.y);
    orw[e] = mk<R>((R)tca.x, (R)tca.y);
  }
}

__global__ void type_check_kernel(const int32_t* __restrict__ type, int64_t N, int64_t n_types, int* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    if (type[i] < 0 || type[i] >= n_types) atomicOr(bad, 1);
}

static int prepare_tblocks(tmat_ctx* ctx, const Tables* t, const TBlockArgs& tb, int64_t N, bool mixed, TBlockDev* d) {
  const int P = t->P;
  const int64_t n = tb.n_types, PP = (int64_t)P * P;
  Staged sb, st;
  TM_TRY(stage_in(ctx, "st_tblk", tb.blocks, sizeof(double2) * n * PP, &sb));
  if (tb.type) {
    TM_TRY(stage_in(ctx, "st_ttype", tb.type, sizeof(int32_t) * N, &st));
    int* flag;
    TM_TRY(scratch(ctx, "tb_flag", sizeof(int), (void**)&flag));
    TM_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    type_check_kernel<<<(unsigned)std::min<int64_t>(cdiv(N, 256), 4096), 256, 0, ctx->stream>>>(
        (const int32_t*)st.dev, N, n, flag);
    TM_LAUNCHED(ctx);
    int* pin = (int*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pin[0]) return set_error(ctx, TMAT_EINVAL, "tmat_solve_tblocks: a type index is outside [0, %lld)", (long long)n);
    d->type = (const int32_t*)st.dev;
  }
  TM_TRY(scratch(ctx, "tb_c64", sizeof(double2) * n * PP, (void**)&d->c64));
  TM_TRY(scratch(ctx, "tb_r64", sizeof(double2) * n * PP, (void**)&d->r64));
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(n * PP, 256), 16384);
  tblock_internal_kernel<double><<<g, 256, 0, ctx->stream>>>((const double2*)sb.dev, t->d_perm, n, P, d->c64, d->r64);
  TM_LAUNCHED(ctx);
  if (mixed) {
    TM_TRY(scratch(ctx, "tb_c32", sizeof(float2) * n * PP, (void**)&d->c32));
    TM_TRY(scratch(ctx, "tb_r32", sizeof(float2) * n * PP, (void**)&d->r32));
    tblock_internal_kernel<float><<<g, 256, 0, ctx->stream>>>((const double2*)sb.dev, t->d_perm, n, P, d->c32, d->r32);
    TM_LAUNCHED(ctx);
  }
  return TMAT_OK;
}

static int solve_impl(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                      const tmat_c128* T_diag, const TBlockArgs* tb, const tmat_c128* a0, int R,
                      const tmat_solve_opts* opts, tmat_c128* s_out, tmat_solution** keep, tmat_solve_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (keep) *keep = nullptr;
  if (N < 0 || R < 1 || R > TMAT_MAX_RHS || !opts || !(wavelength > 0) || !(n_bg > 0) ||
      (N > 0 && (!pos || (!T_diag && !tb) || !a0 || !s_out)))
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: bad arguments (R must be 1..%d)", TMAT_MAX_RHS);
  if (tb && (!tb->blocks || tb->n_types < 1 || (!tb->type && tb->n_types != N)))
    return set_error(ctx, TMAT_EINVAL, "tmat_solve_tblocks: need blocks, n_types >= 1 and a type array unless n_types == N");
  if (tb && opts->precision == TMAT_PREC_FP64_TC)
    return set_error(ctx, TMAT_ENOTSUP, "tmat_solve_tblocks: TMAT_PREC_FP64_TC is not supported with T-blocks");
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
  int pflags;
  TM_TRY(position_flags(ctx, (const double*)spos.dev, N, &pflags));
  if (pflags & 2) return set_error(ctx, TMAT_EINVAL, "tmat_solve: positions must be finite");
  const bool threed = (pflags & 1) != 0;
  if (opts->enclosing_radii) {
    Staged srad;
    TM_TRY(stage_in(ctx, "st_rad", opts->enclosing_radii, sizeof(double) * N, &srad));
    TM_TRY(check_overlap(ctx, (const double*)spos.dev, (const double*)srad.dev, N, nullptr));
  }
  if (threed && path == TMAT_PATH_LATTICE)
    return set_error(ctx, TMAT_EINVAL, "tmat_solve: the lattice path needs coplanar positions");
  if (!tb) TM_TRY(stage_in(ctx, "st_T", T_diag, sizeof(double2) * N * P, &sT));
  TM_TRY(stage_in(ctx, "st_a0", a0, sizeof(double2) * R * N * P, &sa));
  TM_TRY(stage_out(ctx, "st_s", s_out, sizeof(double2) * R * N * P, &ss));
  const bool mixed = sp.precision == TMAT_PREC_MIXED;
  void *T64, *T32 = nullptr;
  TBlockDev tbd;
  if (tb) {
    // the operators carry T = 1; the blocks are applied around them (op_apply)
    TM_TRY(prepare_tblocks(ctx, t, *tb, N, mixed, &tbd));
    TM_TRY(unit_T(ctx, N * P, false, "sv_one64", &T64));
    if (mixed) TM_TRY(unit_T(ctx, N * P, true, "sv_one32", &T32));
  } else {
    TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, false, "sv_T64", &T64));
    if (mixed) TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, true, "sv_T32", &T32));
  }
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
                        (const double2*)T64, (const float2*)T32, mixed, &ops, threed));
  } else {
    TM_TRY(make_lattice_ops(ctx, t, (const double*)spos.dev, N, k, opts->lattice_nx, opts->lattice_ny,
                            opts->lattice_pitch, opts->cutoff, opts->taper, (const double2*)T64, (const float2*)T32, mixed, &ops,
                            sp.precision == TMAT_PREC_FP64_TC ? 2 : (mixed && !tb ? 1 : 0)));
  }
  if (tb) attach_tblocks(&ops, tbd);
  // b = T a0 (internal layout)
  double2 *a0i, *b, *x;
  TM_TRY(scratch(ctx, "sv_a0", sizeof(double2) * R * N * P, (void**)&a0i));
  TM_TRY(scratch(ctx, "sv_b", sizeof(double2) * R * N * P, (void**)&b));
  TM_TRY(scratch(ctx, "sv_x", sizeof(double2) * R * N * P, (void**)&x));
  TM_TRY(to_internal(ctx, t, (const double2*)sa.dev, a0i, false, (int64_t)R * N));
  if (tb) {
    TM_TRY(tblock_mul(ctx, tbd.c64, tbd.type, a0i, nullptr, b, N, P, R, false));
  } else {
    tdiag_mul_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)R * N * P, 256), 65535), 256, 0, ctx->stream>>>(
        (const double2*)T64, a0i, b, N * P, (int64_t)R * N * P);
    TM_LAUNCHED(ctx);
  }
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
    so->threed = threed;
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
      if (tb) {
        const size_t nb = sizeof(double2) * tb->n_types * P * P;
        so->tblocks = true;
        so->n_types = tb->n_types;
        if ((rc = dmalloc_copy(ctx, &so->tb64c, tbd.c64, nb))) break;
        if ((rc = dmalloc_copy(ctx, &so->tb64r, tbd.r64, nb))) break;
        if (mixed && (rc = dmalloc_copy(ctx, &so->tb32c, tbd.c32, nb / 2))) break;
        if (mixed && (rc = dmalloc_copy(ctx, &so->tb32r, tbd.r32, nb / 2))) break;
        if (tbd.type && (rc = dmalloc_copy(ctx, &so->ttype, tbd.type, sizeof(int32_t) * N))) break;
      }
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

extern "C" int tmat_solve(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                          const tmat_c128* T_diag, const tmat_c128* a0, int R, const tmat_solve_opts* opts,
                          tmat_c128* s_out, tmat_solution** keep, tmat_solve_info* info) {
  return solve_impl(ctx, pos, N, wavelength, n_bg, nmax, T_diag, nullptr, a0, R, opts, s_out, keep, info);
}

extern "C" int tmat_solve_tblocks(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                                  const tmat_c128* T_blocks, const int32_t* type, int64_t n_types, const tmat_c128* a0,
                                  int R, const tmat_solve_opts* opts, tmat_c128* s_out, tmat_solution** keep,
                                  tmat_solve_info* info) {
  TBlockArgs tb;
  tb.blocks = T_blocks;
  tb.type = type;
  tb.n_types = n_types;
  return solve_impl(ctx, pos, N, wavelength, n_bg, nmax, nullptr, &tb, a0, R, opts, s_out, keep, info);
}

extern "C" int tmat_adjoint(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* v, const tmat_c128* dTdr,
                            double* grad_out, tmat_c128* mu_out, tmat_solve_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (!sol || !v || !dTdr || !grad_out) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint: bad arguments");
  if (sol->device != ctx->device) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint: solution is on another device");
  if (sol->tblocks) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint: a T-block solution needs tmat_adjoint_tblocks");
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
                        sol->T32, mixed, &ops, sol->threed));
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

// grad[i] = 2 Re sum_a mu[i][a] sum_c dT[type_i][a][c] e[i][c], e = a0 + A s; dTc in the
// column storage dTc[(ty P + c) P + a] = dT[a][c]
__global__ void grad_blocks_kernel(const double2* __restrict__ mu, const double2* __restrict__ dTc,
                                   const int32_t* __restrict__ type, const double2* __restrict__ a0,
                                   const double2* __restrict__ As, int64_t N, int P, double* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double2* D = dTc + (int64_t)(type ? type[i] : i) * P * P;
  double acc = 0;
  for (int c = 0; c < P; ++c) {
    const int64_t oc = i * P + c;
    const double2 e = make_double2(a0[oc].x + As[oc].x, a0[oc].y + As[oc].y);
    double2 row = make_double2(0.0, 0.0);  // sum_a mu[a] dT[a][c]
    for (int a = 0; a < P; ++a) row = cadd(row, cmul(mu[i * P + a], D[(int64_t)c * P + a]));
    acc += cmul(row, e).x;
  }
  grad[i] = 2.0 * acc;
}

extern "C" int tmat_adjoint_tblocks(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* v,
                                    const tmat_c128* dT_blocks, double* grad_out, tmat_c128* mu_out,
                                    tmat_solve_info* info) {
  auto t_start = std::chrono::steady_clock::now();
  if (!ctx) return TMAT_EINVAL;
  if (!sol || !v || !dT_blocks || !grad_out) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint_tblocks: bad arguments");
  if (sol->device != ctx->device) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint_tblocks: solution is on another device");
  if (!sol->tblocks) return set_error(ctx, TMAT_EINVAL, "tmat_adjoint_tblocks: not a T-block solution (use tmat_adjoint)");
  Tables* t;
  TM_TRY(get_tables(ctx, sol->nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t N = sol->N;
  const int P = t->P;
  if (info) {
    *info = tmat_solve_info();
    info->n_rhs = 1;
  }
  const bool mixed = sol->params.precision == TMAT_PREC_MIXED;
  Staged sv, sd, sg, sm;
  TM_TRY(stage_in(ctx, "st_v", v, sizeof(double2) * N * P, &sv));
  TM_TRY(stage_in(ctx, "st_dTb", dT_blocks, sizeof(double2) * sol->n_types * P * P, &sd));
  TM_TRY(stage_out(ctx, "st_grad", grad_out, sizeof(double) * N, &sg));
  TM_TRY(stage_out(ctx, "st_mu", mu_out, sizeof(double2) * N * P, &sm));
  void *one64, *one32 = nullptr;
  TM_TRY(unit_T(ctx, N * P, false, "sv_one64", &one64));
  if (mixed) TM_TRY(unit_T(ctx, N * P, true, "sv_one32", &one32));
  OpPair ops;
  if (sol->path == TMAT_PATH_NEIGHBOUR) {
    TM_TRY(make_nbr_ops(t, sol->pos, N, sol->k, sol->nmax, sol->row_ptr, sol->col, sol->cutoff, sol->taper,
                        (const double2*)one64, (const float2*)one32, mixed, &ops, sol->threed));
  } else {
    TM_TRY(make_lattice_ops(ctx, t, sol->pos, N, sol->k, sol->lattice_nx, sol->lattice_ny, sol->lattice_pitch,
                            sol->cutoff, sol->taper, (const double2*)one64, (const float2*)one32, mixed, &ops, 0));
  }
  TBlockDev d;
  d.c64 = sol->tb64c;
  d.r64 = sol->tb64r;
  d.c32 = sol->tb32c;
  d.r32 = sol->tb32r;
  d.type = sol->ttype;
  attach_tblocks(&ops, d);
  // derivative blocks in the column storage (the row storage is not needed)
  double2 *dTc, *dTr, *vi, *mu, *As;
  TM_TRY(scratch(ctx, "adjb_dTc", sizeof(double2) * sol->n_types * P * P, (void**)&dTc));
  TM_TRY(scratch(ctx, "adjb_dTr", sizeof(double2) * sol->n_types * P * P, (void**)&dTr));
  tblock_internal_kernel<double><<<(unsigned)std::min<int64_t>(cdiv(sol->n_types * P * P, 256), 16384), 256, 0,
                                   ctx->stream>>>((const double2*)sd.dev, t->d_perm, sol->n_types, P, dTc, dTr);
  TM_LAUNCHED(ctx);
  TM_TRY(scratch(ctx, "adj_v", sizeof(double2) * N * P, (void**)&vi));
  TM_TRY(scratch(ctx, "adj_mu", sizeof(double2) * N * P, (void**)&mu));
  TM_TRY(scratch(ctx, "adj_As", sizeof(double2) * N * P, (void**)&As));
  TM_TRY(to_internal(ctx, t, (const double2*)sv.dev, vi, false, N));
  SolveStats st;
  TM_TRY(solve_with(ctx, ops, sol->params.precision, TMAT_OP_ADJOINT, vi, mu, 1, sol->params, &st));
  TM_TRY(op_apply(ctx, ops.A64, TMAT_OP_COUPLE, sol->s, As, 1));  // e = a0 + A s (fp64)
  TM_TRY(check_tc_errors(ctx, ops));
  grad_blocks_kernel<<<(unsigned)cdiv(N, 128), 128, 0, ctx->stream>>>(mu, dTc, sol->ttype, sol->a0, As, N, P,
                                                                       (double*)sg.dev);
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
  if (!st.converged)
    return set_error(ctx, TMAT_ENOCONV, "tmat_adjoint_tblocks: not converged after %d iterations", st.iterations);
  return TMAT_OK;
}

// ---- position gradient (App. IV with the in-plane positions as parameters) ---------
//
// With s = T e, e = a0 + A s and the adjoint solution mu of (I - A^T T) mu = v (as in
// tmat_adjoint), the variation of the figure of merit at fixed T is
//   dFoM = 2 Re[ (T mu)^T (da0 + dA s) ] + (explicit dependence of E(x_f) on the positions).
// A block A_jl = F(x_j - x_l) depends on both ends: for position q_i of scatterer i,
//   (T mu)^T (dA/dq_i) s = (T mu)_i . (A'_q s)_i - (A'_q^T T mu)_i . s_i,
// where A'_q is the lattice operator whose blocks are dF/dd_q at the lattice offsets (the
// coupling window's derivative included). The explicit term is
//   2 Re sum_c conj(E_c) s_i . d/dq_i Phi_c(k(x_f - x_i)),
// taken as a central difference of the fp64 wave functions in x_f (step 1e-4 / k; error
// ~ (k h)^2 / 6 relative). The derivative operators are applied in fp64, by FFT
// convolution with their own block spectra where the operator's grid fits.
namespace tmat {

// BX/BY[k][c][u'][u] = d/dd_x, d/dd_y of w(rho) e^{i(m_u' - m_u) phi} sum_q G[c][u][u'][q] h_q(k rho)
// at d = -(dx, dy) pitch, the layout of the lattice blocks
template <int NMAX>
__global__ void lattice_dblocks_kernel(const int2* __restrict__ off, int K, double pitch, double k, double cutoff,
                                       double taper, const double2* __restrict__ G, const int* __restrict__ mval,
                                       int LP, double2* __restrict__ BX, double2* __restrict__ BY) {
  constexpr int L = NMAX * (NMAX + 2), Q = 2 * NMAX + 1;
  __shared__ double2 h[Q], hp[Q];                // h_q(k rho) and d/d rho of it
  __shared__ double2 eph[2 * (2 * NMAX) + 1];    // e^{i mu phi}
  const int kk = blockIdx.x;
  if (kk >= K) return;
  const double dx = -(double)off[kk].x * pitch, dy = -(double)off[kk].y * pitch;
  const double rho = sqrt(dx * dx + dy * dy);
  if (off[kk].x == 0 && off[kk].y == 0) {
    for (int e = threadIdx.x; e < 2 * L * L; e += blockDim.x) {
      const int c = e / (L * L), u = (e / L) % L, up = e % L;
      const size_t o = (((size_t)kk * 2 + c) * L + up) * LP + u;
      BX[o] = make_double2(0, 0);
      BY[o] = make_double2(0, 0);
    }
    return;
  }
  if (threadIdx.x == 0) {
    double2 hh[Q];
    hankel_up<double, Q>(k * rho, hh);
    const double z = k * rho;
    for (int q = 0; q < Q; ++q) {
      h[q] = hh[q];
      // h_q'(z) = h_{q-1}(z) - (q + 1) / z h_q(z), h_0' = -h_1
      double2 d;
      if (q == 0) d = make_double2(-hh[1].x, -hh[1].y);
      else d = make_double2(hh[q - 1].x - (q + 1) / z * hh[q].x, hh[q - 1].y - (q + 1) / z * hh[q].y);
      hp[q] = make_double2(k * d.x, k * d.y);
    }
    double2 e1 = make_double2(dx / rho, dy / rho), e = make_double2(1, 0);
    for (int mu = 0; mu <= 2 * NMAX; ++mu) {
      eph[2 * NMAX + mu] = e;
      eph[2 * NMAX - mu] = cconj(e);
      e = cmul(e, e1);
    }
  }
  __syncthreads();
  const double w = taper_weight(rho, cutoff, taper), wp = taper_dweight(rho, cutoff, taper);
  const double cphi = dx / rho, sphi = dy / rho;
  for (int e = threadIdx.x; e < 2 * L * L; e += blockDim.x) {
    const int c = e / (L * L), u = (e / L) % L, up = e % L;
    const double2* g = G + ((size_t)(c * L + u) * L + up) * Q;
    double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      cfma(s0, g[q], h[q]);
      cfma(s1, g[q], hp[q]);
    }
    const int mu = mval[c * L + up] - mval[c * L + u];
    const double2 E = eph[2 * NMAX + mu];
    const double2 b0 = cmul(E, s0), b1 = cmul(E, s1);
    // d rho / d dx = cos phi, d phi / d dx = -sin phi / rho; d rho / d dy = sin phi, d phi / d dy = cos phi / rho
    const double2 imb0 = make_double2(-mu * b0.y, mu * b0.x);  // i mu b0
    const double2 dbx = make_double2(wp * cphi * b0.x + w * (cphi * b1.x - sphi / rho * imb0.x),
                                     wp * cphi * b0.y + w * (cphi * b1.y - sphi / rho * imb0.y));
    const double2 dby = make_double2(wp * sphi * b0.x + w * (sphi * b1.x + cphi / rho * imb0.x),
                                     wp * sphi * b0.y + w * (sphi * b1.y + cphi / rho * imb0.y));
    const size_t o = (((size_t)kk * 2 + c) * L + up) * LP + u;
    BX[o] = dbx;
    BY[o] = dby;
  }
}

__global__ void fill_one_kernel(double2* __restrict__ x, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = make_double2(1.0, 0.0);
}

// grad[i][q] = 2 Re sum_u [ tmu (ys_q) - (tmu - yz_q) s + tmu da0_q ]  (internal layout)
//              - Re sum_f s_api (vp_q - vm_q) / h                       (API layout)
__global__ void posgrad_kernel(const double2* __restrict__ tmu, const double2* __restrict__ s,
                               const double2* __restrict__ ys, const double2* __restrict__ yz,
                               const double2* __restrict__ da0, const double2* __restrict__ s_api,
                               const double2* __restrict__ vpm, double inv_h, int64_t N, int P,
                               double* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t NP = N * P;
  for (int q = 0; q < 2; ++q) {
    double acc = 0.0, ex = 0.0;
    for (int u = 0; u < P; ++u) {
      const int64_t o = i * P + u;
      const double2 t = tmu[o];
      double2 g = cmul(t, ys[q * NP + o]);
      const double2 atz = make_double2(t.x - yz[q * NP + o].x, t.y - yz[q * NP + o].y);  // (A'^T T mu)
      g = csub(g, cmul(atz, s[o]));
      if (da0) g = cadd(g, cmul(t, da0[q * NP + o]));
      acc += g.x;
      const double2 dv = csub(vpm[(2 * q) * NP + o], vpm[(2 * q + 1) * NP + o]);
      ex += cmul(s_api[o], dv).x;
    }
    grad[2 * i + q] = 2.0 * acc - ex * inv_h;
  }
}

}  // namespace tmat

extern "C" int tmat_position_gradient(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* mu,
                                      const tmat_c128* da0_dx, const tmat_c128* da0_dy, const double* x_f,
                                      const tmat_c128* E_f, double* grad_out) {
  if (!ctx) return TMAT_EINVAL;
  if (!sol || !mu || !x_f || !E_f || !grad_out || ((da0_dx == nullptr) != (da0_dy == nullptr)))
    return set_error(ctx, TMAT_EINVAL, "tmat_position_gradient: bad arguments");
  if (sol->device != ctx->device)
    return set_error(ctx, TMAT_EINVAL, "tmat_position_gradient: solution is on another device");
  if (sol->path != TMAT_PATH_LATTICE || sol->tblocks)
    return set_error(ctx, TMAT_ENOTSUP, "tmat_position_gradient: lattice solutions with diagonal T only");
  Tables* t;
  TM_TRY(get_tables(ctx, sol->nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t N = sol->N;
  const int P = t->P, L = t->L;
  if (N == 0) return TMAT_OK;
  Staged smu, sdx, sdy, sxf, sef, sg;
  TM_TRY(stage_in(ctx, "st_mu_in", mu, sizeof(double2) * N * P, &smu));
  TM_TRY(stage_in(ctx, "st_da0x", da0_dx, da0_dx ? sizeof(double2) * N * P : 0, &sdx));
  TM_TRY(stage_in(ctx, "st_da0y", da0_dy, da0_dy ? sizeof(double2) * N * P : 0, &sdy));
  TM_TRY(stage_in(ctx, "st_xf", x_f, sizeof(double) * 3, &sxf));
  TM_TRY(stage_in(ctx, "st_ef", E_f, sizeof(double2) * 3, &sef));
  TM_TRY(stage_out(ctx, "st_pgrad", grad_out, sizeof(double) * 2 * N, &sg));
  OpPair ops;
  TM_TRY(make_lattice_ops(ctx, t, sol->pos, N, sol->k, sol->lattice_nx, sol->lattice_ny, sol->lattice_pitch,
                          sol->cutoff, sol->taper, sol->T64, nullptr, false, &ops, 0));
  const LatOp& a = ops.lat64;
  const size_t nblk = (size_t)std::max(a.K, 1) * 2 * L * a.LP;
  double2 *BX, *BY, *one, *mui, *tmu, *da0, *ys, *yz, *s_api, *vpm, *xf4;
  TM_TRY(scratch(ctx, "pg_BX", sizeof(double2) * nblk, (void**)&BX));
  TM_TRY(scratch(ctx, "pg_BY", sizeof(double2) * nblk, (void**)&BY));
  TM_TRY(scratch(ctx, "pg_one", sizeof(double2) * N * P, (void**)&one));
  TM_TRY(scratch(ctx, "pg_mu", sizeof(double2) * N * P, (void**)&mui));
  TM_TRY(scratch(ctx, "pg_tmu", sizeof(double2) * N * P, (void**)&tmu));
  TM_TRY(scratch(ctx, "pg_da0", sizeof(double2) * 2 * N * P, (void**)&da0));
  TM_TRY(scratch(ctx, "pg_ys", sizeof(double2) * 2 * N * P, (void**)&ys));
  TM_TRY(scratch(ctx, "pg_yz", sizeof(double2) * 2 * N * P, (void**)&yz));
  TM_TRY(scratch(ctx, "pg_sapi", sizeof(double2) * N * P, (void**)&s_api));
  TM_TRY(scratch(ctx, "pg_vpm", sizeof(double2) * 4 * N * P, (void**)&vpm));
  TM_TRY(scratch(ctx, "pg_xf4", sizeof(double) * 12 + 64, (void**)&xf4));
  if (a.K > 0) {
    switch (sol->nmax) {
#define DB(NM)                                                                                                    \
  case NM:                                                                                                        \
    lattice_dblocks_kernel<NM><<<a.K, 256, 0, ctx->stream>>>(a.off, a.K, sol->lattice_pitch, sol->k, sol->cutoff, \
                                                             sol->taper, t->d_gdense, t->d_mval, a.LP, BX, BY);   \
    break;
      DB(1) DB(2) DB(3) DB(4) DB(5) DB(6)
#undef DB
    }
    TM_LAUNCHED(ctx);
  }
  fill_one_kernel<<<(unsigned)cdiv(N * P, 256), 256, 0, ctx->stream>>>(one, N * P);
  TM_LAUNCHED(ctx);
  TM_TRY(to_internal(ctx, t, (const double2*)smu.dev, mui, false, N));
  tdiag_mul_kernel<<<(unsigned)cdiv(N * P, 256), 256, 0, ctx->stream>>>(sol->T64, mui, tmu, N * P, N * P);
  TM_LAUNCHED(ctx);
  if (da0_dx) {
    TM_TRY(to_internal(ctx, t, (const double2*)sdx.dev, da0, false, N));
    TM_TRY(to_internal(ctx, t, (const double2*)sdy.dev, da0 + N * P, false, N));
  }
  // (A'_q s) and T mu - A'_q^T (1 . T mu) for q = x, y: by FFT convolution with their own
  // block spectra where the operator's grid fits (the dy-derivative blocks are odd under the
  // y mirror), else on the fp64 CUDA-core lattice kernel
  for (int q = 0; q < 2; ++q) {
    LatOp d = a;
    d.BT = q == 0 ? BX : BY;
    d.T = one;
    d.use_oz = false;
    d.use_tc = false;
    d.fp32 = false;
    d.fft_mirror_sign = q == 0 ? 1 : -1;
    d.fft_quad_ok = false;  // dF/dd is odd under d -> -d: no quad form
    if (a.use_fft) TM_TRY(lattice_fft_prepare(ctx, &d, q == 0 ? "pg_Bh_x" : "pg_Bh_y"));
    TM_TRY(lattice_apply(ctx, d, TMAT_OP_COUPLE, sol->s, ys + q * N * P, 1));
    TM_TRY(lattice_apply(ctx, d, TMAT_OP_ADJOINT, tmu, yz + q * N * P, 1));
  }
  // explicit term: v at the focal point moved by +-h along x and y, with E fixed
  TM_TRY(from_internal(ctx, t, sol->s, false, s_api, N));
  double hxf[3];
  TM_CUDA(ctx, cudaMemcpyAsync(hxf, sxf.dev, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double hstep = 1e-4 / sol->k;
  double pts[12];
  for (int j = 0; j < 4; ++j) {
    for (int c = 0; c < 3; ++c) pts[3 * j + c] = hxf[c];
    pts[3 * j + j / 2] += (j % 2 == 0) ? hstep : -hstep;  // +x, -x, +y, -y
  }
  double* dpts = (double*)xf4;
  TM_CUDA(ctx, cudaMemcpyAsync(dpts, pts, sizeof(pts), cudaMemcpyHostToDevice, ctx->stream));
  for (int j = 0; j < 4; ++j)
    TM_TRY(adjoint_source_dev(ctx, sol->pos, N, sol->k, sol->nmax, dpts + 3 * j, (const double2*)sef.dev,
                              vpm + j * N * P));
  posgrad_kernel<<<(unsigned)cdiv(N, 128), 128, 0, ctx->stream>>>(tmu, sol->s, ys, yz, da0_dx ? da0 : nullptr, s_api,
                                                                   vpm, 1.0 / hstep, N, P, (double*)sg.dev);
  TM_LAUNCHED(ctx);
  TM_TRY(finish_out(ctx, &sg));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // pts is a host stack array
  return TMAT_OK;
}
