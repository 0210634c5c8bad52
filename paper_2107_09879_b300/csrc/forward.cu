// One forward simulation in a single call (App. I): T-matrices, incident coefficients,
// the solve and the fields, with the intermediates kept in device scratch.
#include "internal.h"

using namespace tmat;

extern "C" int tmat_forward(tmat_ctx* ctx, const double* pos, int64_t N, const tmat_atom* atoms, double wavelength,
                            double n_bg, int nmax, const double* dirs, const tmat_c128* pol, int R,
                            const tmat_solve_opts* opts, const double* pts, int64_t M, tmat_c128* s_out,
                            tmat_c128* E_out, tmat_solve_info* info) {
  if (!ctx) return TMAT_EINVAL;
  if (N <= 0 || !pos || !atoms || !dirs || !pol || !opts) return set_error(ctx, TMAT_EINVAL, "tmat_forward: bad arguments");
  if (R < 1 || R > TMAT_MAX_RHS) return set_error(ctx, TMAT_EINVAL, "tmat_forward: R = %d outside 1..%d", R, TMAT_MAX_RHS);
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "tmat_forward: nmax %d", nmax);
  if (M < 0 || (M > 0 && (!pts || !E_out))) return set_error(ctx, TMAT_EINVAL, "tmat_forward: bad field points");
  const int64_t P = num_coeffs(nmax);
  const size_t vec = sizeof(tmat_c128) * (size_t)N * P;
  Staged spos, satoms, sdirs, spol, spts, ss, sE;
  TM_TRY(stage_in(ctx, "fwd_pos", pos, sizeof(double) * 3 * (size_t)N, &spos));
  TM_TRY(stage_in(ctx, "fwd_atoms", atoms, sizeof(tmat_atom) * (size_t)N, &satoms));
  TM_TRY(stage_in(ctx, "fwd_dirs", dirs, sizeof(double) * 2 * (size_t)R, &sdirs));
  TM_TRY(stage_in(ctx, "fwd_pol", pol, sizeof(tmat_c128) * 3 * (size_t)R, &spol));
  TM_TRY(stage_in(ctx, "fwd_pts", M > 0 ? pts : nullptr, sizeof(double) * 3 * (size_t)M, &spts));
  void *T = nullptr, *a0 = nullptr;
  TM_TRY(scratch(ctx, "fwd_T", vec, &T));
  TM_TRY(scratch(ctx, "fwd_a0", vec * R, &a0));
  if (s_out) {
    TM_TRY(stage_out(ctx, "fwd_s", s_out, vec * R, &ss));
  } else {
    TM_TRY(scratch(ctx, "fwd_s", vec * R, &ss.dev));
  }
  TM_TRY(stage_out(ctx, "fwd_E", M > 0 ? E_out : nullptr, sizeof(tmat_c128) * 3 * (size_t)M * R, &sE));
  const double* d_pos = (const double*)spos.dev;
  TM_TRY(tmat_build(ctx, (const tmat_atom*)satoms.dev, N, wavelength, n_bg, nmax, (tmat_c128*)T, nullptr));
  TM_TRY(tmat_incident_planewave(ctx, d_pos, N, wavelength, n_bg, nmax, (const double*)sdirs.dev,
                                 (const tmat_c128*)spol.dev, R, (tmat_c128*)a0));
  tmat_c128* s = (tmat_c128*)ss.dev;
  const int rc = tmat_solve(ctx, d_pos, N, wavelength, n_bg, nmax, (const tmat_c128*)T, (const tmat_c128*)a0, R, opts,
                            s, nullptr, info);
  if (rc != TMAT_OK && rc != TMAT_ENOCONV) return rc;
  // a host solution buffer is filled on the side stream while the fields are computed
  const bool s_aside = s_out && ss.host && M > 0;
  if (s_aside) {
    TM_TRY(aux_stream_ready(ctx));
    TM_CUDA(ctx, cudaEventRecord(ctx->aux_event, ctx->stream));
    TM_CUDA(ctx, cudaStreamWaitEvent(ctx->aux_stream, ctx->aux_event, 0));
    TM_CUDA(ctx, cudaMemcpyAsync(s_out, ss.dev, ss.bytes, cudaMemcpyDeviceToHost, ctx->aux_stream));
  }
  int frc = TMAT_OK;
  if (M > 0) {
    for (int r = 0; r < R && frc == TMAT_OK; ++r)
      frc = tmat_field(ctx, d_pos, N, wavelength, n_bg, nmax, s + (int64_t)r * N * P, (const double*)spts.dev, M,
                       (tmat_c128*)sE.dev + (int64_t)r * M * 3);
  }
  if (frc == TMAT_OK && s_out && !s_aside) frc = finish_out(ctx, &ss);
  if (frc == TMAT_OK) frc = finish_out(ctx, &sE);
  if (s_aside) TM_CUDA(ctx, cudaStreamSynchronize(ctx->aux_stream));  // the copy ends before the scratch is reused
  return frc != TMAT_OK ? frc : rc;
}
