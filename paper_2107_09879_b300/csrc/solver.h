// Solver-side declarations: operator dispatch and the GMRES engine.
#pragma once
#include "apply.h"
#include "internal.h"

namespace tmat {

// An operator instance in one precision. kind 0: neighbour list; kind 1: lattice.
struct LatOp;
struct Operator {
  int kind = 0;
  NbrOp nbr;
  const LatOp* lat = nullptr;
  bool fp32() const;
  int64_t N() const;
  int nmax() const;
};
int op_apply(tmat_ctx* ctx, const Operator& A, int mode, const void* x, void* y, int R);

struct GmresParams {
  double tol = 1e-6;
  int restart = 40;
  int max_iter = 2000;
};
struct GmresStats {
  int iterations = 0;
  bool converged = false;
  double rel_res[TMAT_MAX_RHS] = {0};
  bool breakdown = false;
};

// Solve K x = b (K = op in `mode`) for R RHS; b, x internal layout, complex128.
// prec: TMAT_PREC_FP64 uses A64 only; TMAT_PREC_MIXED refines with A32 inside.
struct SolveParams {
  int precision = TMAT_PREC_FP64;
  double tol = 1e-6;
  double inner_tol = 1e-4;
  int restart = 40;
  int max_iter = 2000;
};
struct SolveStats {
  int iterations = 0;
  int refinements = 0;
  bool converged = false;
  double rel_res[TMAT_MAX_RHS] = {0};
};
int solve_system(tmat_ctx* ctx, const Operator& A64, const Operator* A32, int mode, const double2* b, double2* x,
                 int R, const SolveParams& p, SolveStats* st);

int prepare_T(tmat_ctx* ctx, const Tables* t, const double2* T_api, int64_t N, bool fp32, const char* name, void** out);

}  // namespace tmat
