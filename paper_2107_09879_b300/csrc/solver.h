// Solver-side declarations: operator dispatch and the GMRES engine.
#pragma once
#include "apply.h"
#include "internal.h"

namespace tmat {

// Lattice operator: row-major nx x ny lattice, one translation block per
// lattice offset o = (dx, dy) (source site = target site + o), stored transposed
// per class: BT[o][c][u'][u] = A_o[c][u][u'] (row stride LP complex).
struct LatOp {
  int64_t N = 0;
  int nx = 0, ny = 0;
  int nmax = 0, L = 0, P = 0, LP = 0;
  bool fp32 = false;
  int K = 0;                   // number of offsets
  const int2* off = nullptr;   // [K] (dx, dy)
  const int* neg = nullptr;    // [K] index of -o
  const void* BT = nullptr;    // [K][2][L][LP] complex64 or complex128
  const void* T = nullptr;     // [N][P] internal layout, kernel precision
  // tensor-core (tcgen05, 3xTF32) variant of the complex64 apply
  bool use_tc = false;
  const void* Wtc_fwd = nullptr;  // split W tables in MMA core layout, forward
  const void* Wtc_adj = nullptr;  // and adjoint
  int* tc_err = nullptr;          // device counter of CTAs that gave up on a wait
  const int* dy_start = nullptr;  // [ndy + 1] first offset of each dy (offsets sorted by dy, dx)
  int ndy = 0;
  int CX = 0;                     // max |dx| over the offsets
  int CY = 0;                     // max |dy| over the offsets
  bool tc2 = false;               // window-view tensor-core kernel usable
  // fp64-class apply on the tensor cores (bf16 slices, exact group sums)
  bool use_oz = false;
  int* oz_err = nullptr;  // device counter of CTAs that gave up on a wait
  // FFT convolution (lattice_fft.cu): grid size and the block spectra B^[2 L L][Mx My]
  bool use_fft = false;
  int fft_Mx = 0, fft_My = 0;
  const void* fft_Bhat = nullptr;
  // [2][L] per class member u: J(u) | p(u) << 16, J the m -> -m partner in the class and p
  // the polarisation; B_(dx,-dy) = D J B_(dx,dy) J D with D = diag((-1)^p)
  const int* fft_mirror = nullptr;
  // +1, or -1 for blocks odd in dy (the dy-derivative blocks): B_(dx,-dy) = -D J B J D
  int fft_mirror_sign = 1;
  // [2][L] per class member u: J(u) | (m mod 2) << 16 | p << 17 (quad-mirror block product)
  const int* fft_sym = nullptr;
  // quad-mirror form of the spectra (complex64, or double-float pairs for complex128
  // operators): per item (kx <= Mx/2, ky <= My/2) and class the symmetric matrix
  // C = B^(kx, ky) S, S = J diag((-1)^m), item-major [items][2][L][L]
  const void* fft_C = nullptr;
  // the blocks obey reciprocity and inversion symmetry (the quad form needs both; the
  // position-derivative blocks are odd under inversion)
  bool fft_quad_ok = true;
  int* fft_err = nullptr;  // device counter of CTAs that gave up on a bounded wait
  // batched operators (one independent problem per RHS, FFT path): per-RHS strides, in
  // complex values, of T ([R][N][P]), of the block spectra and of the quad-form spectra;
  // 0 = one operator shared by every RHS
  int64_t t_stride = 0, fft_bstride = 0, fft_cstride = 0;
};
// An operator instance in one precision. kind 0: neighbour list; kind 1: lattice.
struct Operator {
  int kind = 0;
  NbrOp nbr;
  const LatOp* lat = nullptr;
  // full per-scatterer T-blocks (internal index order, the operator's precision). When set,
  // the operator above carries T = 1 and op_apply multiplies by the blocks:
  //   forward y = x - T (A x); transposed y = x - A^T (T^T x); coupling y = A x.
  // tbc[(type P + c) P + a] = T[a][c] (for T z), tbr[(type P + c) P + a] = T[c][a] (for T^T x)
  const void* tbc = nullptr;
  const void* tbr = nullptr;
  const int32_t* ttype = nullptr;  // [N] block of each scatterer
  bool fp32() const;
  int64_t N() const;
  int nmax() const;
};
int op_apply(tmat_ctx* ctx, const Operator& A, int mode, const void* x, void* y, int R);

struct GmresParams {
  double tol = 1e-6;
  int restart = 40;
  int max_iter = 2000;
  bool compress_basis = false;  // complex64 operator: final basis vectors stored as scaled fp16
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
// res64 (nullable): operator of the mixed solve's fp64-accurate refinement residual
// (default A64).
int solve_system(tmat_ctx* ctx, const Operator& A64, const Operator* A32, int mode, const double2* b, double2* x,
                 int R, const SolveParams& p, SolveStats* st, const Operator* res64 = nullptr);

int prepare_T(tmat_ctx* ctx, const Tables* t, const double2* T_api, int64_t N, bool fp32, const char* name, void** out);
// out[r][i][a] = sum_c Tm[(type_i P + c) P + a] in[r][i][c]; with xsub: xsub - that
int tblock_mul(tmat_ctx* ctx, const void* Tm, const int32_t* type, const void* in, const void* xsub, void* out,
               int64_t N, int P, int R, bool fp32);

}  // namespace tmat

namespace tmat {
int build_neighbors(tmat_ctx* ctx, const double* d_pos, int64_t N, double cutoff, int64_t* d_row_ptr, int32_t* d_col,
                    int64_t* nnz_out);
int lattice_apply(tmat_ctx* ctx, const LatOp& L, int mode, const void* x, void* y, int R);
bool lattice_tc_supported(int nmax);
bool lattice_tc_fits(int nmax, int CX);
bool lattice_tc2_fits(int nmax, int CX);
int lattice_tc2_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R);
int lattice_tc_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R);
int lattice_tc_prepare(tmat_ctx* ctx, LatOp* a, const double2* BT64);
bool lattice_fft_fits(int nx, int ny, int CX, int CY);
// name: the scratch buffer of the block spectra (default: one per precision and context)
int lattice_fft_prepare(tmat_ctx* ctx, LatOp* a, const char* name = nullptr);
int lattice_fft_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R);
bool lattice_oz_fits(int nmax, int CX);
int lattice_oz_prepare(tmat_ctx* ctx, LatOp* a, const double2* BT64);
int lattice_oz_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R);
inline int64_t lattice_N(const LatOp& L) { return L.N; }
inline int lattice_nmax(const LatOp& L) { return L.nmax; }
inline bool lattice_fp32(const LatOp& L) { return L.fp32; }
// Operators (fp64 and, for mixed, fp32) for one solve.
// R64: the fp64-class tensor-core operator (have_oz), for refinement residuals (when the
// fp64 operator is not the FFT one) and TMAT_PREC_FP64_TC solves. want_oz: 0 none,
// 1 for a refinement residual, 2 for TMAT_PREC_FP64_TC.
struct OpPair {
  Operator A64, A32, R64;
  bool have32 = false, have_oz = false;
  LatOp lat64, lat32, lat64oz;
};
int adjoint_source_dev(tmat_ctx* ctx, const double* pos, int64_t N, double k, int nmax, const double* xf,
                       const double2* E, double2* v);
int make_lattice_ops(tmat_ctx* ctx, const Tables* t, const double* d_pos, int64_t N, double k, int nx, int ny,
                     double pitch, double cutoff, double taper, const double2* T64, const float2* T32, bool mixed,
                     OpPair* ops, int want_oz = 0);
}  // namespace tmat
