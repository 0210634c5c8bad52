// Operator descriptors shared by the apply kernels and the solver.
#pragma once
#include "internal.h"

namespace tmat {

// Neighbour-list operator: positions, T in internal layout and precision, CSR.
struct NbrOp {
  const double* pos = nullptr;  // [N][3] device
  int64_t N = 0;
  double k = 0;
  int nmax = 0;
  bool fp32 = false;
  const void* T = nullptr;      // [N][P] internal layout, complex64 if fp32 else complex128
  const int64_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const Tables* tab = nullptr;
  double cutoff = 0, taper = 0;  // coupling window (taper 0: hard cutoff)
  bool threed = false;           // positions not coplanar: full 3-D blocks (apply_nbr3d_kernel)
};

int nbr_apply(tmat_ctx* ctx, const NbrOp& a, int op, const void* x, void* y, int R);

// layout conversion between the API order (flat p*L + n) and the internal
// class-split order, with precision conversion; `rows` rows of P coefficients.
int to_internal(tmat_ctx* ctx, const Tables* t, const double2* api, void* internal, bool fp32, int64_t rows);
int from_internal(tmat_ctx* ctx, const Tables* t, const void* internal, bool fp32, double2* api, int64_t rows);

// flags: bit 0 some z differs from pos[2] (not coplanar), bit 1 a non-finite coordinate
// (synchronises)
int position_flags(tmat_ctx* ctx, const double* d_pos, int64_t N, int* flags);

}  // namespace tmat
