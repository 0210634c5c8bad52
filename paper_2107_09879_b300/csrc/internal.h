// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/tmat.h"

namespace tmat {

// Constant tables of one multipole order (built on the host once per nmax).
//
// Planar tables: for coplanar scatterers the translation blocks split exactly
// into two classes c = (l + m + p) mod 2 (entries linking different classes
// vanish because Pbar_q^{|mu|}(0) = 0 for q + mu odd and (l l' q; 0 0 0) = 0 for
// l + l' + q odd). Inside a class, output u couples to input u' through
//    B[u,u'] = sum_q G[u,u',q] h_q(k d),
// with G real for equal polarisations (alpha part) and imaginary for different
// ones (beta part); the azimuthal phases are applied to the vectors.
struct Tables {
  int nmax = 0, L = 0, P = 0, Q = 0;  // Q = 2 nmax + 1 Hankel orders
  // class-split order: member u of class c is flat index perm[c*L + u]
  std::vector<int> perm;  // [2L] internal -> flat
  std::vector<int> mval;  // [2L] azimuthal m of each internal index
  int* d_perm = nullptr;
  int* d_mval = nullptr;
  // planar coupling triples, per op (0 = forward, 1 = adjoint), host only:
  //   seg[op][(c*L+u)*(Q+1) + q] .. [.. + 1] index the triples of output (c,u), order q
  //   tri_idx: input index u' | (imag << 15); tri_val: the real factor
  int n_tri[2] = {0, 0};
  std::vector<int> seg[2], tri_idx[2];
  std::vector<double> tri_val[2];
  // the same triples for the pair-sum apply, per op: zseg[o] .. zseg[o+1] index the
  // entries of internal output o; zidx = column (c*L+u') | combination a << 8 | imag << 16
  // with a = q(q+1)/2 + (mu+q)/2; zval the real factor (times i where imag)
  std::vector<int> zseg[2], zidx[2];
  std::vector<double> zval[2];
  int* d_zseg[2] = {nullptr, nullptr};
  int* d_zidx[2] = {nullptr, nullptr};
  float* d_zval_f32[2] = {nullptr, nullptr};
  double* d_zval_f64[2] = {nullptr, nullptr};
  // the same off the plane: every (n, n') pair of the full block, combination
  // a = q^2 + mu + q (no class split; columns in the internal order)
  std::vector<int> z3seg[2], z3idx[2];
  std::vector<double> z3val[2];
  int* d_z3seg[2] = {nullptr, nullptr};
  int* d_z3idx[2] = {nullptr, nullptr};
  float* d_z3val_f32[2] = {nullptr, nullptr};
  double* d_z3val_f64[2] = {nullptr, nullptr};
  // dense planar forward coefficients G[c][u][u'][q] as complex (alpha real, beta imaginary)
  double2* d_gdense = nullptr;
  // full (3-D) coupling constants a5/b5 as complex [L][L][Q] (zero where absent)
  double2* d_a5 = nullptr;
  double2* d_b5 = nullptr;
};

// A device buffer the context owns and grows on demand.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace tmat

struct tmat_ctx {
  // mixed solves: inner solves with tolerance >= 1e-2 store the final Krylov vectors as
  // scaled fp16 (tmat_ctx_set_compressed_basis)
  bool compress_basis = true;
  // kernel timing (off by default): event pairs recorded around operator launches; with
  // timing_every = n > 1 only one Arnoldi iteration in n of the complex64 inner solves is
  // timed (timing_skip marks the others), every call is still counted
  bool timing = false;
  int timing_every = 1;
  bool timing_skip = false;
  int64_t timing_iter = 0;
  std::map<std::string, int64_t> timed_calls;
  std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> timed;
  std::vector<cudaEvent_t> event_pool;          // recycled timing events
  std::map<std::string, double> timed_bytes;    // algorithmic bytes of the timed launches
  std::map<const void*, int> occupancy;         // resident CTAs per SM queried per kernel (fixed shapes)
  int device = 0;
  cudaStream_t stream = nullptr;
  char err[512] = {0};
  int64_t launches = 0;
  std::map<int, tmat::Tables*> tables;
  std::map<std::string, tmat::DevBuf> bufs;
  int num_sms = 148;
  bool tensor_cores = true;  // use the tcgen05 kernels where they exist
  int tc_variant = 0;        // 0: window-view kernel where it fits, 1: gather kernel
  bool lattice_fft = true;   // lattice operators by FFT convolution where the grid fits
  bool fft_quad = true;      // complex64 FFT block products in the quad-mirror form
  bool field_mixed = false;  // near fields in fp32 with fp64 phases (tmat_ctx_set_field_precision)
  void* pinned = nullptr;  // small pinned host staging area (status words)
  cudaEvent_t flag_event = nullptr;  // marks the copy of convergence flags into `pinned`
  // mapped pinned words the Arnoldi step kernel publishes its convergence flags to:
  // [0, TMAT_MAX_RHS) active flags, [TMAT_MAX_RHS, 2 TMAT_MAX_RHS) the tag of the step
  int* flag_host = nullptr;
  int* flag_dev = nullptr;
  int flag_tag = 0;
  // a second stream (created on first use) for copies that overlap work on `stream`
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_event = nullptr;
};

namespace tmat {

int set_error(tmat_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(tmat_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);
#define TM_CUDA(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) return ::tmat::cuda_fail((ctx), _e, #call, __FILE__, __LINE__); \
  } while (0)
// after a kernel launch: check the launch itself and count it
#define TM_LAUNCHED(ctx)                                                                                 \
  do {                                                                                                   \
    (ctx)->launches++;                                                                                   \
    cudaError_t _e = cudaGetLastError();                                                                 \
    if (_e != cudaSuccess) return ::tmat::cuda_fail((ctx), _e, "kernel launch", __FILE__, __LINE__); \
  } while (0)
#define TM_TRY(x)                   \
  do {                              \
    int _rc = (x);                  \
    if (_rc != TMAT_OK) return _rc; \
  } while (0)

// Kernel timing: returns a start event (or nullptr when timing is off) and
// records the matching stop event after the launch.
cudaEvent_t timing_begin(tmat_ctx* ctx);
// bytes: the launch's algorithmic traffic (what it must read and write), summed per kind
void timing_end(tmat_ctx* ctx, const char* kind, cudaEvent_t start, double bytes = 0.0);

// Grow-only scratch owned by the context, keyed by name.
int scratch(tmat_ctx* ctx, const char* name, size_t bytes, void** out);
// Enclosing-sphere overlap check of N scatterers (device arrays): TMAT_OK or TMAT_EOVERLAP
// with the first intersecting pair in pair_out[2] (nullable); synchronises.
int check_overlap(tmat_ctx* ctx, const double* d_pos, const double* d_rad, int64_t N, int64_t* pair_out);
// Tables of order nmax (built and uploaded on first use).
int get_tables(tmat_ctx* ctx, int nmax, Tables** out);
void free_tables(Tables* t);

// Host/device pointer staging. An input that is host memory is copied to a
// scratch buffer; an output that is host memory gets a scratch buffer and is
// copied back by finish_out().
bool is_device_ptr(const void* p);
// Raise a kernel's dynamic shared memory limit once per context (the driver call is not free).
int set_smem_limit(tmat_ctx* ctx, const void* func, size_t bytes);
struct Staged {
  const void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool host = false;
};
int stage_in(tmat_ctx* ctx, const char* name, const void* user, size_t bytes, Staged* s);
int stage_out(tmat_ctx* ctx, const char* name, void* user, size_t bytes, Staged* s);
int finish_out(tmat_ctx* ctx, Staged* s);
// The side stream and its event, created once per context.
int aux_stream_ready(tmat_ctx* ctx);

__host__ __device__ inline int num_coeffs(int nmax) { return 2 * nmax * (nmax + 2); }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Host-side constant generators (tables.cpp).
double wigner3j_host(int j1, int j2, int j3, int m1, int m2, int m3);
void coupling_a5b5(int l, int m, int lp, int mp, int q, double2* a, double2* b);
double pbar_at_zero(int q, int mu);  // normalised Legendre Pbar_q^mu(0), mu >= 0

}  // namespace tmat
