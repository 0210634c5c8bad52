// Lattice path of the operator apply. On a rectangular lattice the translation
// block of a pair depends only on the lattice offset o = source - target, so
// one block per offset inside the cutoff is generated (App. I-C, Eqs.
// tran_coeff, in fp64) and reused by every pair with that offset: the apply
// becomes a block-Toeplitz product
//     (A x)_i = sum_o A_o x_{i+o}   (i + o inside the lattice),
// which is a dense contraction with no per-pair generation left.
//
// Kernel mapping: one thread per target site (consecutive sites per warp, so
// a warp's sources for one offset are consecutive too); each thread keeps UPT
// outputs x NR right-hand sides in registers; the offset's block is staged in
// shared memory (double-buffered) and read as broadcasts; the source's inputs
// stream from L1/L2 one coefficient at a time (outer-product order).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "dev.cuh"
#include "solver.h"

namespace tmat {

// ---- block generation ---------------------------------------------------------
// BT[k][c][u'][u] = e^{i(m_u' - m_u) phi} sum_q G[c][u][u'][q] h_q(k rho), with
// d = x_target - x_source = -(dx, dy) * pitch, rho = |d|, phi = angle of d.
template <int NMAX>
__global__ void lattice_blocks_kernel(const int2* __restrict__ off, int K, double pitch, double k, double cutoff,
                                      double taper, const double2* __restrict__ G, const int* __restrict__ mval,
                                      int LP, double2* __restrict__ B64, float2* __restrict__ B32) {
  constexpr int L = NMAX * (NMAX + 2), Q = 2 * NMAX + 1;
  __shared__ double2 h[Q];
  __shared__ double2 eph[2 * (2 * NMAX) + 1];  // e^{i mu phi}, mu = -2NMAX..2NMAX
  const int kk = blockIdx.x;
  if (kk >= K) return;
  const double dx = -(double)off[kk].x * pitch, dy = -(double)off[kk].y * pitch;
  const double rho = sqrt(dx * dx + dy * dy);
  if (off[kk].x == 0 && off[kk].y == 0) {  // the self offset: no coupling
    for (int e = threadIdx.x; e < 2 * L * L; e += blockDim.x) {
      const int c = e / (L * L), u = (e / L) % L, up = e % L;
      const size_t o = (((size_t)kk * 2 + c) * L + up) * LP + u;
      B64[o] = make_double2(0, 0);
      if (B32) B32[o] = make_float2(0.f, 0.f);
    }
    return;
  }
  if (threadIdx.x == 0) {
    double2 hh[Q];
    hankel_up<double, Q>(k * rho, hh);
    for (int q = 0; q < Q; ++q) h[q] = hh[q];
    double2 e1 = make_double2(dx / rho, dy / rho), e = make_double2(1, 0);
    for (int mu = 0; mu <= 2 * NMAX; ++mu) {
      eph[2 * NMAX + mu] = e;
      eph[2 * NMAX - mu] = cconj(e);
      e = cmul(e, e1);
    }
  }
  __syncthreads();
  const double wgt = taper_weight(rho, cutoff, taper);
  for (int e = threadIdx.x; e < 2 * L * L; e += blockDim.x) {
    const int c = e / (L * L), u = (e / L) % L, up = e % L;
    const double2* g = G + ((size_t)(c * L + u) * L + up) * Q;
    double2 acc = make_double2(0, 0);
#pragma unroll
    for (int q = 0; q < Q; ++q) cfma(acc, g[q], h[q]);
    const int mu = mval[c * L + up] - mval[c * L + u];
    acc = cscale(cmul(acc, eph[2 * NMAX + mu]), wgt);
    const size_t o = (((size_t)kk * 2 + c) * L + up) * LP + u;
    B64[o] = acc;
    if (B32) B32[o] = to_c64(acc);
  }
}

// ---- apply -------------------------------------------------------------------
constexpr int LAT_THREADS = 128;
#ifndef LAT_MIN_BLOCKS
#define LAT_MIN_BLOCKS 1  // resident blocks per SM the register budget is sized for
#endif

template <typename R> struct LatCfg;
// outputs per thread so that UPT * NR complex accumulators stay ~<= 48 complex (fp32) / 24 (fp64)
template <typename R, int L, int NR>
struct Split {
  static constexpr int budget = sizeof(R) == 4 ? 48 : 12;
  static constexpr int S = (L * NR + budget - 1) / budget;
  static constexpr int UPT = (L + S - 1) / S;
};

// MODE 0: y = x - T (A x); 1: y = x - A^T (T x); 2: y = A x
template <typename R, int NMAX, int NR, int MODE>
__global__ void __launch_bounds__(LAT_THREADS, LAT_MIN_BLOCKS)
lattice_apply_kernel(const int2* __restrict__ off, const int* __restrict__ neg, int K, int nx, int ny, int64_t N,
                     const C<R>* __restrict__ BT, int LP, const C<R>* __restrict__ T, const C<R>* __restrict__ x,
                     C<R>* __restrict__ y, int64_t rstride) {
  constexpr int L = NMAX * (NMAX + 2), P = 2 * L;
  constexpr int S = Split<R, L, NR>::S, UPT = Split<R, L, NR>::UPT;
  static_assert(sizeof(R) == 8 || S == 1 || UPT % 2 == 0, "fp32 output split must keep 16-byte alignment");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<R>* sB = reinterpret_cast<C<R>*>(smem_raw);  // [2][L][LP]
  const int c = blockIdx.y / S, part = blockIdx.y % S;
  const int u0 = part * UPT;
  const int64_t i = (int64_t)blockIdx.x * LAT_THREADS + threadIdx.x;
  const bool live = i < N;
  const int ix = live ? (int)(i % nx) : 0, iy = live ? (int)(i / nx) : 0;
  C<R> acc[NR][UPT];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int u = 0; u < UPT; ++u) acc[r][u] = mk<R>(0, 0);
  const int blk = L * LP;
  auto stage = [&](int kk, int buf) {
    C<R>* dst = sB + buf * blk;
    if (MODE == 1) {
      // adjoint: S[u'][u] = A_{-o}[u'][u] = BT[neg][c][u][u']
      const C<R>* src = BT + ((size_t)neg[kk] * 2 + c) * blk;
      for (int e = threadIdx.x; e < L * L; e += LAT_THREADS) {
        int up = e / L, u = e % L;
        dst[up * LP + u] = src[u * LP + up];
      }
    } else {
      const C<R>* src = BT + ((size_t)kk * 2 + c) * blk;
      for (int e = threadIdx.x; e < blk; e += LAT_THREADS) dst[e] = src[e];
    }
  };
  if (K > 0) stage(0, 0);
  __syncthreads();
  for (int kk = 0; kk < K; ++kk) {
    const int buf = kk & 1;
    if (kk + 1 < K) stage(kk + 1, buf ^ 1);
    const int2 o = off[kk];
    const int sx = ix + o.x, sy = iy + o.y;
    if (live && sx >= 0 && sx < nx && sy >= 0 && sy < ny) {
      const int64_t j = (int64_t)sy * nx + sx;
      const C<R>* sb = sB + buf * blk;
      const C<R>* xj = x + j * P + c * L;
#pragma unroll 2
      for (int up = 0; up < L; ++up) {
        C<R> xv[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          xv[r] = xj[r * rstride + up];
          if (MODE == 1) xv[r] = cmul(xv[r], T[j * P + c * L + up]);
        }
        const C<R>* brow = sb + up * LP + u0;
        if constexpr (sizeof(R) == 4) {
          // two complex block entries per 16-byte shared load (LP and u0 are even)
#pragma unroll
          for (int u = 0; u < UPT; u += 2) {
            const float4 bb = *reinterpret_cast<const float4*>(brow + u);
            const C<R> b0 = mk<R>(bb.x, bb.y), b1 = mk<R>(bb.z, bb.w);
            if (u0 + u < L) {
#pragma unroll
              for (int r = 0; r < NR; ++r) cfma(acc[r][u], b0, xv[r]);
            }
            if (u + 1 < UPT && u0 + u + 1 < L) {
#pragma unroll
              for (int r = 0; r < NR; ++r) cfma(acc[r][u + 1], b1, xv[r]);
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < UPT; ++u) {
            if (u0 + u < L) {
              const C<R> b = brow[u];
#pragma unroll
              for (int r = 0; r < NR; ++r) cfma(acc[r][u], b, xv[r]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (!live) return;
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int uu = u0 + u;
    if (uu < L) {
      const int64_t o = i * P + c * L + uu;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        C<R> out;
        if (MODE == 2) out = acc[r][u];
        else if (MODE == 0) out = csub(x[r * rstride + o], cmul(T[o], acc[r][u]));
        else out = csub(x[r * rstride + o], acc[r][u]);
        y[r * rstride + o] = out;
      }
    }
  }
}

template <typename R, int NMAX, int NR, int MODE>
static int launch_lat(tmat_ctx* ctx, const LatOp& a, const void* x, void* y, int64_t rstride) {
  constexpr int L = NMAX * (NMAX + 2);
  constexpr int S = Split<R, L, NR>::S;
  dim3 grid((unsigned)cdiv(a.N, LAT_THREADS), 2 * S);
  size_t smem = sizeof(C<R>) * 2 * L * a.LP;
  auto kern = lattice_apply_kernel<R, NMAX, NR, MODE>;
  if (smem > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
  cudaEvent_t ev = timing_begin(ctx);
  kern<<<grid, LAT_THREADS, smem, ctx->stream>>>(a.off, a.neg, a.K, a.nx, a.ny, a.N, (const C<R>*)a.BT, a.LP,
                                                  (const C<R>*)a.T, (const C<R>*)x, (C<R>*)y, rstride);
  TM_LAUNCHED(ctx);
  timing_end(ctx, sizeof(R) == 4 ? "lattice_apply_fp32" : "lattice_apply_fp64", ev);
  return TMAT_OK;
}

template <typename R, int NR, int MODE>
static int lat_nmax(tmat_ctx* ctx, const LatOp& a, const void* x, void* y, int64_t rs) {
  switch (a.nmax) {
    case 1: return launch_lat<R, 1, NR, MODE>(ctx, a, x, y, rs);
    case 2: return launch_lat<R, 2, NR, MODE>(ctx, a, x, y, rs);
    case 3: return launch_lat<R, 3, NR, MODE>(ctx, a, x, y, rs);
    case 4: return launch_lat<R, 4, NR, MODE>(ctx, a, x, y, rs);
    case 5: return launch_lat<R, 5, NR, MODE>(ctx, a, x, y, rs);
    case 6: return launch_lat<R, 6, NR, MODE>(ctx, a, x, y, rs);
  }
  return set_error(ctx, TMAT_EINVAL, "nmax %d unsupported", a.nmax);
}

template <typename R, int NR>
static int lat_mode(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int64_t rs) {
  if (mode == TMAT_OP_FORWARD) return lat_nmax<R, NR, 0>(ctx, a, x, y, rs);
  if (mode == TMAT_OP_ADJOINT) return lat_nmax<R, NR, 1>(ctx, a, x, y, rs);
  return lat_nmax<R, NR, 2>(ctx, a, x, y, rs);
}

int lattice_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  if (a.N == 0) return TMAT_OK;
  if (a.use_fft) return lattice_fft_apply(ctx, a, mode, x, y, R_);
  if (!a.fp32 && a.use_oz) return lattice_oz_apply(ctx, a, mode, x, y, R_);
  if (a.fp32 && a.use_tc && ctx->tensor_cores) {
    if (a.tc2 && ctx->tc_variant != 1) return lattice_tc2_apply(ctx, a, mode, x, y, R_);
    return lattice_tc_apply(ctx, a, mode, x, y, R_);
  }
  const int64_t rs = a.N * a.P;
  const size_t esz = a.fp32 ? sizeof(float2) : sizeof(double2);
  for (int r0 = 0; r0 < R_; r0 += 2) {
    const int nr = (R_ - r0) >= 2 ? 2 : 1;
    const char* xp = (const char*)x + esz * rs * r0;
    char* yp = (char*)y + esz * rs * r0;
    int rc;
    if (a.fp32) rc = nr == 2 ? lat_mode<float, 2>(ctx, a, mode, xp, yp, rs) : lat_mode<float, 1>(ctx, a, mode, xp, yp, rs);
    else rc = nr == 2 ? lat_mode<double, 2>(ctx, a, mode, xp, yp, rs) : lat_mode<double, 1>(ctx, a, mode, xp, yp, rs);
    if (rc) return rc;
  }
  return TMAT_OK;
}

// positions must be the row-major lattice x0 + ix*pitch, y0 + iy*pitch, z0
__global__ void lattice_check_kernel(const double* __restrict__ pos, int64_t N, int nx, double pitch, int* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ex = pos[0] + (double)(i % nx) * pitch, ey = pos[1] + (double)(i / nx) * pitch;
  double tol = 1e-9 * pitch;
  if (!(fabs(pos[3 * i] - ex) <= tol && fabs(pos[3 * i + 1] - ey) <= tol && pos[3 * i + 2] == pos[2])) atomicOr(bad, 1);
}

int make_lattice_ops(tmat_ctx* ctx, const Tables* t, const double* d_pos, int64_t N, double k, int nx, int ny,
                     double pitch, double cutoff, double taper, const double2* T64, const float2* T32, bool mixed,
                     OpPair* ops, int want_oz) {
  if (nx <= 0 || ny <= 0 || (int64_t)nx * ny != N || !(pitch > 0))
    return set_error(ctx, TMAT_EINVAL, "lattice path: need lattice_nx * lattice_ny == N and pitch > 0");
  {
    int* flag;
    TM_TRY(scratch(ctx, "lat_flag", sizeof(int), (void**)&flag));
    TM_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    lattice_check_kernel<<<(unsigned)cdiv(N, 256), 256, 0, ctx->stream>>>(d_pos, N, nx, pitch, flag);
    TM_LAUNCHED(ctx);
    int* pin = (int*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pin[0]) return set_error(ctx, TMAT_EINVAL, "lattice path: positions are not the row-major %d x %d lattice", nx, ny);
  }
  // offsets within the cutoff: d2 = (dx a)(dx a) + (dy a)(dy a) <= c c, as the neighbour test
  std::vector<int2> offs;
  const double c2 = cutoff * cutoff;
  for (int dy = -(ny - 1); dy <= ny - 1; ++dy)
    for (int dx = -(nx - 1); dx <= nx - 1; ++dx) {
      // (0, 0) stays in the list with an all-zero block (no self coupling): it keeps dx
      // contiguous inside the dy = 0 group, which the tensor-core kernel relies on
      double ax = dx * pitch, ay = dy * pitch;
      volatile double d2 = ax * ax;
      volatile double d2b = ay * ay;
      double d2s = d2 + d2b;
      if (cutoff > 0 && !(d2s <= c2) && !(dx == 0 && dy == 0)) continue;
      offs.push_back(make_int2(dx, dy));
    }
  const int K = (int)offs.size();
  // dy groups (offsets are generated dy-major with dx ascending) and the widest dx
  std::vector<int> dy_start;
  int CX = 0;
  int CY = 0;
  for (int a = 0; a < K; ++a) {
    if (a == 0 || offs[a].y != offs[a - 1].y) dy_start.push_back(a);
    CX = std::max(CX, std::abs(offs[a].x));
    CY = std::max(CY, std::abs(offs[a].y));
  }
  const int ndy = (int)dy_start.size();
  dy_start.push_back(K);
  // the tensor-core kernel steps dx by one inside a dy group
  bool dx_contiguous = true;
  for (int d = 0; d < ndy; ++d)
    for (int a = dy_start[d]; a < dy_start[d + 1]; ++a)
      if (offs[a].x != offs[dy_start[d]].x + (a - dy_start[d])) dx_contiguous = false;
  // index of -o for every offset o (the set is symmetric): a (2nx-1) x (2ny-1) lookup grid
  std::vector<int> negs(K), slot((size_t)(2 * nx - 1) * (2 * ny - 1), -1);
  for (int a = 0; a < K; ++a) slot[(size_t)(offs[a].y + ny - 1) * (2 * nx - 1) + (offs[a].x + nx - 1)] = a;
  for (int a = 0; a < K; ++a) negs[a] = slot[(size_t)(ny - 1 - offs[a].y) * (2 * nx - 1) + (nx - 1 - offs[a].x)];
  const int L = t->L, LP = (L % 2) ? L + 1 : L;
  int2* d_off;
  int* d_neg;
  double2* B64;
  float2* B32 = nullptr;
  TM_TRY(scratch(ctx, "lat_off", sizeof(int2) * std::max(K, 1), (void**)&d_off));
  TM_TRY(scratch(ctx, "lat_neg", sizeof(int) * std::max(K, 1), (void**)&d_neg));
  int* d_dys;
  TM_TRY(scratch(ctx, "lat_dys", sizeof(int) * (ndy + 1), (void**)&d_dys));
  TM_CUDA(ctx, cudaMemcpyAsync(d_dys, dy_start.data(), sizeof(int) * (ndy + 1), cudaMemcpyHostToDevice, ctx->stream));
  TM_TRY(scratch(ctx, "lat_B64", sizeof(double2) * (size_t)std::max(K, 1) * 2 * L * LP, (void**)&B64));
  if (mixed) TM_TRY(scratch(ctx, "lat_B32", sizeof(float2) * (size_t)std::max(K, 1) * 2 * L * LP, (void**)&B32));
  if (K > 0) {
    TM_CUDA(ctx, cudaMemcpyAsync(d_off, offs.data(), sizeof(int2) * K, cudaMemcpyHostToDevice, ctx->stream));
    TM_CUDA(ctx, cudaMemcpyAsync(d_neg, negs.data(), sizeof(int) * K, cudaMemcpyHostToDevice, ctx->stream));
    TM_CUDA(ctx, cudaMemsetAsync(B64, 0, sizeof(double2) * (size_t)K * 2 * L * LP, ctx->stream));
    if (B32) TM_CUDA(ctx, cudaMemsetAsync(B32, 0, sizeof(float2) * (size_t)K * 2 * L * LP, ctx->stream));
    switch (t->nmax) {
#define LB(NM) \
  case NM: lattice_blocks_kernel<NM><<<K, 256, 0, ctx->stream>>>(d_off, K, pitch, k, cutoff, taper, t->d_gdense, t->d_mval, LP, B64, B32); break;
      LB(1) LB(2) LB(3) LB(4) LB(5) LB(6)
#undef LB
    }
    TM_LAUNCHED(ctx);
  }
  const bool fft = ctx->lattice_fft && K > 0 && lattice_fft_fits(nx, ny, CX, CY);
  // mirror table of the class members for the FFT block product (lattice_fft.cu)
  std::vector<int> mir(2 * L, 0), sym(2 * L, 0);
  int* d_mir = nullptr;
  int* d_sym = nullptr;
  if (fft) {
    for (int c = 0; c < 2; ++c)
      for (int u = 0; u < L; ++u) {
        const int f = t->perm[c * L + u], p = f / L, n = f % L;
        int l = 1;
        while ((l + 1) * (l + 1) <= n + 1) ++l;
        const int m = n + 1 - l * (l + 1);
        const int f2 = p * L + l * (l + 1) - m - 1;
        int u2 = -1;
        for (int v = 0; v < L; ++v)
          if (t->perm[c * L + v] == f2) u2 = v;
        if (u2 < 0) return set_error(ctx, TMAT_ENOTSUP, "mirror partner missing in class %d", c);
        mir[c * L + u] = u2 | (p << 16);
        sym[c * L + u] = u2 | ((m & 1) << 16) | (p << 17);
      }
    char nm[32];
    snprintf(nm, sizeof nm, "fft_mirror%d", t->nmax);
    TM_TRY(scratch(ctx, nm, sizeof(int) * 2 * L, (void**)&d_mir));
    TM_CUDA(ctx, cudaMemcpyAsync(d_mir, mir.data(), sizeof(int) * 2 * L, cudaMemcpyHostToDevice, ctx->stream));
    snprintf(nm, sizeof nm, "fft_sym%d", t->nmax);
    TM_TRY(scratch(ctx, nm, sizeof(int) * 2 * L, (void**)&d_sym));
    TM_CUDA(ctx, cudaMemcpyAsync(d_sym, sym.data(), sizeof(int) * 2 * L, cudaMemcpyHostToDevice, ctx->stream));
  }
  // host copies above are from stack vectors: wait before they go out of scope
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  LatOp a;
  a.N = N;
  a.nx = nx;
  a.ny = ny;
  a.nmax = t->nmax;
  a.L = L;
  a.P = t->P;
  a.LP = LP;
  a.K = K;
  a.off = d_off;
  a.neg = d_neg;
  a.dy_start = d_dys;
  a.ndy = ndy;
  a.CX = CX;
  a.CY = CY;
  a.fp32 = false;
  a.BT = B64;
  a.T = T64;
  a.fft_mirror = d_mir;
  a.fft_sym = d_sym;
  if (fft) TM_TRY(lattice_fft_prepare(ctx, &a));
  ops->lat64 = a;
  a.use_fft = false;
  a.fft_Bhat = nullptr;
  ops->A64.kind = 1;
  ops->A64.lat = &ops->lat64;
  // the fp64-class tensor-core operator: for TMAT_PREC_FP64_TC, or for the refinement
  // residual when the fp64 operator is not already the (fp64) FFT one
  if ((want_oz == 2 || (want_oz == 1 && !fft)) && ctx->tensor_cores && t->nmax <= 4 && K > 0 && dx_contiguous &&
      lattice_oz_fits(t->nmax, CX)) {
    LatOp z = a;
    TM_TRY(lattice_oz_prepare(ctx, &z, B64));
    z.use_oz = true;
    ops->lat64oz = z;
    ops->R64.kind = 1;
    ops->R64.lat = &ops->lat64oz;
    ops->have_oz = true;
  }
  if (mixed) {
    a.fp32 = true;
    a.BT = B32;
    a.T = T32;
    if (fft) {
      TM_TRY(lattice_fft_prepare(ctx, &a));
    } else if (lattice_tc_supported(t->nmax) && K > 0 && dx_contiguous && lattice_tc_fits(t->nmax, CX)) {
      TM_TRY(lattice_tc_prepare(ctx, &a, B64));
      a.use_tc = true;
      a.tc2 = lattice_tc2_fits(t->nmax, CX);
    }
    ops->lat32 = a;
    ops->A32.kind = 1;
    ops->A32.lat = &ops->lat32;
    ops->have32 = true;
  }
  return TMAT_OK;
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_apply_lattice(tmat_ctx* ctx, int op, int precision, int nx, int ny, double pitch, double cutoff,
                                  double taper, double k, int nmax, const tmat_c128* T_diag, const tmat_c128* x, int R,
                                  tmat_c128* y) {
  if (!ctx) return TMAT_EINVAL;
  const int64_t N = (int64_t)nx * ny;
  if (nx < 0 || ny < 0 || R < 1 || !(k > 0) || !(pitch > 0) || !(taper >= 0) || (taper > 0 && !(taper <= cutoff)) || (N > 0 && (!x || !y)) || op < 0 || op > 2 ||
      (op != TMAT_OP_COUPLE && N > 0 && !T_diag) ||
      (precision != TMAT_PREC_FP64 && precision != TMAT_PREC_MIXED && precision != TMAT_PREC_FP64_TC))
    return set_error(ctx, TMAT_EINVAL, "tmat_apply_lattice: bad arguments");
  Tables* t;
  TM_TRY(get_tables(ctx, nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  if (N == 0) return TMAT_OK;
  const int P = t->P;
  const bool fp32 = precision == TMAT_PREC_MIXED;
  Staged sT, sx, sy;
  TM_TRY(stage_in(ctx, "st_T", T_diag, sizeof(double2) * N * P, &sT));
  TM_TRY(stage_in(ctx, "st_x", x, sizeof(double2) * R * N * P, &sx));
  TM_TRY(stage_out(ctx, "st_y", y, sizeof(double2) * R * N * P, &sy));
  // implied positions (origin 0) for the lattice check
  std::vector<double> hpos(3 * N);
  for (int64_t i = 0; i < N; ++i) {
    hpos[3 * i] = (double)(i % nx) * pitch;
    hpos[3 * i + 1] = (double)(i / nx) * pitch;
    hpos[3 * i + 2] = 0.0;
  }
  double* dpos;
  TM_TRY(scratch(ctx, "al_pos", sizeof(double) * 3 * N, (void**)&dpos));
  TM_CUDA(ctx, cudaMemcpyAsync(dpos, hpos.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, ctx->stream));
  void *T64 = nullptr, *T32 = nullptr;
  if (T_diag) {
    TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, false, "al_T64", &T64));
    if (fp32) TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, true, "al_T32", &T32));
  }
  OpPair ops;
  const bool emu = precision == TMAT_PREC_FP64_TC;
  TM_TRY(make_lattice_ops(ctx, t, dpos, N, k, nx, ny, pitch, cutoff, taper, (const double2*)T64, (const float2*)T32, fp32,
                          &ops, emu ? 2 : 0));
  if (emu && !ops.have_oz)
    return set_error(ctx, TMAT_ENOTSUP, "TMAT_PREC_FP64_TC needs tensor cores enabled, nmax <= 4 and a cutoff window that fits");
  const size_t esz = fp32 ? sizeof(float2) : sizeof(double2);
  void *xi, *yi;
  TM_TRY(scratch(ctx, "ap_x", esz * R * N * P, &xi));
  TM_TRY(scratch(ctx, "ap_y", esz * R * N * P, &yi));
  TM_TRY(to_internal(ctx, t, (const double2*)sx.dev, xi, fp32, (int64_t)R * N));
  TM_TRY(op_apply(ctx, fp32 ? ops.A32 : (emu ? ops.R64 : ops.A64), op, xi, yi, R));
  if (emu) {
    int* pin = (int*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, ops.lat64oz.oz_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pin[0]) return set_error(ctx, TMAT_ECUDA, "tensor-core fp64 apply: %d tiles gave up on a bounded wait", pin[0]);
  }
  TM_TRY(from_internal(ctx, t, yi, fp32, (double2*)sy.dev, (int64_t)R * N));
  TM_TRY(finish_out(ctx, &sy));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
