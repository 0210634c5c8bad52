// Neighbour-list apply of the preconditioned Maxwell operator (App. I-C/I-D), with the
// translation of every pair generated on the fly and discarded (App. I-D).
//
// Coplanar scatterers: inside the parity classes c = (l+m+p) mod 2 the block of pair
// (i, j), d = x_i - x_j = rho (cos phi, sin phi), is a combination of fixed sparse
// matrices with pair-dependent scalar weights:
//   A_ij = sum_{q, mu} H_ij[q, mu] G^(q, mu),   H_ij[q, mu] = w(rho) h_q(k rho) e^{i mu phi},
// mu in {-q, -q+2, .., q} (Pbar_q^{|mu|}(0) vanishes otherwise; it sits in G with the
// coupling constants a5/b5), w the coupling window. Hence
//   (A x)_i = sum_{q, mu} G^(q, mu) Z_i[q, mu],   Z_i[q, mu] = sum_j H_ij[q, mu] x_j,
// and a target's sum over its neighbours is one dense complex product
//   Z_i (NQM x P) = H_i (NQM x n_i) X_i (n_i x P),   NQM = (nmax+1)(2nmax+1) combinations,
// computed in register tiles on CUDA cores; the sparse G contraction (the same tables for
// every target) runs once per target instead of once per pair. The adjoint uses the
// transposed tables (mu = m - m', signs of the inverted offset) on T_j x_j.
//
// Mapping: one thread block per (target, group of NR right-hand sides). The neighbour row
// is taken in chunks of KC pairs, double-buffered: while the tile warps accumulate their
// A x B tiles of Z from chunk c (each thread forming its own rows of H from the weights),
// every thread issues the asynchronous copies of chunk c+1's x_j rows (T_j x_j for the
// adjoint, formed beforehand) and a producer warp forms its weights (w h_q and
// e^{i mu phi}, distance and phase reduction in fp64). Compute types: fp32 (complex64 vectors) and
// double-float (complex128 vectors, fp64 distances, Hankel functions and phases, the
// products and sums in fp32 pairs: the fp64 pipe runs at 1/64 of the fp32 one).
#include <algorithm>
#include <type_traits>

#include "apply.h"
#include "dev.cuh"
#include "dfloat.cuh"
#include "internal.h"

namespace tmat {

// Tiles of the pair-sum product for NR right-hand sides per block: A x TR rows cover the
// NQM combinations, B x TC columns the NR * P coefficients (B * TC == NR * P).
template <int NMAX, bool DBL, int NR> struct PsCfg;
#define PS_CFG(NM, D, NR_, A_, TR_, B_, TC_)                    \
  template <> struct PsCfg<NM, D, NR_> {                        \
    static constexpr int A = A_, TR = TR_, B = B_, TC = TC_;    \
  };
// complex64, one right-hand side
PS_CFG(1, false, 1, 1, 6, 1, 6)
PS_CFG(2, false, 1, 3, 5, 2, 8)
PS_CFG(3, false, 1, 2, 14, 5, 6)
PS_CFG(4, false, 1, 3, 15, 6, 8)
PS_CFG(5, false, 1, 6, 11, 7, 10)
PS_CFG(6, false, 1, 7, 13, 6, 16)
// complex64, two right-hand sides (the weights H shared)
PS_CFG(1, false, 2, 1, 6, 2, 6)
PS_CFG(2, false, 2, 3, 5, 4, 8)
PS_CFG(3, false, 2, 2, 14, 10, 6)
PS_CFG(4, false, 2, 3, 15, 12, 8)
PS_CFG(5, false, 2, 3, 22, 14, 10)
PS_CFG(6, false, 2, 7, 13, 6, 32)
// double-float, one right-hand side (16-byte elements)
PS_CFG(1, true, 1, 1, 6, 1, 6)
PS_CFG(2, true, 1, 3, 5, 2, 8)
PS_CFG(3, true, 1, 2, 14, 5, 6)
PS_CFG(4, true, 1, 3, 15, 6, 8)
PS_CFG(5, true, 1, 3, 22, 7, 10)
PS_CFG(6, true, 1, 7, 13, 3, 32)
#undef PS_CFG

template <typename R, int NMAX, int NR> struct PsShape {
  using Cf = PsCfg<NMAX, sizeof(C<R>) == 16, NR>;
  static constexpr int L = NMAX * (NMAX + 2), P = 2 * L, Q = 2 * NMAX + 1;
  static constexpr int NP = NR * P;  // columns of Z
  static constexpr int NQM = (NMAX + 1) * (2 * NMAX + 1);
  static constexpr int NQP = Cf::A * Cf::TR;  // rows of the tiles
  static constexpr int TT = ((Cf::TR * Cf::TC + 31) / 32) * 32;  // tile threads
  static constexpr int THREADS = TT + 32;                         // + one producer warp
  // resident blocks per SM asked of the register allocator (the shared memory allows them)
  static constexpr int MINB = THREADS > 160 || NMAX > 4 ? 1 : sizeof(C<R>) == 16 ? 2 : NR == 2 ? 3 : 4;
  // pairs per chunk: 32, or 16 where two buffers of gathered rows would pass 64 KB
  static constexpr int KC = 2 * 32 * NP * sizeof(C<R>) <= 64 * 1024 ? 32 : 16;
  static_assert(Cf::B * Cf::TC == NP, "column tiles cover NR * P");
  static_assert(NQP >= NQM, "row tiles cover the combinations");
  static_assert(THREADS >= NP, "one thread per output");
  // shared memory (units of C<R>): W[2][2][KC][Q] (per buffer: w h_q, then e^{i mu phi}),
  // then Xs[2][KC][NP] which Z[NQM][NP] reuses after the last chunk
  static constexpr int WSZ = 2 * KC * Q;  // one buffer of weights
  static constexpr int PROD = 2 * KC * NP > NQM * NP ? 2 * KC * NP : NQM * NP;
  static constexpr size_t SMEM = sizeof(C<R>) * (2 * WSZ + PROD);
};

// real type of the per-pair geometry, Hankel functions and phases, and of the G factors
template <typename R> using PsReal = std::conditional_t<std::is_same_v<R, float>, float, double>;
template <typename R> __device__ __forceinline__ C<R> ps_conv(C<PsReal<R>> v) { return v; }
template <> __device__ __forceinline__ dfc ps_conv<DF>(double2 v) { return cfrom64<DF>(v.x, v.y); }
// conjugate where neg (the weights of mu < 0)
__device__ __forceinline__ float2 ps_cond_conj(float2 e, bool neg) { return neg ? cconj(e) : e; }
__device__ __forceinline__ dfc ps_cond_conj(dfc e, bool neg) { return neg ? cconj(e) : e; }

// Column of tile element b of column group tc. With B even the groups interleave in pairs
// (b/2) * 2 TC + 2 tc + b % 2, so that the 16-byte loads of the TC groups of a warp fall on
// consecutive addresses (no shared-memory bank conflicts); otherwise tc * B + b.
template <int B, int TC> __device__ __forceinline__ int ps_col(int tc, int b) {
  if constexpr (B % 2 == 0) return (b >> 1) * (2 * TC) + 2 * tc + (b & 1);
  else return tc * B + b;
}

__device__ __forceinline__ void ps_cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void ps_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void ps_cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The source rows of one chunk for the NR right-hand sides, in the compute format
// (16-byte asynchronous copies by every thread of the block), zero-filled past the row's end.
template <typename R, int NMAX, int NR>
__device__ __forceinline__ void ps_gather_async(int tid, int nthr, int64_t c0, int64_t je,
                                                const int32_t* __restrict__ col, const C<R>* __restrict__ xg,
                                                int64_t rhs_stride, int r0, C<R>* Xb) {
  using S = PsShape<R, NMAX, NR>;
  constexpr int P = S::P, NP = S::NP, KC = S::KC;
  constexpr int EPC = 16 / (int)sizeof(C<R>);  // elements per copy
  constexpr int CPR = NP / EPC;                // copies per pair
  static_assert(P % EPC == 0, "copies stay inside one right-hand side");
  for (int idx = tid; idx < KC * CPR; idx += nthr) {
    const int t = idx / CPR, c = (idx - t * CPR) * EPC;
    const int rl = c / P, cc = c - rl * P;
    const int64_t e = c0 + t;
    const bool ok = e < je;
    const int jj = ok ? col[e] : 0;
    ps_cp_async16(Xb + t * NP + c, xg + (int64_t)(r0 + rl) * rhs_stride + (int64_t)jj * P + cc, ok ? 16 : 0);
  }
  ps_cp_async_commit();
}

// The weights of one chunk of a target's neighbour row, by the producer warp (lane = its
// lane): per pair w h_q into W[t][q] and e^{i mu phi} into W[KC + t][mu] (fp64 distance
// and phase reduction); zero past the row's end.
template <typename R, int NMAX, int NR>
__device__ __forceinline__ void ps_weights(int lane, int64_t c0, int64_t je, double xi0, double yi0,
                                           const double* __restrict__ pos, double k, const int32_t* __restrict__ col,
                                           double cutoff, double taper, double inv_taper, C<R>* W) {
  using S = PsShape<R, NMAX, NR>;
  using RG = PsReal<R>;
  constexpr int Q = S::Q, KC = S::KC;
  if (lane >= KC) return;
  C<R>* hw = W + lane * Q;
  C<R>* ep = W + (KC + lane) * Q;
  const int64_t e = c0 + lane;
  if (e < je) {
    const int jj = col[e];
    const double dx = xi0 - pos[3 * jj], dy = yi0 - pos[3 * jj + 1];
    const double r2 = dx * dx + dy * dy;
    double rho;
    if constexpr (std::is_same_v<R, float>) {
      const double r0d = (double)rsqrtf((float)r2);  // one Newton step to fp64 accuracy
      rho = r2 * r0d;
      rho += 0.5 * r0d * (r2 - rho * rho);
    } else {
      rho = sqrt(r2);
    }
    C<RG> h[Q];
    hankel_up<RG, Q>(k * rho, h);
    RG wgt = (RG)1;
    if (taper > 0) {
      const double d0 = cutoff - taper;
      if (rho > d0) {
        if constexpr (std::is_same_v<RG, float>) wgt = 0.5f * (1.0f + cospif((float)(rho - d0) * (float)inv_taper));
        else wgt = 0.5 * (1.0 + cospi((rho - d0) * inv_taper));
      }
    }
    const RG ir = (RG)1 / (RG)rho;
    const C<RG> e1 = mk<RG>((RG)dx * ir, (RG)dy * ir);
    C<RG> z = mk<RG>((RG)1, (RG)0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      hw[q] = ps_conv<R>(cscale(h[q], wgt));
      ep[q] = ps_conv<R>(z);
      z = cmul(z, e1);
    }
  } else {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      hw[q] = czero<R>();
      ep[q] = czero<R>();
    }
  }
}

template <typename R, int NMAX, int OP, int NR>
__global__ void __launch_bounds__(PsShape<R, NMAX, NR>::THREADS, PsShape<R, NMAX, NR>::MINB)
pairsum_kernel(const double* __restrict__ pos, int64_t N, double k, const G<R>* __restrict__ T,
               const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const G<R>* __restrict__ x, const C<R>* __restrict__ xg, G<R>* __restrict__ y, int64_t rhs_stride,
               const int* __restrict__ zseg, const int* __restrict__ zidx, const PsReal<R>* __restrict__ zval,
               double cutoff, double taper, double inv_taper) {
  using S = PsShape<R, NMAX, NR>;
  using Cf = typename S::Cf;
  using RG = PsReal<R>;
  constexpr int P = S::P, Q = S::Q, NQM = S::NQM, NP = S::NP, KC = S::KC, WSZ = S::WSZ;
  constexpr int A = Cf::A, B = Cf::B, TC = Cf::TC, TR = Cf::TR;
  extern __shared__ __align__(16) unsigned char ps_smem[];
  C<R>* W = reinterpret_cast<C<R>*>(ps_smem);  // [2][2 KC][Q]
  C<R>* Xs = W + 2 * WSZ;                       // [2][KC][NP]
  C<R>* Z = Xs;                                 // [NQM][NP] after the last chunk

  const int64_t i = blockIdx.x;
  const int r0 = blockIdx.y * NR;
  const int tid = threadIdx.x;
  const bool producer = tid >= S::TT;
  const int lane = tid - S::TT;
  const int tr = tid / TC, tc = tid % TC;
  const bool tile = !producer && tr < TR;
  const double xi0 = pos[3 * i], yi0 = pos[3 * i + 1];
  const int64_t jb = row_ptr[i], je = row_ptr[i + 1];
  const int nch = (int)((je - jb + KC - 1) / KC);
  // this thread's rows of H: a = tr A + s -> (q, |mu|, mu < 0), a = q(q+1)/2 + (mu+q)/2
  int qa[A], ma[A];
  bool na[A];
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const int a = tile ? min(tr * A + s, NQM - 1) : 0;
    int q = 0;
    while ((q + 1) * (q + 2) / 2 <= a) ++q;
    const int mu = 2 * (a - q * (q + 1) / 2) - q;
    qa[s] = q;
    ma[s] = mu < 0 ? -mu : mu;
    na[s] = mu < 0;
  }
  if (nch > 0) {
    if (producer) ps_weights<R, NMAX, NR>(lane, jb, je, xi0, yi0, pos, k, col, cutoff, taper, inv_taper, W);
    ps_gather_async<R, NMAX, NR>(tid, S::THREADS, jb, je, col, xg, rhs_stride, r0, Xs);
  }
  ps_cp_async_wait_all();
  __syncthreads();

  C<R> acc[A][B];
#pragma unroll
  for (int a = 0; a < A; ++a)
#pragma unroll
    for (int b = 0; b < B; ++b) acc[a][b] = czero<R>();

  // chunk c (buffer c & 1) is multiplied while the rows of chunk c + 1 arrive (copies
  // issued by every thread) and the producer warp forms its weights
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    if (c + 1 < nch) {
      const int64_t c1 = jb + (int64_t)(c + 1) * KC;
      if (producer) ps_weights<R, NMAX, NR>(lane, c1, je, xi0, yi0, pos, k, col, cutoff, taper, inv_taper, W + (buf ^ 1) * WSZ);
      ps_gather_async<R, NMAX, NR>(tid, S::THREADS, c1, je, col, xg, rhs_stride, r0, Xs + (buf ^ 1) * KC * NP);
    }
    if (tile) {
      const C<R>* hw = W + buf * WSZ;
      const C<R>* ep = hw + KC * Q;
      const C<R>* Xb = Xs + buf * KC * NP;
#pragma unroll 2
      for (int t = 0; t < KC; ++t) {
        C<R> hv[A], xv[B];
#pragma unroll
        for (int s = 0; s < A; ++s) hv[s] = cmul(hw[t * Q + qa[s]], ps_cond_conj(ep[t * Q + ma[s]], na[s]));
#pragma unroll
        for (int b = 0; b < B; ++b) xv[b] = Xb[t * NP + ps_col<B, TC>(tc, b)];
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) cfma(acc[a][b], hv[a], xv[b]);
      }
    }
    ps_cp_async_wait_all();
    __syncthreads();
  }
  // Z to shared memory, then the sparse contraction per output
  if (tile) {
#pragma unroll
    for (int a = 0; a < A; ++a)
      if (tr * A + a < NQM) {
#pragma unroll
        for (int b = 0; b < B; ++b) Z[(tr * A + a) * NP + ps_col<B, TC>(tc, b)] = acc[a][b];
      }
  }
  __syncthreads();
  if (tid < NP) {
    const int rl = tid / P, o = tid - rl * P;
    const C<R>* Zr = Z + rl * P;
    C<R> s = czero<R>();
    for (int e = zseg[o]; e < zseg[o + 1]; ++e) {
      const int pk = __ldg(zidx + e);
      const RG v = __ldg(zval + e);
      const C<R> zv = Zr[((pk >> 8) & 0xff) * NP + (pk & 0xff)];
      const bool im = (pk >> 16) & 1;
      if constexpr (std::is_same_v<R, DF>) {
        float vh, vl;
        df_split(v, vh, vl);
        const dfc zr = im ? dfc{-zv.ih, -zv.il, zv.rh, zv.rl} : zv;  // i z where imag
        s = cadd(s, cscale_df(zr, vh, vl));
      } else {
        s.x = fma(v, im ? -zv.y : zv.x, s.x);
        s.y = fma(v, im ? zv.x : zv.y, s.y);
      }
    }
    const int64_t oi = i * P + o;
    const G<R>* xr = x + (int64_t)(r0 + rl) * rhs_stride;
    const G<R> sg = gstore<R>(s);
    G<R> out;
    if (OP == 2) out = sg;
    else if (OP == 0) out = csub(xr[oi], cmul(T[oi], sg));
    else out = csub(xr[oi], sg);
    y[(int64_t)(r0 + rl) * rhs_stride + oi] = out;
  }
}

template <typename R, int NMAX, int OP, int NR>
static int launch_pairsum(tmat_ctx* ctx, const NbrOp& a, const void* x, const void* xg, void* y, int ngroups,
                          int64_t stride) {
  using S = PsShape<R, NMAX, NR>;
  auto kern = pairsum_kernel<R, NMAX, OP, NR>;
  if (S::SMEM > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, S::SMEM));
  const int op = OP == 1 ? 1 : 0;
  const PsReal<R>* zv = std::is_same_v<R, float> ? (const PsReal<R>*)a.tab->d_zval_f32[op]
                                                 : (const PsReal<R>*)a.tab->d_zval_f64[op];
  kern<<<dim3((unsigned)a.N, (unsigned)ngroups), S::THREADS, S::SMEM, ctx->stream>>>(
      a.pos, a.N, a.k, (const G<R>*)a.T, a.row_ptr, a.col, (const G<R>*)x, (const C<R>*)xg, (G<R>*)y, stride,
      a.tab->d_zseg[op], a.tab->d_zidx[op], zv, a.cutoff, a.taper, a.taper > 0 ? 1.0 / a.taper : 0.0);
  return TMAT_OK;
}

// nrhs right-hand sides: complex64 in blocks of two (the pair weights shared), then one
template <typename R, int NMAX, int OP>
static int launch_rhs(tmat_ctx* ctx, const NbrOp& a, const void* x, const void* xg, void* y, int nrhs,
                      int64_t stride) {
  constexpr int NR = std::is_same_v<R, float> ? 2 : 1;
  const int ng = nrhs / NR;
  if (ng > 0) TM_TRY((launch_pairsum<R, NMAX, OP, NR>(ctx, a, x, xg, y, ng, stride)));
  if (NR == 2 && (nrhs & 1)) {
    const size_t off = sizeof(G<R>) * (size_t)stride * (nrhs - 1);
    const size_t offg = sizeof(C<R>) * (size_t)stride * (nrhs - 1);
    TM_TRY((launch_pairsum<R, NMAX, OP, 1>(ctx, a, (const char*)x + off, (const char*)xg + offg, (char*)y + off, 1,
                                           stride)));
  }
  return TMAT_OK;
}

// The gathered sources in the compute format: xg[r] = x[r] (times T elementwise for the
// adjoint), n = N P coefficients per right-hand side
template <typename R, bool MULT>
__global__ void ps_sources_kernel(const G<R>* __restrict__ x, const G<R>* __restrict__ T, C<R>* __restrict__ xg,
                                  int64_t n, int nrhs, int64_t stride) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * nrhs;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / n, e = idx - r * n;
    G<R> v = x[r * stride + e];
    if (MULT) v = cmul(v, T[e]);
    xg[r * stride + e] = gload<R>(v);
  }
}

template <typename R, int OP>
static int dispatch_nmax(tmat_ctx* ctx, const NbrOp& a, const void* x, void* y, int nrhs, int64_t stride) {
  cudaEvent_t ev = timing_begin(ctx);
  const void* xg = x;
  if (OP == 1 || !std::is_same_v<R, float>) {  // T_j x_j for the adjoint; double-float pairs
    void* xt = nullptr;
    TM_TRY(scratch(ctx, "nbr_sources", sizeof(C<R>) * (size_t)stride * nrhs, &xt));
    const int64_t n = a.N * num_coeffs(a.nmax);
    const unsigned grid = (unsigned)std::min<int64_t>(cdiv(n * nrhs, 256), 8 * (int64_t)ctx->num_sms);
    if (OP == 1)
      ps_sources_kernel<R, true><<<grid, 256, 0, ctx->stream>>>((const G<R>*)x, (const G<R>*)a.T, (C<R>*)xt, n, nrhs,
                                                                stride);
    else
      ps_sources_kernel<R, false><<<grid, 256, 0, ctx->stream>>>((const G<R>*)x, (const G<R>*)a.T, (C<R>*)xt, n, nrhs,
                                                                 stride);
    TM_LAUNCHED(ctx);
    xg = xt;
  }
  int rc;
  switch (a.nmax) {
    case 1: rc = launch_rhs<R, 1, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    case 2: rc = launch_rhs<R, 2, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    case 3: rc = launch_rhs<R, 3, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    case 4: rc = launch_rhs<R, 4, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    case 5: rc = launch_rhs<R, 5, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    case 6: rc = launch_rhs<R, 6, OP>(ctx, a, x, xg, y, nrhs, stride); break;
    default: return set_error(ctx, TMAT_EINVAL, "nmax %d unsupported", a.nmax);
  }
  if (rc) return rc;
  TM_LAUNCHED(ctx);
  timing_end(ctx, std::is_same_v<R, float> ? "nbr_apply_fp32" : "nbr_apply_fp64", ev);
  return TMAT_OK;
}

constexpr int MAXR = 4;  // right-hand sides per launch

// ---- general 3-D positions ------------------------------------------------------
// Without a common plane the blocks do not split into parity classes. The block of pair
// (i, j) is formed in full from the 3-D coupling constants: xi(k d) with
//   alpha[n][n'] (= xi[n][n'] = xi[L+n][L+n']) = e^{i mu phi} sum_q a5[n][n'][q] h_q(k r) Pbar_q^{|mu|}(cos theta),
//   beta[n][n']  (= xi[n][L+n'] = xi[L+n][n'])  the same with b5, mu = m - m',
// and applied as (A x)_i = sum_j xi(k(x_i - x_j))^T x_j (forward) or
// (A^T z)_i = sum_j xi(k(x_j - x_i)) z_j (adjoint). One block of threads per target;
// block entries in fp64, vectors in the operator's precision.
constexpr int NBR3_THREADS = 128;
template <typename R, int NMAX, int OP>
__global__ void __launch_bounds__(NBR3_THREADS)
apply_nbr3d_kernel(const double* __restrict__ pos, int64_t N, double k, const C<R>* __restrict__ T,
                   const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                   const C<R>* __restrict__ x, C<R>* __restrict__ y, int nrhs, int64_t rhs_stride,
                   const double2* __restrict__ a5, const double2* __restrict__ b5, const int* __restrict__ perm,
                   double cutoff, double taper) {
  constexpr int L = NMAX * (NMAX + 2), P = 2 * L, Q = 2 * NMAX + 1;
  static_assert(P <= NBR3_THREADS, "one output per thread");
  __shared__ double2 al[L * L], be[L * L];
  __shared__ double2 h[Q];
  __shared__ double Pq[Q][Q];
  __shared__ double2 eph[2 * Q - 1];
  __shared__ double2 xs[MAXR][P];  // source coefficients in flat order
  const int64_t i = blockIdx.x;
  if (i >= N) return;
  const int tid = threadIdx.x;
  const int fo = tid < P ? perm[tid] : 0;  // flat index of this thread's output (internal index tid)
  const int po = fo / L, no = fo % L;
  double2 acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) acc[r] = make_double2(0, 0);
  const int64_t jb = row_ptr[i], je = row_ptr[i + 1];
  for (int64_t e = jb; e < je; ++e) {
    const int64_t j = col[e];
    const double sg = OP == 1 ? -1.0 : 1.0;  // adjoint: d = x_j - x_i
    const double dx = sg * (pos[3 * i] - pos[3 * j]), dy = sg * (pos[3 * i + 1] - pos[3 * j + 1]),
                 dz = sg * (pos[3 * i + 2] - pos[3 * j + 2]);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double ct = dz / r, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double rho = sqrt(dx * dx + dy * dy);
    const double cp = rho > 0 ? dx / rho : 1.0, sp = rho > 0 ? dy / rho : 0.0;
    const double w = taper_weight(r, cutoff, taper);
    if (tid == 0) {
      double2 hh[Q];
      hankel_up<double, Q>(k * r, hh);
      for (int q = 0; q < Q; ++q) h[q] = cscale(hh[q], w);
      double2 ee = make_double2(1, 0), e1 = make_double2(cp, sp);
      for (int mu = 0; mu < Q; ++mu) {
        eph[Q - 1 + mu] = ee;
        eph[Q - 1 - mu] = cconj(ee);
        ee = cmul(ee, e1);
      }
    }
    if (tid < Q) {  // Pbar_q^mu(cos theta), mu = tid, upward in q
      const int mu = tid;
      double df = 1.0, f2 = 1.0;
      for (int t = 1; t < 2 * mu; t += 2) df *= t;
      for (int t = 2; t <= 2 * mu; ++t) f2 *= t;
      double pprev = 0.0, pcur = sqrt((2 * mu + 1) / (2.0 * f2)) * df * pow(st, (double)mu);
      for (int q = 0; q < mu; ++q) Pq[q][mu] = 0.0;
      Pq[mu][mu] = pcur;
      for (int q = mu + 1; q < Q; ++q) {
        const double a = sqrt((4.0 * q * q - 1) / ((double)q * q - (double)mu * mu));
        const double b = sqrt(((q - 1.0) * (q - 1.0) - (double)mu * mu) / (4.0 * (q - 1.0) * (q - 1.0) - 1));
        const double pn = a * (ct * pcur - b * pprev);
        pprev = pcur;
        pcur = pn;
        Pq[q][mu] = pn;
      }
    }
    for (int t = tid; t < nrhs * P; t += NBR3_THREADS) {
      const int rr = t / P, u = t % P;
      C<R> v = x[rr * rhs_stride + j * P + u];
      if (OP == 1) v = cmul(v, T[j * P + u]);
      xs[rr][perm[u]] = make_double2((double)v.x, (double)v.y);
    }
    __syncthreads();
    for (int t = tid; t < L * L; t += NBR3_THREADS) {
      const int n = t / L, np = t % L;
      int l = 1, lp = 1;
      while ((l + 1) * (l + 1) - 1 <= n) ++l;
      while ((lp + 1) * (lp + 1) - 1 <= np) ++lp;
      const int m = n + 1 - l * (l + 1), mp = np + 1 - lp * (lp + 1);
      const int mu = m - mp, amu = abs(mu);
      double2 a_ = make_double2(0, 0), b_ = make_double2(0, 0);
      for (int q = abs(l - lp); q <= l + lp; ++q) {
        if (amu > q) continue;
        const double2 hp = cscale(h[q], Pq[q][amu]);
        cfma(a_, a5[((size_t)n * L + np) * Q + q], hp);
        cfma(b_, b5[((size_t)n * L + np) * Q + q], hp);
      }
      al[t] = cmul(a_, eph[Q - 1 + mu]);
      be[t] = cmul(b_, eph[Q - 1 + mu]);
    }
    __syncthreads();
    if (tid < P) {
      for (int np = 0; np < L; ++np) {
        // forward: xi^T, entry (f', f) of xi; adjoint: xi, entry (f, f')
        const double2 ga = OP == 1 ? al[no * L + np] : al[np * L + no];
        const double2 gb = OP == 1 ? be[no * L + np] : be[np * L + no];
        for (int rr = 0; rr < nrhs; ++rr) {
          cfma(acc[rr], ga, xs[rr][po * L + np]);
          cfma(acc[rr], gb, xs[rr][(1 - po) * L + np]);
        }
      }
    }
    __syncthreads();
  }
  if (tid < P) {
    const int64_t o = i * P + tid;
    for (int rr = 0; rr < nrhs; ++rr) {
      const C<R> a = mk<R>((R)acc[rr].x, (R)acc[rr].y);
      C<R> out;
      if (OP == 2) out = a;
      else if (OP == 0) out = csub(x[rr * rhs_stride + o], cmul(T[o], a));
      else out = csub(x[rr * rhs_stride + o], a);
      y[rr * rhs_stride + o] = out;
    }
  }
}

template <typename R, int OP>
static int dispatch3d(tmat_ctx* ctx, const NbrOp& a, const void* x, void* y, int nrhs, int64_t stride) {
  cudaEvent_t ev = timing_begin(ctx);
  const unsigned grid = (unsigned)a.N;
  const Tables* t = a.tab;
#define N3(NM)                                                                                                    \
  case NM:                                                                                                        \
    apply_nbr3d_kernel<R, NM, OP><<<grid, NBR3_THREADS, 0, ctx->stream>>>(                                      \
        a.pos, a.N, a.k, (const C<R>*)a.T, a.row_ptr, a.col, (const C<R>*)x, (C<R>*)y, nrhs, stride, t->d_a5, \
        t->d_b5, t->d_perm, a.cutoff, a.taper);                                                                  \
    break;
  switch (a.nmax) {
    N3(1) N3(2) N3(3) N3(4) N3(5)
    default: return set_error(ctx, TMAT_ENOTSUP, "non-coplanar positions: nmax %d above 5", a.nmax);
  }
#undef N3
  TM_LAUNCHED(ctx);
  timing_end(ctx, "nbr_apply3d", ev);
  return TMAT_OK;
}

// x, y: internal layout [R][N][P] in precision a.fp32 ? complex64 : complex128
int nbr_apply(tmat_ctx* ctx, const NbrOp& a, int op, const void* x, void* y, int R_) {
  if (a.N == 0) return TMAT_OK;
  const int64_t stride = a.N * num_coeffs(a.nmax);
  const size_t esz = a.fp32 ? sizeof(float2) : sizeof(double2);
  for (int r0 = 0; r0 < R_; r0 += MAXR) {
    int nr = R_ - r0 < MAXR ? R_ - r0 : MAXR;
    const char* xp = (const char*)x + esz * stride * r0;
    char* yp = (char*)y + esz * stride * r0;
    int rc;
    if (a.threed) {
      if (a.fp32) {
        if (op == TMAT_OP_FORWARD) rc = dispatch3d<float, 0>(ctx, a, xp, yp, nr, stride);
        else if (op == TMAT_OP_ADJOINT) rc = dispatch3d<float, 1>(ctx, a, xp, yp, nr, stride);
        else rc = dispatch3d<float, 2>(ctx, a, xp, yp, nr, stride);
      } else {
        if (op == TMAT_OP_FORWARD) rc = dispatch3d<double, 0>(ctx, a, xp, yp, nr, stride);
        else if (op == TMAT_OP_ADJOINT) rc = dispatch3d<double, 1>(ctx, a, xp, yp, nr, stride);
        else rc = dispatch3d<double, 2>(ctx, a, xp, yp, nr, stride);
      }
    } else if (a.fp32) {
      if (op == TMAT_OP_FORWARD) rc = dispatch_nmax<float, 0>(ctx, a, xp, yp, nr, stride);
      else if (op == TMAT_OP_ADJOINT) rc = dispatch_nmax<float, 1>(ctx, a, xp, yp, nr, stride);
      else rc = dispatch_nmax<float, 2>(ctx, a, xp, yp, nr, stride);
    } else {
      if (op == TMAT_OP_FORWARD) rc = dispatch_nmax<DF, 0>(ctx, a, xp, yp, nr, stride);
      else if (op == TMAT_OP_ADJOINT) rc = dispatch_nmax<DF, 1>(ctx, a, xp, yp, nr, stride);
      else rc = dispatch_nmax<DF, 2>(ctx, a, xp, yp, nr, stride);
    }
    if (rc) return rc;
  }
  return TMAT_OK;
}

// ---- layout conversion ------------------------------------------------------

template <typename R>
__global__ void to_internal_kernel(const double2* __restrict__ api, C<R>* __restrict__ out, const int* __restrict__ perm,
                                   int P, int64_t rows) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * P) return;
  int64_t row = t / P;
  int u = (int)(t % P);
  double2 v = api[row * P + perm[u]];
  out[t] = mk<R>((R)v.x, (R)v.y);
}

template <typename R>
__global__ void from_internal_kernel(const C<R>* __restrict__ in, double2* __restrict__ api, const int* __restrict__ perm,
                                     int P, int64_t rows) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * P) return;
  int64_t row = t / P;
  int u = (int)(t % P);
  C<R> v = in[t];
  api[row * P + perm[u]] = make_double2((double)v.x, (double)v.y);
}

int to_internal(tmat_ctx* ctx, const Tables* t, const double2* api, void* internal, bool fp32, int64_t rows) {
  int64_t tot = rows * t->P;
  if (tot == 0) return TMAT_OK;
  unsigned g = (unsigned)cdiv(tot, 256);
  if (fp32) to_internal_kernel<float><<<g, 256, 0, ctx->stream>>>(api, (float2*)internal, t->d_perm, t->P, rows);
  else to_internal_kernel<double><<<g, 256, 0, ctx->stream>>>(api, (double2*)internal, t->d_perm, t->P, rows);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

int from_internal(tmat_ctx* ctx, const Tables* t, const void* internal, bool fp32, double2* api, int64_t rows) {
  int64_t tot = rows * t->P;
  if (tot == 0) return TMAT_OK;
  unsigned g = (unsigned)cdiv(tot, 256);
  if (fp32) from_internal_kernel<float><<<g, 256, 0, ctx->stream>>>((const float2*)internal, api, t->d_perm, t->P, rows);
  else from_internal_kernel<double><<<g, 256, 0, ctx->stream>>>((const double2*)internal, api, t->d_perm, t->P, rows);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

__global__ void position_flags_kernel(const double* __restrict__ pos, int64_t N, int* __restrict__ flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(flags, 2);
  else if (z != pos[2]) atomicOr(flags, 1);
}

int position_flags(tmat_ctx* ctx, const double* d_pos, int64_t N, int* flags) {
  *flags = 0;
  if (N == 0) return TMAT_OK;
  int* f;
  TM_TRY(scratch(ctx, "posflag", sizeof(int), (void**)&f));
  TM_CUDA(ctx, cudaMemsetAsync(f, 0, sizeof(int), ctx->stream));
  position_flags_kernel<<<(unsigned)cdiv(N, 256), 256, 0, ctx->stream>>>(d_pos, N, f);
  TM_LAUNCHED(ctx);
  int* pin = (int*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, f, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *flags = pin[0];
  return TMAT_OK;
}


// T diagonal (API layout, complex128) -> internal layout in the kernel precision
int prepare_T(tmat_ctx* ctx, const Tables* t, const double2* T_api, int64_t N, bool fp32, const char* name, void** out) {
  size_t esz = fp32 ? sizeof(float2) : sizeof(double2);
  TM_TRY(scratch(ctx, name, esz * N * t->P, out));
  return to_internal(ctx, t, T_api, *out, fp32, N);
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_apply(tmat_ctx* ctx, int op, int precision, const double* pos, int64_t N, double k, int nmax,
                          const tmat_c128* T_diag, const int64_t* row_ptr, const int32_t* col, double cutoff,
                          double taper, const tmat_c128* x, int R, tmat_c128* y) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || R < 1 || !(k > 0) || !(taper >= 0) || (taper > 0 && !(taper <= cutoff)) || (N > 0 && (!pos || !row_ptr || !col || !x || !y)) ||
      (op != TMAT_OP_COUPLE && N > 0 && !T_diag) || op < 0 || op > 2 ||
      (precision != TMAT_PREC_FP64 && precision != TMAT_PREC_MIXED))
    return set_error(ctx, TMAT_EINVAL, "tmat_apply: bad arguments");
  Tables* t;
  TM_TRY(get_tables(ctx, nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  if (N == 0) return TMAT_OK;
  const int P = t->P;
  Staged sp, sT, sr, sc, sx, sy;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  int pflags;
  TM_TRY(position_flags(ctx, (const double*)sp.dev, N, &pflags));
  if (pflags & 2) return set_error(ctx, TMAT_EINVAL, "tmat_apply: positions must be finite");
  TM_TRY(stage_in(ctx, "st_T", T_diag, sizeof(double2) * N * P, &sT));
  TM_TRY(stage_in(ctx, "st_rowptr", row_ptr, sizeof(int64_t) * (N + 1), &sr));
  int64_t nnz = 0;
  {
    int64_t* pin = (int64_t*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, (const int64_t*)sr.dev + N, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    nnz = pin[0];
  }
  TM_TRY(stage_in(ctx, "st_col", col, sizeof(int32_t) * nnz, &sc));
  TM_TRY(stage_in(ctx, "st_x", x, sizeof(double2) * R * N * P, &sx));
  TM_TRY(stage_out(ctx, "st_y", y, sizeof(double2) * R * N * P, &sy));
  const bool fp32 = precision == TMAT_PREC_MIXED;
  const size_t esz = fp32 ? sizeof(float2) : sizeof(double2);
  void *xi, *yi, *Ti = nullptr;
  TM_TRY(scratch(ctx, "ap_x", esz * R * N * P, &xi));
  TM_TRY(scratch(ctx, "ap_y", esz * R * N * P, &yi));
  if (op != TMAT_OP_COUPLE) TM_TRY(prepare_T(ctx, t, (const double2*)sT.dev, N, fp32, "ap_T", &Ti));
  TM_TRY(to_internal(ctx, t, (const double2*)sx.dev, xi, fp32, (int64_t)R * N));
  NbrOp a;
  a.pos = (const double*)sp.dev;
  a.N = N;
  a.k = k;
  a.nmax = nmax;
  a.fp32 = fp32;
  a.T = Ti;
  a.row_ptr = (const int64_t*)sr.dev;
  a.col = (const int32_t*)sc.dev;
  a.tab = t;
  a.cutoff = cutoff;
  a.taper = taper;
  a.threed = (pflags & 1) != 0;  // not coplanar: full 3-D blocks
  TM_TRY(nbr_apply(ctx, a, op, xi, yi, R));
  TM_TRY(from_internal(ctx, t, yi, fp32, (double2*)sy.dev, (int64_t)R * N));
  TM_TRY(finish_out(ctx, &sy));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
