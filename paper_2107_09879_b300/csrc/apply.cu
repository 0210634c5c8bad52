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
// NQM combinations, B x TC columns the NR * P coefficients (B * TC == NR * P); D3: off the
// plane (NQM = (2 nmax + 1)^2 combinations).
template <int NMAX, bool DBL, int NR, bool D3> struct PsCfg;
#define PS_CFG(NM, D, NR_, D3_, A_, TR_, B_, TC_)              \
  template <> struct PsCfg<NM, D, NR_, D3_> {                  \
    static constexpr int A = A_, TR = TR_, B = B_, TC = TC_;   \
  };
// complex64, one right-hand side
PS_CFG(1, false, 1, false, 1, 6, 1, 6)
PS_CFG(2, false, 1, false, 3, 5, 2, 8)
PS_CFG(3, false, 1, false, 2, 14, 5, 6)
PS_CFG(4, false, 1, false, 3, 15, 6, 8)
PS_CFG(5, false, 1, false, 6, 11, 7, 10)
PS_CFG(6, false, 1, false, 7, 13, 6, 16)
// complex64, two right-hand sides (the weights H shared)
PS_CFG(1, false, 2, false, 1, 6, 2, 6)
PS_CFG(2, false, 2, false, 3, 5, 4, 8)
PS_CFG(3, false, 2, false, 2, 14, 10, 6)
PS_CFG(4, false, 2, false, 3, 15, 12, 8)
PS_CFG(5, false, 2, false, 3, 22, 14, 10)
PS_CFG(6, false, 2, false, 7, 13, 6, 32)
// double-float, one right-hand side (16-byte elements)
PS_CFG(1, true, 1, false, 1, 6, 1, 6)
PS_CFG(2, true, 1, false, 3, 5, 2, 8)
PS_CFG(3, true, 1, false, 2, 14, 5, 6)
PS_CFG(4, true, 1, false, 3, 15, 6, 8)
PS_CFG(5, true, 1, false, 3, 22, 7, 10)
PS_CFG(6, true, 1, false, 7, 13, 3, 32)
// off the plane (nmax <= 5): complex64 one and two right-hand sides, double-float one
PS_CFG(1, false, 1, true, 3, 3, 1, 6)
PS_CFG(2, false, 1, true, 5, 5, 2, 8)
PS_CFG(3, false, 1, true, 7, 7, 5, 6)
PS_CFG(4, false, 1, true, 3, 27, 6, 8)
PS_CFG(5, false, 1, true, 4, 31, 7, 10)
PS_CFG(1, false, 2, true, 3, 3, 2, 6)
PS_CFG(2, false, 2, true, 5, 5, 4, 8)
PS_CFG(3, false, 2, true, 7, 7, 5, 12)
PS_CFG(4, false, 2, true, 3, 27, 12, 8)
PS_CFG(5, false, 2, true, 4, 31, 14, 10)
PS_CFG(1, true, 1, true, 3, 3, 1, 6)
PS_CFG(2, true, 1, true, 5, 5, 2, 8)
PS_CFG(3, true, 1, true, 7, 7, 5, 6)
PS_CFG(4, true, 1, true, 3, 27, 6, 8)
PS_CFG(5, true, 1, true, 4, 31, 7, 10)
#undef PS_CFG

template <typename R, int NMAX, int NR, bool D3> struct PsShape {
  using Cf = PsCfg<NMAX, sizeof(C<R>) == 16, NR, D3>;
  static constexpr int L = NMAX * (NMAX + 2), P = 2 * L, Q = 2 * NMAX + 1;
  static constexpr int NP = NR * P;  // columns of Z
  static constexpr int NQM = D3 ? Q * Q : (NMAX + 1) * (2 * NMAX + 1);
  // per pair: HWN radial weights (w h_q; off the plane w h_q Pbar_q^m(cos theta), m <= q)
  // and the Q phases e^{i m phi}
  static constexpr int HWN = D3 ? Q * (Q + 1) / 2 : Q;
  static constexpr int NQP = Cf::A * Cf::TR;  // rows of the tiles
  static constexpr int TT = ((Cf::TR * Cf::TC + 31) / 32) * 32;  // tile threads
  static constexpr int THREADS = TT + 32;                         // + one producer warp
  // resident blocks per SM asked of the register allocator (the shared memory allows them)
  static constexpr int MINB_F = 65536 / (THREADS * 128), MINB_D = 65536 / (THREADS * 200);
  static constexpr int MINB = (NMAX > 4 && !D3) ? 1
                              : sizeof(C<R>) == 16 ? (MINB_D < 1 ? 1 : MINB_D > 2 ? 2 : MINB_D)
                                                   : (MINB_F < 1 ? 1 : MINB_F > 4 ? 4 : MINB_F);
  // pairs per chunk: 32, or 16 where two buffers of gathered rows would pass 64 KB
  static constexpr int KC = 2 * 32 * NP * sizeof(C<R>) <= 64 * 1024 ? 32 : 16;
  static_assert(Cf::B * Cf::TC == NP, "column tiles cover NR * P");
  static_assert(NQP >= NQM, "row tiles cover the combinations");
  static_assert(THREADS >= NP, "one thread per output");
  // shared memory (units of C<R>): W[2][KC][HWN + Q] (per buffer: the radial weights, then
  // the phases), then Xs[2][KC][NP] which Z[NQM][NP] reuses after the last chunk
  static constexpr int WSZ = KC * (HWN + Q);  // one buffer of weights
  static constexpr int PROD = 2 * KC * NP > NQM * NP ? 2 * KC * NP : NQM * NP;
  // off the plane, after these: the Legendre recurrence factors (a, b)[q][m] and the
  // starting values' factors c[m] in the geometry's real type
  static constexpr size_t LEG = D3 ? sizeof(std::conditional_t<std::is_same_v<R, float>, float, double>) *
                                         (size_t)(2 * Q * Q + Q) : 0;
  static constexpr size_t SMEM = sizeof(C<R>) * (2 * WSZ + PROD) + LEG;
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
template <typename R, int NMAX, int NR, bool D3>
__device__ __forceinline__ void ps_gather_async(int tid, int nthr, int64_t c0, int64_t je,
                                                const int32_t* __restrict__ col, const C<R>* __restrict__ xg,
                                                int64_t rhs_stride, int r0, C<R>* Xb) {
  using S = PsShape<R, NMAX, NR, D3>;
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

// Recurrence factors of the normalised associated Legendre functions, Q orders:
// Pbar_q^m = a (x Pbar_{q-1}^m - b Pbar_{q-2}^m), a = sqrt((4q^2-1)/(q^2-m^2)),
// b = sqrt(((q-1)^2-m^2)/(4(q-1)^2-1)) at [2(q Q + m)], [2(q Q + m) + 1]; and
// Pbar_m^m = c[m] sin^m theta, c[m] = sqrt((2m+1)/(2 (2m)!)) (2m-1)!! at [2 Q Q + m].
template <typename RG, int Q>
__device__ __forceinline__ void ps_legendre_factors(int lane, RG* leg) {
  for (int e = lane; e < Q * Q; e += 32) {
    const int q = e / Q, m = e - q * Q;
    RG a = 0, b = 0;
    if (q > m) {
      a = sqrt((RG)(4 * q * q - 1) / (RG)(q * q - m * m));
      b = sqrt((RG)((q - 1) * (q - 1) - m * m) / (RG)(4 * (q - 1) * (q - 1) - 1));
    }
    leg[2 * e] = a;
    leg[2 * e + 1] = b;
  }
  for (int m = lane; m < Q; m += 32) {
    RG df = 1, f2 = 1;
    for (int t = 1; t < 2 * m; t += 2) df *= (RG)t;
    for (int t = 2; t <= 2 * m; ++t) f2 *= (RG)t;
    leg[2 * Q * Q + m] = sqrt((RG)(2 * m + 1) / ((RG)2 * f2)) * df;
  }
}

// The weights of one chunk of a target's neighbour row, by the producer warp (lane = its
// lane): per pair the radial weights into W[t][0..HWN) (on the plane w h_q; off the plane
// w h_q Pbar_q^m(cos theta) at q(q+1)/2 + m, m <= q) and e^{i m phi} into
// W[KC HWN + t Q + m] (fp64 distance and phase reduction); zero past the row's end.
template <typename R, int NMAX, int NR, bool D3>
__device__ __forceinline__ void ps_weights(int lane, int64_t c0, int64_t je, double xi0, double yi0, double zi0,
                                           const double* __restrict__ pos, double k, const int32_t* __restrict__ col,
                                           double cutoff, double taper, double inv_taper, C<R>* W,
                                           const PsReal<R>* leg) {
  using S = PsShape<R, NMAX, NR, D3>;
  using RG = PsReal<R>;
  constexpr int Q = S::Q, KC = S::KC, HWN = S::HWN;
  if (lane >= KC) return;
  C<R>* hw = W + lane * HWN;
  C<R>* ep = W + KC * HWN + lane * Q;
  const int64_t e = c0 + lane;
  if (e >= je) {
#pragma unroll
    for (int q = 0; q < HWN; ++q) hw[q] = czero<R>();
#pragma unroll
    for (int q = 0; q < Q; ++q) ep[q] = czero<R>();
    return;
  }
  const int jj = col[e];
  const double dx = xi0 - pos[3 * jj], dy = yi0 - pos[3 * jj + 1];
  const double dz = D3 ? zi0 - pos[3 * jj + 2] : 0.0;
  const double r2 = dx * dx + dy * dy + dz * dz;
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
  C<RG> e1;
  if constexpr (D3) {  // theta, phi of d; phi = 0 on the axis
    const RG ir = (RG)1 / (RG)rho, rxy = (RG)sqrt(dx * dx + dy * dy);
    const RG ct = (RG)dz * ir, st = rxy * ir;
    e1 = rxy > (RG)0 ? mk<RG>((RG)dx / rxy, (RG)dy / rxy) : mk<RG>((RG)1, (RG)0);
    // Pbar_q^m(cos theta) row by row in q (all m <= q), upward from Pbar_m^m = c[m] sin^m
    // theta with the factors of the block's table (ps_legendre_factors); every index static
    RG p1[Q], p2[Q];  // rows q - 1 and q - 2
#pragma unroll
    for (int m = 0; m < Q; ++m) p1[m] = p2[m] = (RG)0;
    RG sq = (RG)1;  // st^q
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      RG cur[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        if (m > q) continue;
        cur[m] = m == q ? leg[2 * Q * Q + q] * sq
                        : leg[2 * (q * Q + m)] * (ct * p1[m] - leg[2 * (q * Q + m) + 1] * p2[m]);
        hw[q * (q + 1) / 2 + m] = ps_conv<R>(cscale(h[q], wgt * cur[m]));
      }
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        p2[m] = p1[m];
        p1[m] = m <= q ? cur[m] : (RG)0;
      }
      sq *= st;
    }
  } else {
    const RG ir = (RG)1 / (RG)rho;
    e1 = mk<RG>((RG)dx * ir, (RG)dy * ir);
#pragma unroll
    for (int q = 0; q < Q; ++q) hw[q] = ps_conv<R>(cscale(h[q], wgt));
  }
  C<RG> z = mk<RG>((RG)1, (RG)0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    ep[q] = ps_conv<R>(z);
    z = cmul(z, e1);
  }
}

template <typename R, int NMAX, int OP, int NR, bool D3>
__global__ void __launch_bounds__(PsShape<R, NMAX, NR, D3>::THREADS, PsShape<R, NMAX, NR, D3>::MINB)
pairsum_kernel(const double* __restrict__ pos, int64_t N, double k, const G<R>* __restrict__ T,
               const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const G<R>* __restrict__ x, const C<R>* __restrict__ xg, G<R>* __restrict__ y, int64_t rhs_stride,
               const int* __restrict__ zseg, const int* __restrict__ zidx, const PsReal<R>* __restrict__ zval,
               double cutoff, double taper, double inv_taper) {
  using S = PsShape<R, NMAX, NR, D3>;
  using Cf = typename S::Cf;
  using RG = PsReal<R>;
  constexpr int P = S::P, Q = S::Q, NQM = S::NQM, NP = S::NP, KC = S::KC, WSZ = S::WSZ, HWN = S::HWN;
  constexpr int A = Cf::A, B = Cf::B, TC = Cf::TC, TR = Cf::TR;
  extern __shared__ __align__(16) unsigned char ps_smem[];
  C<R>* W = reinterpret_cast<C<R>*>(ps_smem);  // [2][KC][HWN + Q]
  C<R>* Xs = W + 2 * WSZ;                       // [2][KC][NP]
  C<R>* Z = Xs;                                 // [NQM][NP] after the last chunk
  PsReal<R>* leg = reinterpret_cast<PsReal<R>*>(Xs + S::PROD);  // off the plane: Legendre factors

  const int64_t i = blockIdx.x;
  const int r0 = blockIdx.y * NR;
  const int tid = threadIdx.x;
  const bool producer = tid >= S::TT;
  const int lane = tid - S::TT;
  const int tr = tid / TC, tc = tid % TC;
  const bool tile = !producer && tr < TR;
  const double xi0 = pos[3 * i], yi0 = pos[3 * i + 1], zi0 = pos[3 * i + 2];
  const int64_t jb = row_ptr[i], je = row_ptr[i + 1];
  const int nch = (int)((je - jb + KC - 1) / KC);
  // this thread's rows of H: a = tr A + s -> (q, |mu|, mu < 0) with a = q(q+1)/2 + (mu+q)/2
  // on the plane, a = q^2 + mu + q off it; qa: the radial weight's slot, ma = |mu|
  int qa[A], ma[A];
  bool na[A];
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const int a = tile ? min(tr * A + s, NQM - 1) : 0;
    int q = 0, mu;
    if constexpr (D3) {
      while ((q + 1) * (q + 1) <= a) ++q;
      mu = a - q * q - q;
    } else {
      while ((q + 1) * (q + 2) / 2 <= a) ++q;
      mu = 2 * (a - q * (q + 1) / 2) - q;
    }
    ma[s] = mu < 0 ? -mu : mu;
    qa[s] = D3 ? q * (q + 1) / 2 + ma[s] : q;
    na[s] = mu < 0;
  }
  if (D3 && producer) {
    ps_legendre_factors<PsReal<R>, Q>(lane, leg);
    __syncwarp();
  }
  if (nch > 0) {
    if (producer)
      ps_weights<R, NMAX, NR, D3>(lane, jb, je, xi0, yi0, zi0, pos, k, col, cutoff, taper, inv_taper, W, leg);
    ps_gather_async<R, NMAX, NR, D3>(tid, S::THREADS, jb, je, col, xg, rhs_stride, r0, Xs);
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
      if (producer)
        ps_weights<R, NMAX, NR, D3>(lane, c1, je, xi0, yi0, zi0, pos, k, col, cutoff, taper, inv_taper,
                                    W + (buf ^ 1) * WSZ, leg);
      ps_gather_async<R, NMAX, NR, D3>(tid, S::THREADS, c1, je, col, xg, rhs_stride, r0, Xs + (buf ^ 1) * KC * NP);
    }
    if (tile) {
      const C<R>* hw = W + buf * WSZ;
      const C<R>* ep = hw + KC * HWN;
      const C<R>* Xb = Xs + buf * KC * NP;
#pragma unroll 2
      for (int t = 0; t < KC; ++t) {
        C<R> hv[A], xv[B];
#pragma unroll
        for (int s = 0; s < A; ++s) hv[s] = cmul(hw[t * HWN + qa[s]], ps_cond_conj(ep[t * Q + ma[s]], na[s]));
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

template <typename R, int NMAX, int OP, int NR, bool D3>
static int launch_pairsum(tmat_ctx* ctx, const NbrOp& a, const void* x, const void* xg, void* y, int ngroups,
                          int64_t stride) {
  using S = PsShape<R, NMAX, NR, D3>;
  auto kern = pairsum_kernel<R, NMAX, OP, NR, D3>;
  if (S::SMEM > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, S::SMEM));
  const int op = OP == 1 ? 1 : 0;
  const Tables* t = a.tab;
  const int* zs = D3 ? t->d_z3seg[op] : t->d_zseg[op];
  const int* zi = D3 ? t->d_z3idx[op] : t->d_zidx[op];
  const void* zv = std::is_same_v<R, float> ? (D3 ? (const void*)t->d_z3val_f32[op] : (const void*)t->d_zval_f32[op])
                                            : (D3 ? (const void*)t->d_z3val_f64[op] : (const void*)t->d_zval_f64[op]);
  kern<<<dim3((unsigned)a.N, (unsigned)ngroups), S::THREADS, S::SMEM, ctx->stream>>>(
      a.pos, a.N, a.k, (const G<R>*)a.T, a.row_ptr, a.col, (const G<R>*)x, (const C<R>*)xg, (G<R>*)y, stride, zs, zi,
      (const PsReal<R>*)zv, a.cutoff, a.taper, a.taper > 0 ? 1.0 / a.taper : 0.0);
  return TMAT_OK;
}

// nrhs right-hand sides: complex64 in blocks of two (the pair weights shared), then one
template <typename R, int NMAX, int OP, bool D3>
static int launch_rhs(tmat_ctx* ctx, const NbrOp& a, const void* x, const void* xg, void* y, int nrhs,
                      int64_t stride) {
  constexpr int NR = std::is_same_v<R, float> ? 2 : 1;
  const int ng = nrhs / NR;
  if (ng > 0) TM_TRY((launch_pairsum<R, NMAX, OP, NR, D3>(ctx, a, x, xg, y, ng, stride)));
  if (NR == 2 && (nrhs & 1)) {
    const size_t off = sizeof(G<R>) * (size_t)stride * (nrhs - 1);
    const size_t offg = sizeof(C<R>) * (size_t)stride * (nrhs - 1);
    TM_TRY((launch_pairsum<R, NMAX, OP, 1, D3>(ctx, a, (const char*)x + off, (const char*)xg + offg, (char*)y + off,
                                               1, stride)));
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
  if (a.threed) {
    switch (a.nmax) {
      case 1: rc = launch_rhs<R, 1, OP, true>(ctx, a, x, xg, y, nrhs, stride); break;
      case 2: rc = launch_rhs<R, 2, OP, true>(ctx, a, x, xg, y, nrhs, stride); break;
      case 3: rc = launch_rhs<R, 3, OP, true>(ctx, a, x, xg, y, nrhs, stride); break;
      case 4: rc = launch_rhs<R, 4, OP, true>(ctx, a, x, xg, y, nrhs, stride); break;
      case 5: rc = launch_rhs<R, 5, OP, true>(ctx, a, x, xg, y, nrhs, stride); break;
      default: return set_error(ctx, TMAT_ENOTSUP, "non-coplanar positions: nmax %d above 5", a.nmax);
    }
  } else {
    switch (a.nmax) {
      case 1: rc = launch_rhs<R, 1, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      case 2: rc = launch_rhs<R, 2, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      case 3: rc = launch_rhs<R, 3, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      case 4: rc = launch_rhs<R, 4, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      case 5: rc = launch_rhs<R, 5, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      case 6: rc = launch_rhs<R, 6, OP, false>(ctx, a, x, xg, y, nrhs, stride); break;
      default: return set_error(ctx, TMAT_EINVAL, "nmax %d unsupported", a.nmax);
    }
  }
  if (rc) return rc;
  TM_LAUNCHED(ctx);
  constexpr bool F32 = std::is_same_v<R, float>;
  timing_end(ctx, a.threed ? (F32 ? "nbr_apply3d_fp32" : "nbr_apply3d_fp64") : (F32 ? "nbr_apply_fp32" : "nbr_apply_fp64"),
             ev);
  return TMAT_OK;
}

constexpr int MAXR = 4;  // right-hand sides per launch

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
    if (a.fp32) {
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
