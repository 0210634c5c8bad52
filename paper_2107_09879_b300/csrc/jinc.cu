// Incident coefficients of a group of jinc sources (App. II).
//
// Each source on the plane z = z0 at x_s with transverse amplitude A_s is
// (a^2/(4 pi^2)) int_{|k^T|<k0} A_s e^{i k^T.(x^T - x_s)} e^{i k_z (z - z0)} d^2k^T
// (a: pitch of the source grid; the paper's lambda/2 grid gives 1/(4 k0^2)),
// every plane-wave component completed to A(k^T) = A^T - z^ (k^T.A^T)/k_z. About a
// sphere at x_j the group's coefficients are
//   a0_j = (a k0/(2 pi))^2 sum_q w_q sin b cos b e^{i k_q.x_j} e^{-i k_z z0} a_lmp(b, a; A(S(k_q))),
//   S(k^T) = sum_s A_s e^{-i k^T.x_s},
// with the Gauss-Legendre (b in [0, pi/2]) x trapezoid (a) rule q = (b, a).
#include <cmath>
#include <vector>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

// e^{i arg} in fp64 (the fp64 path)
__device__ __forceinline__ double2 jinc_phase64(double arg) {
  double s, c;
  sincos(arg, &s, &c);
  return make_double2(c, s);
}

// ---- complex64 path: phases from double-float (hi + lo fp32 pairs) arithmetic ----
// The FP64 pipe of this part runs at a small fraction of the FP32 rate, so the
// complex64 path keeps fp64 out of every per-(node, sphere) and per-(node, source)
// step: positions and wave vectors are split once into hi + lo float pairs, the
// argument k.x is formed as a double-float (48-bit significand, error-free products
// and sums: Dekker / Knuth), reduced modulo 2 pi by a three-piece Cody-Waite
// reduction, and only the reduced angle goes to sincosf, whose first-order
// correction by the low word keeps the phase at the complex64 rounding level
// (|error| ~ 1e-7) for |k.x| up to 2^13 * 2 pi.
struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl df_split(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
// s + e = a + b exactly (Knuth's two-sum; the _rn intrinsics are never contracted)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.h, -p);  // exact rounding error of the product
  return {p, fmaf(a.h, b.l, fmaf(a.l, b.h, e))};
}
// 2 pi = RC1 + RC2 + RC3: RC1 has 8 significant bits and RC2 11, so n * RC1 and n * RC2
// are exact for |n| < 2^13
constexpr float RC1 = 6.28125f;
constexpr float RC2 = 2029.0f / 1048576.0f;
constexpr float RC3 = 3.0199159819567529e-7f;
constexpr float INV_2PI_F = 0.15915494309189535f;
// (cos, sin) of the double-float angle s + lo
__device__ __forceinline__ float2 sincos_df(float s, float lo) {
  const float n = rintf(s * INV_2PI_F);
  const float t = fmaf(-n, RC1, s);  // exact
  float r, er;
  two_sum(t, __fmul_rn(-n, RC2), r, er);
  float a, al;
  two_sum(r, er + fmaf(-n, RC3, lo), a, al);  // |al| <= ulp(a) / 2: the correction below is first order
  float sn, cs;
  sincosf(a, &sn, &cs);
  return make_float2(cs - sn * al, sn + cs * al);
}
// (cos, sin) of kx x + ky y + kz z
__device__ __forceinline__ float2 phase_df3(dfl kx, dfl ky, dfl kz, dfl x, dfl y, dfl z) {
  const dfl px = df_mul(kx, x), py = df_mul(ky, y), pz = df_mul(kz, z);
  float s1, e1, s2, e2;
  two_sum(px.h, py.h, s1, e1);
  two_sum(s1, pz.h, s2, e2);
  return sincos_df(s2, e1 + e2 + px.l + py.l + pz.l);
}
// (cos, sin) of kx x + ky y
__device__ __forceinline__ float2 phase_df2(dfl kx, dfl ky, dfl x, dfl y) {
  const dfl px = df_mul(kx, x), py = df_mul(ky, y);
  float s1, e1;
  two_sum(px.h, py.h, s1, e1);
  return sincos_df(s1, e1 + px.l + py.l);
}
// (hi, lo) += v with the rounding error kept
__device__ __forceinline__ void df_acc(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  hi = s;
  lo += e;
}

// one block per node: spectrum of the group for every RHS, then the node's coefficients
// c[q][r][f] = (w_b w_a / 4) sin b cos b e^{-i kz z0} a_f(b, a; A(S_r))
// FAST (complex64 path): the spectrum is summed over double-float phases with two-sum
// accumulation per thread, and c is written as complex64; otherwise all in fp64.
template <bool FAST, int RR>
__global__ void __launch_bounds__(64)
jinc_node_kernel(const double* __restrict__ beta, const double* __restrict__ wbeta, int n_alpha, int q0, int nq,
                 double k0, double z0, double cell, const double* __restrict__ src_xy,
                 const double2* __restrict__ src_A, const float4* __restrict__ src_df,
                 const float2* __restrict__ src_A32, int64_t S, int nmax, void* __restrict__ cout,
                 double4* __restrict__ kvec) {
  const int ql = blockIdx.x;
  if (ql >= nq) return;
  const int q = q0 + ql;
  const int ib = q / n_alpha, ia = q % n_alpha;
  const double b = beta[ib], a = 2.0 * M_PI * ia / n_alpha;
  double sb, cb, sa, ca;
  sincos(b, &sb, &cb);
  sincos(a, &sa, &ca);
  const double kx = k0 * sb * ca, ky = k0 * sb * sa, kz = k0 * cb;
  if (threadIdx.x == 0) kvec[ql] = make_double4(kx, ky, kz, 0.0);
  __shared__ double2 red[RR][2][64];
  __shared__ double2 Sv[RR][2];
  if (FAST) {
    // S_r(k) = sum_s A_s e^{-i k.x_s}: complex64 partial sums over 8 sources of the
    // thread's stride, two-sum accumulated into hi + lo pairs
    float hi[RR][2][2], lo[RR][2][2];
    float2 part[RR][2];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        hi[r][u][0] = hi[r][u][1] = lo[r][u][0] = lo[r][u][1] = 0.f;
        part[r][u] = make_float2(0.f, 0.f);
      }
    const dfl mkx = df_split(-kx), mky = df_split(-ky);
    int cnt = 0;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
      const float4 sp = src_df[s];
      const float2 ph = phase_df2(mkx, mky, {sp.x, sp.y}, {sp.z, sp.w});
#pragma unroll
      for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int u = 0; u < 2; ++u) cfma(part[r][u], ph, src_A32[((int64_t)r * S + s) * 2 + u]);
      if (++cnt == 8 || s + (int64_t)blockDim.x >= S) {
        cnt = 0;
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            df_acc(hi[r][u][0], lo[r][u][0], part[r][u].x);
            df_acc(hi[r][u][1], lo[r][u][1], part[r][u].y);
            part[r][u] = make_float2(0.f, 0.f);
          }
      }
    }
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int u = 0; u < 2; ++u)
        red[r][u][threadIdx.x] = make_double2((double)hi[r][u][0] + (double)lo[r][u][0],
                                              (double)hi[r][u][1] + (double)lo[r][u][1]);
  } else {
    double2 acc[RR][2];
#pragma unroll
    for (int r = 0; r < RR; ++r) acc[r][0] = acc[r][1] = make_double2(0, 0);
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
      const double2 ph = jinc_phase64(-(kx * src_xy[2 * s] + ky * src_xy[2 * s + 1]));
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        cfma(acc[r][0], ph, src_A[((int64_t)r * S + s) * 2]);
        cfma(acc[r][1], ph, src_A[((int64_t)r * S + s) * 2 + 1]);
      }
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      red[r][0][threadIdx.x] = acc[r][0];
      red[r][1][threadIdx.x] = acc[r][1];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * RR) {
    const int r = threadIdx.x / 2, comp = threadIdx.x % 2;
    double2 t = make_double2(0, 0);
    for (int i = 0; i < (int)blockDim.x; ++i) t = cadd(t, red[r][comp][i]);  // fixed order
    Sv[r][comp] = t;
  }
  __syncthreads();
  const int L = nmax * (nmax + 2), P = 2 * L;
  // angular factors per (l, m), shared by both parities and every RHS
  __shared__ double pis[TMAT_NMAX_MAX * (TMAT_NMAX_MAX + 2)], taus[TMAT_NMAX_MAX * (TMAT_NMAX_MAX + 2)];
  __shared__ double2 ema[2 * TMAT_NMAX_MAX + 1];  // e^{-i m a}, m = -nmax..nmax
  for (int n = threadIdx.x; n < L; n += blockDim.x) {
    int l = 1;
    while ((l + 1) * (l + 1) - 1 <= n) ++l;
    const int m = n + 1 - l * (l + 1);
    double pi, tau;
    pi_tau(l, abs(m), b, &pi, &tau);
    pis[n] = pi;
    taus[n] = tau;
  }
  if (threadIdx.x < 2 * nmax + 1) {
    const int m = (int)threadIdx.x - nmax;
    double sm, cm;
    sincos(m * a, &sm, &cm);
    ema[threadIdx.x] = make_double2(cm, -sm);
  }
  __syncthreads();
  double sz, cz;
  sincos(-kz * z0, &sz, &cz);
  const double wq = cell * wbeta[ib] * (2.0 * M_PI / n_alpha) * sb * cb;
  const double2 pre = make_double2(wq * cz, wq * sz);
  for (int t = threadIdx.x; t < RR * P; t += blockDim.x) {
    const int r = t / P, f = t % P;
    const int p = f / L, n = f % L;
    int l = 1;
    while ((l + 1) * (l + 1) - 1 <= n) ++l;
    const int m = n + 1 - l * (l + 1);
    const double2 Sx = Sv[r][0], Sy = Sv[r][1];
    // beta^.A = (k^T^.S)/cos b ; alpha^.A = -sin a Sx + cos a Sy
    const double2 kS = make_double2(ca * Sx.x + sa * Sy.x, ca * Sx.y + sa * Sy.y);
    const double2 bA = make_double2(kS.x / cb, kS.y / cb);
    const double2 aA = make_double2(-sa * Sx.x + ca * Sy.x, -sa * Sx.y + ca * Sy.y);
    const double pi = pis[n], tau = taus[n];
    const double mpi = m * pi;
    const double cl = 1.0 / sqrt(2.0 * l * (l + 1));
    double2 brk;
    if (p == 0) brk = make_double2(-mpi * bA.y + tau * aA.x, mpi * bA.x + tau * aA.y);
    else brk = make_double2(tau * bA.x + mpi * aA.y, tau * bA.y - mpi * aA.x);
    // i^{l+p} e^{-i m a}
    const int e4 = (l + p) & 3;
    const double ir = e4 == 0 ? 1.0 : (e4 == 2 ? -1.0 : 0.0), ii = e4 == 1 ? 1.0 : (e4 == 3 ? -1.0 : 0.0);
    double2 v = cmul(cmul(make_double2(ir, ii), ema[m + nmax]), brk);
    v = cmul(pre, make_double2(-4.0 * cl * v.x, -4.0 * cl * v.y));
    const int64_t o = ((int64_t)ql * RR + r) * P + f;
    if (FAST) reinterpret_cast<float2*>(cout)[o] = make_float2((float)v.x, (float)v.y);
    else reinterpret_cast<double2*>(cout)[o] = v;
  }
}

// complex64 path, per source: position as (x_hi, x_lo, y_hi, y_lo) and amplitudes as complex64
__global__ void jinc_src_split_kernel(const double* __restrict__ src_xy, const double2* __restrict__ src_A, int64_t S,
                                      int R, float4* __restrict__ src_df, float2* __restrict__ src_A32) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const dfl x = df_split(src_xy[2 * s]), y = df_split(src_xy[2 * s + 1]);
  src_df[s] = make_float4(x.h, x.l, y.h, y.l);
  for (int r = 0; r < R; ++r)
    for (int u = 0; u < 2; ++u) {
      const double2 A = src_A[((int64_t)r * S + s) * 2 + u];
      src_A32[((int64_t)r * S + s) * 2 + u] = make_float2((float)A.x, (float)A.y);
    }
}

// complex64 path, E[q][j] = e^{i k_q.x_j} for the chunk's nodes (rows j >= N are zero).
// block: 256 spheres x JP_NODES nodes; the nodes' wave vectors are split once per block.
constexpr int JP_NODES = 32;
__global__ void __launch_bounds__(256)
jinc_phase32_kernel(const double4* __restrict__ kvec, int nq, const double* __restrict__ pos, int64_t N, int ldE,
                    float2* __restrict__ E) {
  __shared__ dfl kd[JP_NODES][3];
  const int q0 = blockIdx.y * JP_NODES;
  if (threadIdx.x < JP_NODES && q0 + (int)threadIdx.x < nq) {
    const double4 k = kvec[q0 + threadIdx.x];
    kd[threadIdx.x][0] = df_split(k.x);
    kd[threadIdx.x][1] = df_split(k.y);
    kd[threadIdx.x][2] = df_split(k.z);
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ldE) return;
  const bool live = j < N;
  const dfl x = df_split(live ? pos[3 * j] : 0.0), y = df_split(live ? pos[3 * j + 1] : 0.0),
            z = df_split(live ? pos[3 * j + 2] : 0.0);
  const int nt = min(JP_NODES, nq - q0);
  for (int t = 0; t < nt; ++t) {
    const float2 ph = live ? phase_df3(kd[t][0], kd[t][1], kd[t][2], x, y, z) : make_float2(0.f, 0.f);
    E[(int64_t)(q0 + t) * ldE + j] = ph;
  }
}

// complex64 path, a0[r][j][f] += sum_q E[q][j] c[q][col], col = r P + f: a complex
// GEMM on the CUDA cores (the node axis q is the contraction). Block tile BM spheres x
// BN columns, JG_BK nodes per stage, register-staged double buffering; each thread
// owns 4 x 4 outputs. Partial sums run in fp32 over JG_FLUSH nodes and are then
// two-sum accumulated into hi + lo pairs, so the result keeps ~1e-7 relative accuracy
// over thousands of nodes.
constexpr int JG_BK = 16;
constexpr int JG_FLUSH = 32;
template <int BN>
__global__ void __launch_bounds__(256, 1)
jinc_gemm32_kernel(const float2* __restrict__ E, int ldE, int64_t N, int nq_all, int kper,
                   const float2* __restrict__ cq_all, int RP, int P, double2* __restrict__ a0,
                   double2* __restrict__ part) {
  // blockIdx.z takes nodes [z kper, (z + 1) kper) of the chunk; with one split the
  // block adds into a0, otherwise it writes its own partial slice part[z] (same layout)
  const int kz0 = blockIdx.z * kper;
  const int nq = min(kper, nq_all - kz0);
  if (nq <= 0) return;
  E += (int64_t)kz0 * ldE;
  const float2* __restrict__ cq = cq_all + (int64_t)kz0 * RP;
  constexpr int BM = 4096 / BN;
  constexpr int TX = BN / 4;
  constexpr int NA = JG_BK * BM / 2 / 256;  // float4 loads per thread per stage
  constexpr int NB = JG_BK * BN / 2 / 256;
  __shared__ __align__(16) float2 As[2][JG_BK][BM];
  __shared__ __align__(16) float2 Bs[2][JG_BK][BN];
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  float4 ra[NA], rb[NB];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int e = tid + 256 * i, k = e / (BM / 2), mm = (e % (BM / 2)) * 2;
      ra[i] = (k0 + k < nq && m0 + mm < ldE)
                  ? *reinterpret_cast<const float4*>(E + (int64_t)(k0 + k) * ldE + m0 + mm)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int e = tid + 256 * i, k = e / (BN / 2), nn = (e % (BN / 2)) * 2;
      rb[i] = (k0 + k < nq && n0 + nn < RP)
                  ? *reinterpret_cast<const float4*>(cq + (int64_t)(k0 + k) * RP + n0 + nn)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int e = tid + 256 * i, k = e / (BM / 2), mm = (e % (BM / 2)) * 2;
      *reinterpret_cast<float4*>(&As[buf][k][mm]) = ra[i];
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int e = tid + 256 * i, k = e / (BN / 2), nn = (e % (BN / 2)) * 2;
      *reinterpret_cast<float4*>(&Bs[buf][k][nn]) = rb[i];
    }
  };
  float2 acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[i][u] = hi[i][u] = lo[i][u] = make_float2(0.f, 0.f);
  const int ntile = (nq + JG_BK - 1) / JG_BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < ntile; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ntile) load((kt + 1) * JG_BK);
#pragma unroll
    for (int k = 0; k < JG_BK; ++k) {
      const float4 a01 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a23 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4 + 2]);
      const float4 b01 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float4 b23 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4 + 2]);
      const float2 av[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                            make_float2(a23.z, a23.w)};
      const float2 bv[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                            make_float2(b23.z, b23.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) cfma(acc[i][u], av[i], bv[u]);
    }
    if (((kt + 1) * JG_BK) % JG_FLUSH == 0 || kt + 1 == ntile) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          df_acc(hi[i][u].x, lo[i][u].x, acc[i][u].x);
          df_acc(hi[i][u].y, lo[i][u].y, acc[i][u].y);
          acc[i][u] = make_float2(0.f, 0.f);
        }
    }
    if (kt + 1 < ntile) {
      store(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= N) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int col = n0 + tx * 4 + u;
      if (col >= RP) continue;
      const int r = col / P, f = col % P;
      const int64_t o = ((int64_t)r * N + m) * P + f;
      const double2 v =
          make_double2((double)hi[i][u].x + (double)lo[i][u].x, (double)hi[i][u].y + (double)lo[i][u].y);
      if (part) part[(int64_t)blockIdx.z * N * RP + o] = v;
      else a0[o] = cadd(a0[o], v);
    }
  }
}

// a0[e] += sum_z part[z][e], z in increasing order
__global__ void jinc_split_reduce_kernel(const double2* __restrict__ part, int nsplit, int64_t n,
                                         double2* __restrict__ a0) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double2 t = a0[e];
  for (int z = 0; z < nsplit; ++z) t = cadd(t, part[(int64_t)z * n + e]);
  a0[e] = t;
}

// fp64 path: a0[r][j][f] += sum_{q in chunk} e^{i k_q.x_j} c[q][r][f]
// block: 16 spheres x 16 lanes; a lane owns f = lane, lane + 16, ... for every r.
constexpr int JN_TILE = 16;
template <typename Rl, int NT>
__global__ void __launch_bounds__(256)
jinc_accum_kernel(const double4* __restrict__ kvec, int nq, const double* __restrict__ pos, int64_t N,
                  const double2* __restrict__ c, int R, int P, double2* __restrict__ a0) {
  constexpr int FMAX = (2 * TMAT_NMAX_MAX * (TMAT_NMAX_MAX + 2) + 15) / 16;
  __shared__ C<Rl> ph[16][NT];
  extern __shared__ __align__(16) unsigned char jsm[];
  C<Rl>* ct = reinterpret_cast<C<Rl>*>(jsm);  // [NT][R][P]
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int64_t j = (int64_t)blockIdx.x * 16 + ty;
  const bool live = j < N;
  const double xj = live ? pos[3 * j] : 0, yj = live ? pos[3 * j + 1] : 0, zj = live ? pos[3 * j + 2] : 0;
  double2 acc64[TMAT_MAX_RHS > 4 ? 4 : TMAT_MAX_RHS][FMAX];
  for (int r = 0; r < R && r < 4; ++r)
    for (int u = 0; u < FMAX; ++u) acc64[r][u] = make_double2(0, 0);
  for (int t0 = 0; t0 < nq; t0 += NT) {
    const int nt = min(NT, nq - t0);
    // phases of this tile for the block's 16 spheres
    {
      const int sj = threadIdx.x / NT, tq = threadIdx.x % NT;  // 256 = 16 x 16 (NT = 16) or 8 x 32
      for (int e = threadIdx.x; e < 16 * NT; e += 256) {
        const int sj2 = e / NT, tq2 = e % NT;
        (void)sj; (void)tq;
        const int64_t jj = (int64_t)blockIdx.x * 16 + sj2;
        C<Rl> v = mk<Rl>(0, 0);
        if (tq2 < nt && jj < N) {
          const double4 kq = kvec[t0 + tq2];
          const double arg = kq.x * pos[3 * jj] + kq.y * pos[3 * jj + 1] + kq.z * pos[3 * jj + 2];
          const double2 e = jinc_phase64(arg);
          v = mk<Rl>((Rl)e.x, (Rl)e.y);
        }
        ph[sj2][tq2] = v;
      }
      for (int e = threadIdx.x; e < nt * R * P; e += 256) {
        const double2 cv = c[(int64_t)(t0) * R * P + e];
        ct[e] = mk<Rl>((Rl)cv.x, (Rl)cv.y);
      }
    }
    __syncthreads();
    if (live) {
      for (int r = 0; r < R && r < 4; ++r) {
        C<Rl> part[FMAX];
        for (int u = 0; u < FMAX; ++u) part[u] = mk<Rl>(0, 0);
        for (int tq = 0; tq < nt; ++tq) {
          const C<Rl> p = ph[ty][tq];
          const C<Rl>* crow = ct + ((size_t)tq * R + r) * P;
#pragma unroll
          for (int u = 0; u < FMAX; ++u) {
            const int f = tx + 16 * u;
            if (f < P) cfma(part[u], p, crow[f]);
          }
        }
        for (int u = 0; u < FMAX; ++u) acc64[r][u] = cadd(acc64[r][u], make_double2(part[u].x, part[u].y));
      }
    }
    __syncthreads();
  }
  if (live) {
    for (int r = 0; r < R && r < 4; ++r)
      for (int u = 0; u < FMAX; ++u) {
        const int f = tx + 16 * u;
        if (f < P) {
          double2* o = a0 + ((int64_t)r * N + j) * P + f;
          *o = cadd(*o, acc64[r][u]);
        }
      }
  }
}

// Gauss-Legendre nodes and weights on [0, pi/2] by Newton iteration on P_n
static void gauss_legendre_half_pi(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      dp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    // node on [-1, 1] -> [0, pi/2]
    x[i] = (z + 1.0) * (M_PI / 4.0);
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp) * (M_PI / 4.0);
  }
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_incident_jinc(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
                                  int nmax, const double* src_xy, const tmat_c128* src_A, int64_t S, int R,
                                  double z0, double src_pitch, int n_beta, int n_alpha, int precision,
                                  tmat_c128* a0_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || S < 0 || R < 1 || R > 4 || (N > 0 && (!pos || !a0_out)) || (S > 0 && (!src_xy || !src_A)) ||
      !(wavelength > 0) || !(n_bg > 0) || (precision != TMAT_PREC_FP64 && precision != TMAT_PREC_MIXED))
    return set_error(ctx, TMAT_EINVAL, "tmat_incident_jinc: bad arguments (R must be 1..4)");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  const double k0 = 2.0 * M_PI * n_bg / wavelength;
  // weight of one source: its grid cell a^2/(4 pi^2) times k0^2 from the measure
  const double cell = src_pitch > 0 ? (src_pitch * k0 / (2.0 * M_PI)) * (src_pitch * k0 / (2.0 * M_PI)) : 0.25;
  Staged sp, ss, sa, so;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  TM_TRY(stage_in(ctx, "st_srcxy", src_xy, sizeof(double) * 2 * S, &ss));
  TM_TRY(stage_in(ctx, "st_srcA", src_A, sizeof(double2) * 2 * S * R, &sa));
  TM_TRY(stage_out(ctx, "st_a0j", a0_out, sizeof(double2) * R * N * P, &so));
  if (N == 0) return TMAT_OK;
  TM_CUDA(ctx, cudaMemsetAsync(so.dev, 0, sizeof(double2) * R * N * P, ctx->stream));
  if (S == 0) return finish_out(ctx, &so);
  if (n_beta <= 0 || n_alpha <= 0) {
    // size the rule from the largest sphere-source separation (bounding boxes)
    std::vector<double> hp(3 * N), hs(2 * S);
    TM_CUDA(ctx, cudaMemcpyAsync(hp.data(), sp.dev, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaMemcpyAsync(hs.data(), ss.dev, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double mx[3] = {1e300, 1e300, 1e300}, Mx[3] = {-1e300, -1e300, -1e300}, ms[2] = {1e300, 1e300}, Ms[2] = {-1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
      for (int d = 0; d < 3; ++d) mx[d] = fmin(mx[d], hp[3 * i + d]), Mx[d] = fmax(Mx[d], hp[3 * i + d]);
    for (int64_t s = 0; s < S; ++s)
      for (int d = 0; d < 2; ++d) ms[d] = fmin(ms[d], hs[2 * s + d]), Ms[d] = fmax(Ms[d], hs[2 * s + d]);
    double ex = fmax(Mx[0] - ms[0], Ms[0] - mx[0]), ey = fmax(Mx[1] - ms[1], Ms[1] - mx[1]);
    double ez = fmax(fabs(Mx[2] - z0), fabs(mx[2] - z0));
    const double kd = k0 * sqrt(ex * ex + ey * ey + ez * ez);
    n_beta = (int)ceil(kd * M_PI / 4.0) + 24;
    n_alpha = (int)ceil(kd) + 32;
    n_alpha += (4 - n_alpha % 4) % 4;
  }
  std::vector<double> gx, gw;
  gauss_legendre_half_pi(n_beta, gx, gw);
  double *dbeta, *dwb;
  TM_TRY(scratch(ctx, "jn_beta", sizeof(double) * n_beta, (void**)&dbeta));
  TM_TRY(scratch(ctx, "jn_wbeta", sizeof(double) * n_beta, (void**)&dwb));
  TM_CUDA(ctx, cudaMemcpyAsync(dbeta, gx.data(), sizeof(double) * n_beta, cudaMemcpyHostToDevice, ctx->stream));
  TM_CUDA(ctx, cudaMemcpyAsync(dwb, gw.data(), sizeof(double) * n_beta, cudaMemcpyHostToDevice, ctx->stream));
  const int64_t NQ = (int64_t)n_beta * n_alpha;
  const bool fp32 = precision == TMAT_PREC_MIXED;
  const int RP = R * P;
  // complex64 path: the phase matrix of a chunk is held in HBM, at most ~128 MB of it
  const int ldE = (int)((N + 3) / 4 * 4);
  int CHUNK = 8192;
  if (fp32) {
    const int64_t fit = ((int64_t)128 << 20) / ((int64_t)ldE * (int64_t)sizeof(float2));
    CHUNK = (int)std::max<int64_t>(JG_FLUSH, std::min<int64_t>(8192, fit / JG_FLUSH * JG_FLUSH));
  }
  void* c;
  TM_TRY(scratch(ctx, "jn_c", sizeof(double2) * (size_t)CHUNK * RP, &c));
  double4* kv;
  TM_TRY(scratch(ctx, "jn_k", sizeof(double4) * (size_t)CHUNK, (void**)&kv));
  float4* sdf = nullptr;
  float2 *sA32 = nullptr, *E = nullptr;
  if (fp32) {
    TM_TRY(scratch(ctx, "jn_sdf", sizeof(float4) * (size_t)S, (void**)&sdf));
    TM_TRY(scratch(ctx, "jn_sa32", sizeof(float2) * 2 * (size_t)S * R, (void**)&sA32));
    TM_TRY(scratch(ctx, "jn_E", sizeof(float2) * (size_t)CHUNK * ldE, (void**)&E));
    jinc_src_split_kernel<<<(unsigned)cdiv(S, 256), 256, 0, ctx->stream>>>((const double*)ss.dev,
                                                                          (const double2*)sa.dev, S, R, sdf, sA32);
    TM_LAUNCHED(ctx);
  }
  const int NT = 16;
  const size_t smem = sizeof(double2) * (size_t)NT * RP;
  if (!fp32 && smem > 48 * 1024)
    TM_CUDA(ctx, cudaFuncSetAttribute(jinc_accum_kernel<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  const bool narrow = RP <= 32;
  for (int64_t q0 = 0; q0 < NQ; q0 += CHUNK) {
    const int nq = (int)std::min<int64_t>(CHUNK, NQ - q0);
    cudaEvent_t ev_n = timing_begin(ctx);
#define JN_NODE(F, RR)                                                                                          \
  jinc_node_kernel<F, RR><<<nq, 64, 0, ctx->stream>>>(dbeta, dwb, n_alpha, (int)q0, nq, k0, z0, cell,          \
                                                      (const double*)ss.dev, (const double2*)sa.dev, sdf, sA32, S, \
                                                      nmax, c, kv)
    switch (R * 2 + (fp32 ? 1 : 0)) {
      case 2: JN_NODE(false, 1); break;
      case 3: JN_NODE(true, 1); break;
      case 4: JN_NODE(false, 2); break;
      case 5: JN_NODE(true, 2); break;
      case 6: JN_NODE(false, 3); break;
      case 7: JN_NODE(true, 3); break;
      case 8: JN_NODE(false, 4); break;
      default: JN_NODE(true, 4); break;
    }
#undef JN_NODE
    TM_LAUNCHED(ctx);
    timing_end(ctx, "jinc_nodes", ev_n);
    if (fp32) {
      cudaEvent_t ev_p = timing_begin(ctx);
      jinc_phase32_kernel<<<dim3((unsigned)cdiv(ldE, 256), (unsigned)cdiv(nq, JP_NODES)), 256, 0, ctx->stream>>>(
          kv, nq, (const double*)sp.dev, N, ldE, E);
      TM_LAUNCHED(ctx);
      timing_end(ctx, "jinc_phase32", ev_p, (double)nq * ldE * sizeof(float2));
      // split the node axis so that the grid fills the SMs (one resident block per SM)
      const int BM = narrow ? 128 : 64, BN = narrow ? 32 : 64;
      const int64_t bxy = cdiv(ldE, BM) * cdiv(RP, BN);
      int nsplit = 1;
      double best = 0.0;
      for (int z = 1; z <= 16 && (int64_t)z * JG_FLUSH <= nq; ++z) {
        const double blocks = (double)(bxy * z), waves = std::ceil(blocks / ctx->num_sms);
        const double eff = blocks / (waves * ctx->num_sms);
        if (eff > best + 0.05) best = eff, nsplit = z;
      }
      const int kper = (int)cdiv(cdiv(nq, nsplit), JG_FLUSH) * JG_FLUSH;
      nsplit = (int)cdiv(nq, kper);
      double2* part = nullptr;
      if (nsplit > 1) TM_TRY(scratch(ctx, "jn_part", sizeof(double2) * (size_t)nsplit * N * RP, (void**)&part));
      cudaEvent_t ev_g = timing_begin(ctx);
      const dim3 grid((unsigned)cdiv(ldE, BM), (unsigned)cdiv(RP, BN), (unsigned)nsplit);
      if (narrow)
        jinc_gemm32_kernel<32><<<grid, 256, 0, ctx->stream>>>(E, ldE, N, nq, kper, (const float2*)c, RP, P,
                                                              (double2*)so.dev, part);
      else
        jinc_gemm32_kernel<64><<<grid, 256, 0, ctx->stream>>>(E, ldE, N, nq, kper, (const float2*)c, RP, P,
                                                              (double2*)so.dev, part);
      TM_LAUNCHED(ctx);
      if (nsplit > 1) {
        const int64_t n = N * (int64_t)RP;
        jinc_split_reduce_kernel<<<(unsigned)cdiv(n, 256), 256, 0, ctx->stream>>>(part, nsplit, n, (double2*)so.dev);
        TM_LAUNCHED(ctx);
      }
      timing_end(ctx, "jinc_gemm32", ev_g);
    } else {
      cudaEvent_t ev_a = timing_begin(ctx);
      jinc_accum_kernel<double, 16><<<(unsigned)cdiv(N, 16), 256, smem, ctx->stream>>>(
          kv, nq, (const double*)sp.dev, N, (const double2*)c, R, P, (double2*)so.dev);
      TM_LAUNCHED(ctx);
      timing_end(ctx, "jinc_accum64", ev_a);
    }
  }
  TM_TRY(finish_out(ctx, &so));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
