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

// one block per node: spectrum of the group for every RHS, then the node's coefficients
// c[q][r][f] = (w_b w_a / 4) sin b cos b e^{-i kz z0} a_f(b, a; A(S_r))
// e^{i arg}: fp64 sincos, or (FAST) the argument reduced modulo 2 pi in fp64 and sincosf
// (|error| ~ 1e-7, the accuracy of the complex64 path)
template <bool FAST>
__device__ __forceinline__ double2 jinc_phase(double arg) {
  if (FAST) {
    const double twopi = 6.283185307179586476925286766559;
    const float red = (float)(arg - twopi * rint(arg * (1.0 / twopi)));
    float s, c;
    sincosf(red, &s, &c);
    return make_double2(c, s);
  }
  double s, c;
  sincos(arg, &s, &c);
  return make_double2(c, s);
}

template <bool FAST>
__global__ void jinc_node_kernel(const double* __restrict__ beta, const double* __restrict__ wbeta, int n_alpha,
                                 int q0, int nq, double k0, double z0, double cell, const double* __restrict__ src_xy,
                                 const double2* __restrict__ src_A, int64_t S, int R, int nmax,
                                 double2* __restrict__ c, double4* __restrict__ kvec) {
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
  __shared__ double2 red[TMAT_MAX_RHS][2][64];
  __shared__ double2 Sv[TMAT_MAX_RHS][2];
  double2 acc[TMAT_MAX_RHS][2];
  for (int r = 0; r < R; ++r) acc[r][0] = acc[r][1] = make_double2(0, 0);
  for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
    const double2 ph = jinc_phase<FAST>(-(kx * src_xy[2 * s] + ky * src_xy[2 * s + 1]));
    for (int r = 0; r < R; ++r) {
      cfma(acc[r][0], ph, src_A[((int64_t)r * S + s) * 2]);
      cfma(acc[r][1], ph, src_A[((int64_t)r * S + s) * 2 + 1]);
    }
  }
  for (int r = 0; r < R; ++r) {
    red[r][0][threadIdx.x] = acc[r][0];
    red[r][1][threadIdx.x] = acc[r][1];
  }
  __syncthreads();
  if (threadIdx.x < 2 * R) {
    const int r = threadIdx.x / 2, comp = threadIdx.x % 2;
    double2 t = make_double2(0, 0);
    for (int i = 0; i < (int)blockDim.x; ++i) t = cadd(t, red[r][comp][i]);  // fixed order
    Sv[r][comp] = t;
  }
  __syncthreads();
  const int L = nmax * (nmax + 2), P = 2 * L;
  double sz, cz;
  sincos(-kz * z0, &sz, &cz);
  const double wq = cell * wbeta[ib] * (2.0 * M_PI / n_alpha) * sb * cb;
  const double2 pre = make_double2(wq * cz, wq * sz);
  for (int t = threadIdx.x; t < R * P; t += blockDim.x) {
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
    double pi, tau;
    pi_tau(l, abs(m), b, &pi, &tau);
    const double mpi = m * pi;
    const double cl = 1.0 / sqrt(2.0 * l * (l + 1));
    double sm, cm;
    sincos(m * a, &sm, &cm);
    const double2 e = make_double2(cm, -sm);
    double2 brk;
    if (p == 0) brk = make_double2(-mpi * bA.y + tau * aA.x, mpi * bA.x + tau * aA.y);
    else brk = make_double2(tau * bA.x + mpi * aA.y, tau * bA.y - mpi * aA.x);
    const int e4 = (l + p) & 3;
    const double ir[4] = {1, 0, -1, 0}, ii[4] = {0, 1, 0, -1};
    double2 v = cmul(cmul(make_double2(ir[e4], ii[e4]), e), brk);
    v = make_double2(-4.0 * cl * v.x, -4.0 * cl * v.y);
    c[((int64_t)ql * R + r) * P + f] = cmul(pre, v);
  }
}

// a0[r][j][f] += sum_{q in chunk} e^{i k_q.x_j} c[q][r][f]
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
          const double2 e = jinc_phase<sizeof(Rl) == 4>(arg);
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
  const int CHUNK = 8192;
  double2* c;
  TM_TRY(scratch(ctx, "jn_c", sizeof(double2) * (size_t)CHUNK * R * P, (void**)&c));
  double4* kv;
  TM_TRY(scratch(ctx, "jn_k", sizeof(double4) * (size_t)CHUNK, (void**)&kv));
  const bool fp32 = precision == TMAT_PREC_MIXED;
  const int NT = 16;
  const size_t smem = (fp32 ? sizeof(float2) : sizeof(double2)) * (size_t)NT * R * P;
  if (smem > 48 * 1024) {
    if (fp32) TM_CUDA(ctx, cudaFuncSetAttribute(jinc_accum_kernel<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else TM_CUDA(ctx, cudaFuncSetAttribute(jinc_accum_kernel<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  for (int64_t q0 = 0; q0 < NQ; q0 += CHUNK) {
    const int nq = (int)std::min<int64_t>(CHUNK, NQ - q0);
    if (fp32)
      jinc_node_kernel<true><<<nq, 64, 0, ctx->stream>>>(dbeta, dwb, n_alpha, (int)q0, nq, k0, z0, cell,
                                                         (const double*)ss.dev, (const double2*)sa.dev, S, R, nmax, c,
                                                         kv);
    else
      jinc_node_kernel<false><<<nq, 64, 0, ctx->stream>>>(dbeta, dwb, n_alpha, (int)q0, nq, k0, z0, cell,
                                                          (const double*)ss.dev, (const double2*)sa.dev, S, R, nmax, c,
                                                          kv);
    TM_LAUNCHED(ctx);
    const unsigned grid = (unsigned)cdiv(N, 16);
    if (fp32)
      jinc_accum_kernel<float, 16><<<grid, 256, smem, ctx->stream>>>(kv, nq, (const double*)sp.dev, N, c, R, P,
                                                                     (double2*)so.dev);
    else
      jinc_accum_kernel<double, 16><<<grid, 256, smem, ctx->stream>>>(kv, nq, (const double*)sp.dev, N, c, R, P,
                                                                      (double2*)so.dev);
    TM_LAUNCHED(ctx);
  }
  TM_TRY(finish_out(ctx, &so));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
