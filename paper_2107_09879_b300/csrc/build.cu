// Per-scatterer T-matrices (Mie), plane-wave incident coefficients and the
// general translation matrices xi(k d).
#include <cmath>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

__device__ __forceinline__ double2 cdiv_(double2 a, double2 b) {
  double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double2 cd(double a) { return make_double2(a, 0.0); }

// Lorenz-Mie coefficients in the logarithmic-derivative form (Bohren & Huffman,
// BHMIE): D_n(mx) = psi_n'(mx)/psi_n(mx) by downward recurrence,
//   a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
//   b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]
// with psi_n = x j_n(x), xi_n = x h_n^(1)(x). Radius derivative by the chain rule
// through x = k r, using D_n' = n(n+1)/z^2 - 1 - D_n^2 and
// psi_n' = psi_{n-1} - n psi_n / x,  psi_{n-1}' = -psi_n + n psi_{n-1} / x (same for xi).
__global__ void mie_kernel(const tmat_atom* __restrict__ atoms, int64_t N, double k, double n_bg, int nmax,
                           double2* __restrict__ T, double2* __restrict__ dT) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int NM = TMAT_NMAX_MAX + 1;
  tmat_atom at = atoms[i];
  double x = k * at.radius;
  double2 m = make_double2(at.n_re / n_bg, at.n_im / n_bg);
  double2 mx = make_double2(m.x * x, m.y * x);
  double sx, cx;
  sincos(x, &sx, &cx);
  // j_n(x) by Miller's downward recurrence, normalised by j_0 or j_1 (whichever is larger)
  double jn[NM + 1];
  {
    int start = nmax + (int)x + 30;
    double jp1 = 0.0, jc = 1e-280, keep0 = 0, keep1 = 0;
    for (int l = start; l >= 1; --l) {
      double jm1 = (2 * l + 1) / x * jc - jp1;
      jp1 = jc;
      jc = jm1;
      if (l - 1 <= nmax) jn[l - 1] = jc;
      if (l - 1 == 0) keep0 = jc;
      if (l - 1 == 1) keep1 = jc;
      if (fabs(jc) > 1e250) {
        jc *= 1e-250;
        jp1 *= 1e-250;
        for (int q = l - 1; q <= nmax; ++q) jn[q] *= 1e-250;
        keep0 *= 1e-250;
        keep1 *= 1e-250;
      }
    }
    double j0 = sx / x, j1 = sx / (x * x) - cx / x;
    double scale = (fabs(j0) >= fabs(j1)) ? j0 / keep0 : j1 / keep1;
    for (int l = 0; l <= nmax; ++l) jn[l] *= scale;
  }
  double yn[NM + 1];
  yn[0] = -cx / x;
  yn[1] = -cx / (x * x) - sx / x;
  for (int l = 1; l < nmax; ++l) yn[l + 1] = (2 * l + 1) / x * yn[l] - yn[l - 1];
  // D_n(mx), n = nmax..1, downward from a high start
  double2 D[NM + 1];
  {
    double amx = sqrt(mx.x * mx.x + mx.y * mx.y);
    int start = (int)fmax((double)nmax, amx) + 20;
    double2 d = cd(0.0);
    for (int n = start; n >= 1; --n) {
      double2 nz = cdiv_(cd((double)n), mx);
      if (n <= nmax) D[n] = d;
      d = csub(nz, cdiv_(cd(1.0), cadd(d, nz)));  // D_{n-1} = n/z - 1/(D_n + n/z)
    }
  }
  const int L = nmax * (nmax + 2);
  for (int n = 1; n <= nmax; ++n) {
    double psi = x * jn[n], psim = x * jn[n - 1];
    double2 xi = make_double2(x * jn[n], x * yn[n]);
    double2 xim = make_double2(x * jn[n - 1], x * yn[n - 1]);
    double nx = n / x;
    double2 A = cadd(cdiv_(D[n], m), cd(nx));
    double2 B = cadd(cmul(m, D[n]), cd(nx));
    double2 Na = csub(cscale(A, psi), cd(psim));
    double2 Da = csub(cmul(A, xi), xim);
    double2 Nb = csub(cscale(B, psi), cd(psim));
    double2 Db = csub(cmul(B, xi), xim);
    double2 a = cdiv_(Na, Da), b = cdiv_(Nb, Db);
    double2 da = cd(0.0), db = cd(0.0);
    if (dT) {
      double2 z2 = cmul(mx, mx);
      double2 Dp = csub(csub(cdiv_(cd(n * (n + 1.0)), z2), cd(1.0)), cmul(D[n], D[n]));
      double2 dA = cscale(csub(Dp, cd(n / (x * x))), k);
      double2 dB = cscale(csub(cmul(cmul(m, m), Dp), cd(n / (x * x))), k);
      double dpsi = k * (psim - n * psi / x);
      double dpsim = k * (-psi + n * psim / x);
      double2 dxi = cscale(csub(xim, cscale(xi, (double)n / x)), k);
      double2 dxim = cscale(cadd(cscale(xi, -1.0), cscale(xim, (double)n / x)), k);
      double2 dNa = csub(cadd(cscale(dA, psi), cscale(A, dpsi)), cd(dpsim));
      double2 dDa = csub(cadd(cmul(dA, xi), cmul(A, dxi)), dxim);
      double2 dNb = csub(cadd(cscale(dB, psi), cscale(B, dpsi)), cd(dpsim));
      double2 dDb = csub(cadd(cmul(dB, xi), cmul(B, dxi)), dxim);
      da = cdiv_(csub(cmul(dNa, Da), cmul(Na, dDa)), cmul(Da, Da));
      db = cdiv_(csub(cmul(dNb, Db), cmul(Nb, dDb)), cmul(Db, Db));
    }
    for (int mm = -n; mm <= n; ++mm) {
      int f = n * (n + 1) + mm - 1;
      T[i * 2 * L + f] = make_double2(-b.x, -b.y);
      T[i * 2 * L + L + f] = make_double2(-a.x, -a.y);
      if (dT) {
        dT[i * 2 * L + f] = make_double2(-db.x, -db.y);
        dT[i * 2 * L + L + f] = make_double2(-da.x, -da.y);
      }
    }
  }
}

// a_{lmp}(b, a) of App. II-A (explicit i^l forms), one thread per (r, flat index)
__global__ void pw_angular_kernel(const double* __restrict__ dirs, const double2* __restrict__ pol, int R, int nmax,
                                  double2* __restrict__ coef) {
  const int L = nmax * (nmax + 2), P = 2 * L;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * P) return;
  int r = t / P, f = t % P;
  int p = f / L, n = f % L;
  int l = 1;
  while ((l + 1) * (l + 1) - 1 <= n) ++l;
  int m = n + 1 - l * (l + 1);
  double beta = dirs[2 * r], alpha = dirs[2 * r + 1];
  double sb, cb, sa, ca;
  sincos(beta, &sb, &cb);
  sincos(alpha, &sa, &ca);
  double2 Ax = pol[3 * r], Ay = pol[3 * r + 1], Az = pol[3 * r + 2];
  double2 bA = make_double2(ca * cb * Ax.x + sa * cb * Ay.x - sb * Az.x, ca * cb * Ax.y + sa * cb * Ay.y - sb * Az.y);
  double2 aA = make_double2(-sa * Ax.x + ca * Ay.x, -sa * Ax.y + ca * Ay.y);
  double pi, tau;
  pi_tau(l, abs(m), beta, &pi, &tau);
  double mpi = m * pi;
  double cl = 1.0 / sqrt(2.0 * l * (l + 1));
  double sm, cm;
  sincos(m * alpha, &sm, &cm);
  double2 e = make_double2(cm, -sm);  // e^{-i m a}
  double2 brk;
  if (p == 0) {  // i m pi (b.A) + tau (a.A)
    brk = make_double2(-mpi * bA.y + tau * aA.x, mpi * bA.x + tau * aA.y);
  } else {       // tau (b.A) - i m pi (a.A)
    brk = make_double2(tau * bA.x + mpi * aA.y, tau * bA.y - mpi * aA.x);
  }
  int e4 = (l + p) & 3;  // i^l (p=0) or i^{l+1} (p=1)
  const double ir[4] = {1, 0, -1, 0}, ii[4] = {0, 1, 0, -1};
  double2 v = cmul(cmul(make_double2(ir[e4], ii[e4]), e), brk);
  coef[t] = make_double2(-4.0 * cl * v.x, -4.0 * cl * v.y);
}

// a0[r][i][f] = e^{i k.x_i} coef[r][f]: the phase of each (r, i) once per block (the block's
// 256 values span at most 256 / P + 2 sites), shared by its P coefficients
__global__ void pw_phase_kernel(const double* __restrict__ pos, int64_t N, double k, const double* __restrict__ dirs,
                                const double2* __restrict__ coef, int R, int P, double2* __restrict__ a0) {
  __shared__ double2 eph[258];
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t tot = (int64_t)R * N * P;
  const int64_t g0 = t0 / P;  // first (r, i) of the block, g = r N + i
  const int64_t glast = (min(t0 + (int64_t)blockDim.x, tot) - 1) / P;
  for (int64_t g = g0 + threadIdx.x; g <= glast; g += blockDim.x) {
    const int r = (int)(g / N);
    const int64_t i = g - (int64_t)r * N;
    double sb, cb, sa, ca;
    sincos(dirs[2 * r], &sb, &cb);
    sincos(dirs[2 * r + 1], &sa, &ca);
    const double ph = k * (sb * ca * pos[3 * i] + sb * sa * pos[3 * i + 1] + cb * pos[3 * i + 2]);
    double s, c;
    sincos(ph, &s, &c);
    eph[g - g0] = make_double2(c, s);
  }
  __syncthreads();
  const int64_t t = t0 + threadIdx.x;
  if (t >= tot) return;
  const int f = (int)(t % P);
  const int r = (int)(t / ((int64_t)P * N));
  a0[t] = cmul(eph[t / P - g0], coef[r * P + f]);
}

// xi(k d) for general displacements: one block per displacement.
template <int NMAX>
__global__ void translation_kernel(const double* __restrict__ disp, int64_t M, double k,
                                   const double2* __restrict__ a5, const double2* __restrict__ b5,
                                   double2* __restrict__ xi) {
  constexpr int L = NMAX * (NMAX + 2), P = 2 * L, Q = 2 * NMAX + 1;
  __shared__ double2 h[Q];
  __shared__ double Pq[Q][Q];     // Pbar_q^mu(cos th)
  __shared__ double2 eph[2 * Q];  // e^{i mu phi}, mu = -(Q-1)..(Q-1)
  int64_t md = blockIdx.x;
  if (md >= M) return;
  double dx = disp[3 * md], dy = disp[3 * md + 1], dz = disp[3 * md + 2];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double ct = dz / r, st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double rho = sqrt(dx * dx + dy * dy);
  double cp = rho > 0 ? dx / rho : 1.0, sp = rho > 0 ? dy / rho : 0.0;
  if (threadIdx.x == 0) {
    double2 hh[Q];
    hankel_up<double, Q>(k * r, hh);
    for (int q = 0; q < Q; ++q) h[q] = hh[q];
    double2 e = make_double2(1, 0), e1 = make_double2(cp, sp);
    for (int mu = 0; mu < Q; ++mu) {
      eph[Q - 1 + mu] = e;
      eph[Q - 1 - mu] = cconj(e);
      e = cmul(e, e1);
    }
  }
  if (threadIdx.x < Q) {
    int mu = threadIdx.x;
    double df = 1.0, f2 = 1.0;
    for (int t = 1; t < 2 * mu; t += 2) df *= t;
    for (int t = 2; t <= 2 * mu; ++t) f2 *= t;
    double pprev = 0.0, pcur = sqrt((2 * mu + 1) / (2.0 * f2)) * df * pow(st, (double)mu);
    for (int q = 0; q < mu; ++q) Pq[q][mu] = 0.0;
    Pq[mu][mu] = pcur;
    for (int q = mu + 1; q < Q; ++q) {
      double a = sqrt((4.0 * q * q - 1) / ((double)q * q - (double)mu * mu));
      double b = sqrt(((q - 1.0) * (q - 1.0) - (double)mu * mu) / (4.0 * (q - 1.0) * (q - 1.0) - 1));
      double pn = a * (ct * pcur - b * pprev);
      pprev = pcur;
      pcur = pn;
      Pq[q][mu] = pn;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    int n = e / L, np = e % L;
    int l = 1, lp = 1;
    while ((l + 1) * (l + 1) - 1 <= n) ++l;
    while ((lp + 1) * (lp + 1) - 1 <= np) ++lp;
    int m = n + 1 - l * (l + 1), mp = np + 1 - lp * (lp + 1);
    int mu = m - mp, amu = abs(mu);
    double2 al = make_double2(0, 0), be = make_double2(0, 0);
    for (int q = abs(l - lp); q <= l + lp; ++q) {
      if (amu > q) continue;
      double2 hp = cscale(h[q], Pq[q][amu]);
      cfma(al, a5[((size_t)n * L + np) * Q + q], hp);
      cfma(be, b5[((size_t)n * L + np) * Q + q], hp);
    }
    al = cmul(al, eph[Q - 1 + mu]);
    be = cmul(be, eph[Q - 1 + mu]);
    double2* X = xi + (size_t)md * P * P;
    X[(size_t)n * P + np] = al;
    X[(size_t)(L + n) * P + L + np] = al;
    X[(size_t)n * P + L + np] = be;
    X[(size_t)(L + n) * P + np] = be;
  }
}

int launch_translation(tmat_ctx* ctx, int nmax, const Tables* t, const double* d_disp, int64_t M, double k,
                       double2* d_xi) {
  if (M == 0) return TMAT_OK;
  dim3 grid((unsigned)M), block(256);
  switch (nmax) {
#define TCASE(NM) \
  case NM: translation_kernel<NM><<<grid, block, 0, ctx->stream>>>(d_disp, M, k, t->d_a5, t->d_b5, d_xi); break;
    TCASE(1) TCASE(2) TCASE(3) TCASE(4) TCASE(5) TCASE(6)
#undef TCASE
    default: return set_error(ctx, TMAT_EINVAL, "nmax %d unsupported", nmax);
  }
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_build(tmat_ctx* ctx, const tmat_atom* atoms, int64_t N, double wavelength, double n_bg, int nmax,
                          tmat_c128* T_diag_out, tmat_c128* dTdr_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || (!atoms && N > 0) || !T_diag_out || !(wavelength > 0) || !(n_bg > 0))
    return set_error(ctx, TMAT_EINVAL, "tmat_build: bad arguments");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX)
    return set_error(ctx, TMAT_EINVAL, "tmat_build: nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  Staged sa, st, sd;
  TM_TRY(stage_in(ctx, "st_atoms", atoms, sizeof(tmat_atom) * N, &sa));
  TM_TRY(stage_out(ctx, "st_T", T_diag_out, sizeof(double2) * N * P, &st));
  TM_TRY(stage_out(ctx, "st_dT", dTdr_out, sizeof(double2) * N * P, &sd));
  double k = 2.0 * M_PI * n_bg / wavelength;
  if (N > 0) {
    mie_kernel<<<(unsigned)cdiv(N, 128), 128, 0, ctx->stream>>>((const tmat_atom*)sa.dev, N, k, n_bg, nmax,
                                                                (double2*)st.dev, (double2*)sd.dev);
    TM_LAUNCHED(ctx);
  }
  TM_TRY(finish_out(ctx, &st));
  TM_TRY(finish_out(ctx, &sd));
  return TMAT_OK;
}

int incident_planewave_dev(tmat_ctx* ctx, const double* d_pos, int64_t N, double k, int nmax, const double* d_dirs,
                           const double2* d_pol, int R, double2* d_a0) {
  const int P = num_coeffs(nmax);
  double2* coef;
  TM_TRY(scratch(ctx, "pw_coef", sizeof(double2) * R * P, (void**)&coef));
  pw_angular_kernel<<<(unsigned)cdiv(R * P, 128), 128, 0, ctx->stream>>>(d_dirs, d_pol, R, nmax, coef);
  TM_LAUNCHED(ctx);
  int64_t tot = (int64_t)R * N * P;
  if (tot > 0) {
    pw_phase_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, ctx->stream>>>(d_pos, N, k, d_dirs, coef, R, P, d_a0);
    TM_LAUNCHED(ctx);
  }
  return TMAT_OK;
}

extern "C" int tmat_incident_planewave(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
                                       int nmax, const double* dirs, const tmat_c128* pol, int R, tmat_c128* a0_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || R < 1 || (!pos && N > 0) || !dirs || !pol || !a0_out || !(wavelength > 0) || !(n_bg > 0))
    return set_error(ctx, TMAT_EINVAL, "tmat_incident_planewave: bad arguments");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  Staged sp, sdir, spol, so;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  TM_TRY(stage_in(ctx, "st_dirs", dirs, sizeof(double) * 2 * R, &sdir));
  TM_TRY(stage_in(ctx, "st_pol", pol, sizeof(double2) * 3 * R, &spol));
  TM_TRY(stage_out(ctx, "st_a0", a0_out, sizeof(double2) * R * N * P, &so));
  double k = 2.0 * M_PI * n_bg / wavelength;
  TM_TRY(incident_planewave_dev(ctx, (const double*)sp.dev, N, k, nmax, (const double*)sdir.dev,
                                (const double2*)spol.dev, R, (double2*)so.dev));
  TM_TRY(finish_out(ctx, &so));
  return TMAT_OK;
}

extern "C" int tmat_translation(tmat_ctx* ctx, int nmax, double k, const double* disp, int64_t M, tmat_c128* xi_out) {
  if (!ctx) return TMAT_EINVAL;
  if (M < 0 || (!disp && M > 0) || !xi_out || !(k > 0)) return set_error(ctx, TMAT_EINVAL, "tmat_translation: bad arguments");
  Tables* t;
  TM_TRY(get_tables(ctx, nmax, &t));
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  Staged sd, so;
  TM_TRY(stage_in(ctx, "st_disp", disp, sizeof(double) * 3 * M, &sd));
  TM_TRY(stage_out(ctx, "st_xi", xi_out, sizeof(double2) * M * P * P, &so));
  TM_TRY(launch_translation(ctx, nmax, t, (const double*)sd.dev, M, k, (double2*)so.dev));
  TM_TRY(finish_out(ctx, &so));
  return TMAT_OK;
}
