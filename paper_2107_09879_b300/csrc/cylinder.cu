// Null-field T-matrices of upright circular cylinders (App. I-B, Eq. def_tmatrix and the P,
// Q surface integrals), in fp64 on the GPU.
//
// For a scatterer with wave number k_s inside and k_b outside, rows nu = (l, m, p) (outside
// index) and columns mu = (l', m', p') (inside index):
//   P[nu, mu] = int_surface [ RPhi_mu(k_s x) x Phi_{l,-m,1-p}(k_b x)
//                             + (k_s / k_b) RPhi_{l',m',1-p'}(k_s x) x Phi_{l,-m,p}(k_b x) ] . n dA
//   Q[nu, mu] = the same with RPhi(k_b x) in place of Phi(k_b x)
//   T = -Q P^-1
// (the integrals over the scatterer surface; the two terms added; T = -Q P^-1: the order that
// reduces to the Lorenz-Mie coefficients on a sphere). For a body of revolution about z the
// surface normal has no azimuthal component and every integrand carries e^{i(m' - m) phi},
// so the azimuthal integral is 2 pi delta_{m m'}: T is block-diagonal in m, and each block
// needs only a line integral over the generating profile (bottom disc, side, top disc), done
// by Gauss-Legendre quadrature with n_quad nodes per face. One CTA per (cylinder, m): the
// VSWF components at a chunk of profile points are staged in shared memory, one thread per
// matrix entry accumulates P and Q, and one thread solves T_m P_m = -Q_m by Gaussian
// elimination with partial pivoting (blocks of at most 2 nmax unknowns).
#include <cmath>
#include <vector>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

constexpr int CYL_NL = TMAT_NMAX_MAX;      // l values per m-block at most
constexpr int CYL_D = 2 * CYL_NL;          // block dimension at most
constexpr int CYL_CHUNK = 16;              // profile points staged per pass
constexpr int CYL_THREADS = 160;           // >= CYL_D^2 entries (144)

struct CylGeom {
  double radius, height;
  double2 m_rel;  // refractive index relative to the background
};

// a / b by Smith's method (no squared magnitudes, so no overflow or underflow of |b|^2)
__host__ __device__ __forceinline__ double2 cd_div(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__host__ __device__ __forceinline__ double2 cd_sin(double2 z) {
  return make_double2(sin(z.x) * cosh(z.y), cos(z.x) * sinh(z.y));
}
__host__ __device__ __forceinline__ double2 cd_cos(double2 z) {
  return make_double2(cos(z.x) * cosh(z.y), -sin(z.x) * sinh(z.y));
}
__host__ __device__ __forceinline__ double cd_abs2(double2 z) { return z.x * z.x + z.y * z.y; }

// j_0 .. j_n (n <= CYL_NL) of a complex argument by Miller's downward recurrence
// j_{l-1} = (2l + 1)/z j_l - j_{l+1}, started far above n and normalised with whichever of
// j_0 = sin z / z and j_1 = sin z / z^2 - cos z / z is larger (their zeros interlace).
__host__ __device__ void sph_j_complex(double2 z, int n, double2* out) {
  const double az = sqrt(cd_abs2(z));
  const int start = n + 24 + (int)az;
  double2 jp1 = make_double2(0.0, 0.0), jc = make_double2(1e-30, 0.0);  // the scale is arbitrary
  double2 keep[CYL_NL + 2];
  for (int l = 0; l <= CYL_NL + 1; ++l) keep[l] = make_double2(0.0, 0.0);
  const double2 iz = cd_div(make_double2(1.0, 0.0), z);
  for (int l = start; l > 0; --l) {
    const double2 jm1 = csub(cscale(cmul(iz, jc), (double)(2 * l + 1)), jp1);
    jp1 = jc;
    jc = jm1;
    if (l - 1 <= n + 1) keep[l - 1] = jc;
    if (cd_abs2(jc) > 1e200) {  // rescale (the ratios are all that matter)
      jp1 = cscale(jp1, 1e-100);
      jc = cscale(jc, 1e-100);
      for (int q = 0; q <= CYL_NL + 1; ++q) keep[q] = cscale(keep[q], 1e-100);
    }
  }
  const double2 s = cd_sin(z), c = cd_cos(z);
  const double2 j0 = cmul(s, iz);
  const double2 j1 = csub(cmul(s, cmul(iz, iz)), cmul(c, iz));
  const double2 scale = cd_abs2(j0) >= cd_abs2(j1) ? cd_div(j0, keep[0]) : cd_div(j1, keep[1]);
  for (int l = 0; l <= n; ++l) out[l] = cmul(keep[l], scale);
}

// normalised Legendre functions (no Condon-Shortley phase) at cos(theta) = ct, sin = st:
// Pbar_l^am, pi_l^am = Pbar_l^am / sin (am >= 1) and tau_l^am = d Pbar_l^am / d theta, l <= nmax
__host__ __device__ void legendre_row(int nmax, int am, double ct, double st, double* Pb, double* pi, double* tau) {
  // Pbar_l^mu for mu = am and, for tau at am = 0, mu = 1
  auto rowP = [&](int mu, double* out, bool over_sin) {
    for (int l = 0; l <= nmax; ++l) out[l] = 0.0;
    if (mu > nmax) return;
    double df = 1.0, f2 = 1.0;
    for (int q = 1; q < 2 * mu; q += 2) df *= q;
    for (int q = 2; q <= 2 * mu; ++q) f2 *= q;
    double base = sqrt((2 * mu + 1) / (2.0 * f2)) * df;
    const int pw = over_sin ? mu - 1 : mu;
    for (int q = 0; q < pw; ++q) base *= st;
    double pm2 = 0.0, pm1 = base;
    out[mu] = base;
    for (int l = mu + 1; l <= nmax; ++l) {
      const double a = sqrt((4.0 * l * l - 1) / ((double)l * l - (double)mu * mu));
      const double b = sqrt(((l - 1.0) * (l - 1.0) - (double)mu * mu) / (4.0 * (l - 1.0) * (l - 1.0) - 1));
      const double v = a * (ct * pm1 - b * pm2);
      pm2 = pm1;
      pm1 = v;
      out[l] = v;
    }
  };
  rowP(am, Pb, false);
  if (am >= 1) {
    rowP(am, pi, true);
    for (int l = 0; l <= nmax; ++l) {
      const double tl = (l >= 1 && am <= l) ? sqrt((2.0 * l + 1) * ((double)l * l - (double)am * am) / (2.0 * l - 1)) : 0.0;
      tau[l] = (am <= l) ? (l * ct * pi[l] - tl * (l >= 1 ? pi[l - 1] : 0.0)) : 0.0;
    }
  } else {
    double p1[CYL_NL + 1];
    rowP(1, p1, false);
    for (int l = 0; l <= nmax; ++l) {
      pi[l] = 0.0;
      tau[l] = -sqrt(l * (l + 1.0)) * p1[l];
    }
  }
}

// One profile point: its spherical position, outward normal components (n_r, n_theta) and
// weight (line element times the profile radius; the 2 pi of the azimuth is applied at the end).
struct ProfilePoint {
  double r, ct, st, nr, nt, w;
};

__host__ __device__ ProfilePoint profile_point(const CylGeom& g, int q, int nq, const double* __restrict__ gx,
                                      const double* __restrict__ gw) {
  const int face = q / nq, j = q % nq;
  const double a = g.radius, h = g.height;
  double rho, z, w, nx, nz;  // normal in the (rho, z) plane
  if (face == 1) {           // side: rho = a, z in [-h/2, h/2], dA / dphi = a dz
    rho = a;
    z = 0.5 * h * gx[j];
    w = 0.5 * h * gw[j] * a;
    nx = 1.0;
    nz = 0.0;
  } else {  // discs: z = -+h/2, rho in [0, a], dA / dphi = rho drho
    rho = 0.5 * a * (gx[j] + 1.0);
    z = face == 0 ? -0.5 * h : 0.5 * h;
    w = 0.5 * a * gw[j] * rho;
    nx = 0.0;
    nz = face == 0 ? -1.0 : 1.0;
  }
  ProfilePoint p;
  p.r = sqrt(rho * rho + z * z);
  p.ct = z / p.r;
  p.st = rho / p.r;
  // r^ = (st, ct), theta^ = (ct, -st) in (rho, z) components
  p.nr = nx * p.st + nz * p.ct;
  p.nt = nx * p.ct - nz * p.st;
  p.w = w;
  return p;
}

// VSWF components (r, theta, phi) without the azimuthal phase, for the block's order m:
// inside RPhi_{l, m, p}(k_s x); outside Phi_{l, -m, p}(k_b x) and RPhi_{l, -m, p}(k_b x).
// Index within the block: i = p * nl + (l - lmin).
template <int NMAX>
__device__ void block_functions(const ProfilePoint& pt, int m, double kb, double2 ks, double2 (*fin)[3],
                                double2 (*fout)[3], double2 (*freg)[3]) {
  const int am = m < 0 ? -m : m, lmin = am > 1 ? am : 1, nl = NMAX - lmin + 1;
  double Pb[NMAX + 1], pi[NMAX + 1], tau[NMAX + 1];
  legendre_row(NMAX, am, pt.ct, pt.st, Pb, pi, tau);
  double2 hk[NMAX + 2];
  hankel_up<double, NMAX + 2>(kb * pt.r, hk);
  double2 jb[CYL_NL + 1], js[CYL_NL + 1];
  sph_j_complex(make_double2(kb * pt.r, 0.0), NMAX, jb);
  const double2 zs = cscale(ks, pt.r);
  sph_j_complex(zs, NMAX, js);
  const double kr = kb * pt.r;
  const double2 izs = cd_div(make_double2(1.0, 0.0), zs);
  for (int l = lmin; l <= NMAX; ++l) {
    const int i = l - lmin;
    const double cl = 1.0 / sqrt(2.0 * l * (l + 1));
    const double ll = l * (l + 1.0);
    // outside, index -m: i(-m) pi
    const double mpi_o = -m * pi[l];
    const double2 zo[2] = {hk[l], jb[l]};
    const double2 zo1[2] = {hk[l - 1], jb[l - 1]};
    double2(*dst[2])[3] = {fout, freg};
    for (int kind = 0; kind < 2; ++kind) {
      const double2 z = zo[kind];
      const double2 dz = csub(zo1[kind], cscale(z, l / kr));
      // p = 0: c z (0, i(-m) pi, -tau)
      dst[kind][i][0] = make_double2(0.0, 0.0);
      dst[kind][i][1] = cscale(make_double2(-z.y, z.x), cl * mpi_o);
      dst[kind][i][2] = cscale(z, -cl * tau[l]);
      // p = 1: c (l(l+1) z/(kr) Pbar, dz tau, dz i(-m) pi)
      dst[kind][nl + i][0] = cscale(z, cl * ll * Pb[l] / kr);
      dst[kind][nl + i][1] = cscale(dz, cl * tau[l]);
      dst[kind][nl + i][2] = cscale(make_double2(-dz.y, dz.x), cl * mpi_o);
    }
    // inside, index m, complex argument
    const double mpi_i = m * pi[l];
    const double2 z = js[l];
    const double2 dz = csub(js[l - 1], cscale(cmul(z, izs), (double)l));
    fin[i][0] = make_double2(0.0, 0.0);
    fin[i][1] = cscale(make_double2(-z.y, z.x), cl * mpi_i);
    fin[i][2] = cscale(z, -cl * tau[l]);
    fin[nl + i][0] = cscale(cmul(z, izs), cl * ll * Pb[l]);
    fin[nl + i][1] = cscale(dz, cl * tau[l]);
    fin[nl + i][2] = cscale(make_double2(-dz.y, dz.x), cl * mpi_i);
  }
}

// (A x B) . n with n = n_r r^ + n_theta theta^
__device__ __forceinline__ double2 cross_dot_n(const double2* A, const double2* B, double nr, double nt) {
  const double2 cr = csub(cmul(A[1], B[2]), cmul(A[2], B[1]));
  const double2 ct = csub(cmul(A[2], B[0]), cmul(A[0], B[2]));
  return cadd(cscale(cr, nr), cscale(ct, nt));
}

template <int NMAX>
__global__ void __launch_bounds__(CYL_THREADS)
cylinder_tmatrix_kernel(const CylGeom* __restrict__ geo, double kb, int nq, const double* __restrict__ gx,
                        const double* __restrict__ gw, double2* __restrict__ T_out) {
  constexpr int L = NMAX * (NMAX + 2), P = 2 * L;
  const int cyl = blockIdx.x;
  const int m = (int)blockIdx.y - NMAX;
  const int am = m < 0 ? -m : m, lmin = am > 1 ? am : 1, nl = NMAX - lmin + 1, d = 2 * nl;
  const CylGeom g = geo[cyl];
  const double2 ks = cscale(g.m_rel, kb);
  const double2 ratio = g.m_rel;  // k_s / k_b
  __shared__ double2 s_in[CYL_CHUNK][CYL_D][3], s_out[CYL_CHUNK][CYL_D][3], s_reg[CYL_CHUNK][CYL_D][3];
  __shared__ double s_nr[CYL_CHUNK], s_nt[CYL_CHUNK], s_w[CYL_CHUNK];
  __shared__ double2 sP[CYL_D][CYL_D], sQ[CYL_D][CYL_D];
  const int e = threadIdx.x;
  const int row = e / d, col = e % d;  // nu = row (outside), mu = col (inside)
  const bool mine = e < d * d;
  double2 accP = make_double2(0.0, 0.0), accQ = make_double2(0.0, 0.0);
  const int npts = 3 * nq;
  for (int q0 = 0; q0 < npts; q0 += CYL_CHUNK) {
    if (e < CYL_CHUNK && q0 + e < npts) {
      const ProfilePoint pt = profile_point(g, q0 + e, nq, gx, gw);
      block_functions<NMAX>(pt, m, kb, ks, s_in[e], s_out[e], s_reg[e]);
      s_nr[e] = pt.nr;
      s_nt[e] = pt.nt;
      s_w[e] = pt.w;
    }
    __syncthreads();
    if (mine) {
      const int p = row / nl, li = row % nl;       // outside (l, p)
      const int pp = col / nl, lj = col % nl;      // inside (l', p')
      const int flip = (1 - p) * nl + li, same = row;
      const int mubar = (1 - pp) * nl + lj;
      const int nc = min(CYL_CHUNK, npts - q0);
      for (int c = 0; c < nc; ++c) {
        const double nr = s_nr[c], nt = s_nt[c], w = s_w[c];
        const double2 a1 = cross_dot_n(s_in[c][col], s_out[c][flip], nr, nt);
        const double2 a2 = cross_dot_n(s_in[c][mubar], s_out[c][same], nr, nt);
        const double2 b1 = cross_dot_n(s_in[c][col], s_reg[c][flip], nr, nt);
        const double2 b2 = cross_dot_n(s_in[c][mubar], s_reg[c][same], nr, nt);
        accP = cadd(accP, cscale(cadd(a1, cmul(ratio, a2)), w));
        accQ = cadd(accQ, cscale(cadd(b1, cmul(ratio, b2)), w));
      }
    }
    __syncthreads();
  }
  if (mine) {
    sP[row][col] = cscale(accP, 2.0 * M_PI);
    sQ[row][col] = cscale(accQ, 2.0 * M_PI);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // T P = -Q  <=>  P^T T^T = -Q^T: eliminate on A = P^T with the right-hand sides B = -Q^T
    double2 A[CYL_D][CYL_D], B[CYL_D][CYL_D];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        A[i][j] = sP[j][i];
        B[i][j] = make_double2(-sQ[j][i].x, -sQ[j][i].y);
      }
    for (int k = 0; k < d; ++k) {
      int piv = k;
      for (int i = k + 1; i < d; ++i)
        if (cd_abs2(A[i][k]) > cd_abs2(A[piv][k])) piv = i;
      if (piv != k)
        for (int j = 0; j < d; ++j) {
          double2 t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t;
          t = B[k][j]; B[k][j] = B[piv][j]; B[piv][j] = t;
        }
      const double2 inv = cd_div(make_double2(1.0, 0.0), A[k][k]);
      for (int i = k + 1; i < d; ++i) {
        const double2 f = cmul(A[i][k], inv);
        for (int j = k; j < d; ++j) A[i][j] = csub(A[i][j], cmul(f, A[k][j]));
        for (int j = 0; j < d; ++j) B[i][j] = csub(B[i][j], cmul(f, B[k][j]));
      }
    }
    for (int k = d - 1; k >= 0; --k)
      for (int j = 0; j < d; ++j) {
        double2 s = B[k][j];
        for (int i = k + 1; i < d; ++i) s = csub(s, cmul(A[k][i], B[i][j]));
        B[k][j] = cd_div(s, A[k][k]);
      }
    // B = T^T: T[nu][mu] = B[mu][nu]; scatter to the flat P x P block of this cylinder
    double2* Tc = T_out + (int64_t)cyl * P * P;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        const int li = lmin + i % nl, pi_ = i / nl, lj = lmin + j % nl, pj = j / nl;
        const int fi = pi_ * L + li * (li + 1) + m - 1, fj = pj * L + lj * (lj + 1) + m - 1;
        Tc[(int64_t)fi * P + fj] = B[j][i];
      }
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n, three-term recurrence)
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static int launch_cylinders(tmat_ctx* ctx, int nmax, const CylGeom* d_geo, int64_t n, double kb, int nq,
                            const double* gx, const double* gw, double2* T) {
  dim3 grid((unsigned)n, (unsigned)(2 * nmax + 1));
  switch (nmax) {
#define CY(NM) \
  case NM: cylinder_tmatrix_kernel<NM><<<grid, CYL_THREADS, 0, ctx->stream>>>(d_geo, kb, nq, gx, gw, T); break;
    CY(1) CY(2) CY(3) CY(4) CY(5) CY(6)
#undef CY
    default: return set_error(ctx, TMAT_EINVAL, "tmat_build_cylinder: nmax %d", nmax);
  }
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

// dT = (T(+) - T(-)) / (2 h)
__global__ void central_difference_kernel(const double2* __restrict__ Tp, const double2* __restrict__ Tm, double inv2h,
                                          int64_t n, double2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cscale(csub(Tp[i], Tm[i]), inv2h);
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_build_cylinder(tmat_ctx* ctx, const tmat_cylinder* cyl, int64_t n, double wavelength, double n_bg,
                                   int nmax, int n_quad, tmat_c128* T_out, tmat_c128* dTdr_out) {
  if (!ctx) return TMAT_EINVAL;
  if (n < 0 || nmax < 1 || nmax > TMAT_NMAX_MAX || !(wavelength > 0) || !(n_bg > 0) || n_quad < 0 || n_quad > 512 ||
      (n > 0 && (!cyl || !T_out)) || n > 65535)
    return set_error(ctx, TMAT_EINVAL, "tmat_build_cylinder: bad arguments (n <= 65535 cylinders per call)");
  if (n == 0) return TMAT_OK;
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  const int nq = n_quad > 0 ? n_quad : 48;
  const double kb = 2.0 * M_PI * n_bg / wavelength;
  Staged sc, sT, sd;
  TM_TRY(stage_in(ctx, "cy_in", cyl, sizeof(tmat_cylinder) * n, &sc));
  // host copy of the geometry for validation and the finite-difference variants
  std::vector<tmat_cylinder> h(n);
  TM_CUDA(ctx, cudaMemcpyAsync(h.data(), sc.dev, sizeof(tmat_cylinder) * n, cudaMemcpyDefault, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<CylGeom> geo(n);
  for (int64_t i = 0; i < n; ++i) {
    if (!(h[i].radius > 0) || !(h[i].height > 0) || !(h[i].n_re > 0) || !(h[i].n_im >= 0) || !std::isfinite(h[i].radius) ||
        !std::isfinite(h[i].height))
      return set_error(ctx, TMAT_EINVAL, "tmat_build_cylinder: cylinder %lld has a bad radius, height or index",
                       (long long)i);
    geo[i].radius = h[i].radius;
    geo[i].height = h[i].height;
    geo[i].m_rel = make_double2(h[i].n_re / n_bg, h[i].n_im / n_bg);
  }
  TM_TRY(stage_out(ctx, "cy_T", T_out, sizeof(double2) * n * P * P, &sT));
  TM_TRY(stage_out(ctx, "cy_dT", dTdr_out, sizeof(double2) * n * P * P, &sd));
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  double *d_gx, *d_gw;
  CylGeom* d_geo;
  TM_TRY(scratch(ctx, "cy_gx", sizeof(double) * nq, (void**)&d_gx));
  TM_TRY(scratch(ctx, "cy_gw", sizeof(double) * nq, (void**)&d_gw));
  TM_TRY(scratch(ctx, "cy_geo", sizeof(CylGeom) * n * 3, (void**)&d_geo));
  TM_CUDA(ctx, cudaMemcpyAsync(d_gx, gx.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, ctx->stream));
  TM_CUDA(ctx, cudaMemcpyAsync(d_gw, gw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, ctx->stream));
  // geometry sets: as given, and radius +- h for the radius derivative (central difference)
  const double hstep = 1e-5 * wavelength / n_bg;
  std::vector<CylGeom> all(geo);
  if (dTdr_out) {
    for (int64_t i = 0; i < n; ++i) all.push_back({geo[i].radius + hstep, geo[i].height, geo[i].m_rel});
    for (int64_t i = 0; i < n; ++i) all.push_back({geo[i].radius - hstep, geo[i].height, geo[i].m_rel});
  }
  TM_CUDA(ctx, cudaMemcpyAsync(d_geo, all.data(), sizeof(CylGeom) * all.size(), cudaMemcpyHostToDevice, ctx->stream));
  TM_CUDA(ctx, cudaMemsetAsync(sT.dev, 0, sizeof(double2) * n * P * P, ctx->stream));
  TM_TRY(launch_cylinders(ctx, nmax, d_geo, n, kb, nq, d_gx, d_gw, (double2*)sT.dev));
  if (dTdr_out) {
    double2* tpm;
    TM_TRY(scratch(ctx, "cy_Tpm", sizeof(double2) * 2 * n * P * P, (void**)&tpm));
    TM_CUDA(ctx, cudaMemsetAsync(tpm, 0, sizeof(double2) * 2 * n * P * P, ctx->stream));
    TM_TRY(launch_cylinders(ctx, nmax, d_geo + n, n, kb, nq, d_gx, d_gw, tpm));
    TM_TRY(launch_cylinders(ctx, nmax, d_geo + 2 * n, n, kb, nq, d_gx, d_gw, tpm + n * P * P));
    central_difference_kernel<<<(unsigned)std::min<int64_t>(cdiv(n * P * P, 256), 4096), 256, 0, ctx->stream>>>(
        tpm, tpm + n * P * P, 0.5 / hstep, n * P * P, (double2*)sd.dev);
    TM_LAUNCHED(ctx);
  }
  TM_TRY(finish_out(ctx, &sT));
  TM_TRY(finish_out(ctx, &sd));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
