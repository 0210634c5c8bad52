// Field evaluation (App. I-C, Eq. sca_fld_concise), the far-field amplitude and
// the point figure of merit with its adjoint source (App. IV).
//
//  Phi_{lm0} = c_l z_l(kr) [ i m pi th^ - tau ph^ ] e^{i m ph}
//  Phi_{lm1} = c_l [ l(l+1) z_l/(kr) Pbar r^ + ((kr z_l)'/(kr)) (tau th^ + i m pi ph^) ] e^{i m ph}
//  c_l = 1/sqrt(2 l (l+1)), (kr z_l)'/(kr) = z_{l-1} - l z_l/(kr), z = h^(1).
// Far field: h_l(z) -> (-i)^{l+1} e^{iz}/z, so F_{lm0} = c_l (-i)^{l+1}[..], F_{lm1} = c_l (-i)^l (tau th^ + i m pi ph^) e^{imph}.
#include <cmath>
#include <mutex>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

constexpr int NM1 = TMAT_NMAX_MAX + 1;

// Constants of the normalised Legendre recurrences (Doicu's normalisation, no
// Condon-Shortley phase), l, m <= TMAT_NMAX_MAX, uploaded once per device:
//   Pbar_m^m = base_m s^m, pi_m^m = base_m s^(m-1), base_m = sqrt((2m+1)/(2 (2m)!)) (2m-1)!!
//   Pbar_l^m = a_lm (c Pbar_{l-1}^m - b_lm Pbar_{l-2}^m) (the same for pi),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
//   tau_l^0 = -sqrt(l(l+1)) Pbar_l^1, tau_l^m = l c pi_l^m - t_lm pi_{l-1}^m,
//   t_lm = sqrt((2l+1)(l^2-m^2)/(2l-1)); c_l = 1/sqrt(2l(l+1)).
struct LegConst {
  double a[NM1][NM1], b[NM1][NM1], t[NM1][NM1], base[NM1], sq[NM1], cl[NM1];
};
__constant__ LegConst c_leg;
// the same constants in fp32 (the mixed-precision near field)
struct LegConstF {
  float a[NM1][NM1], b[NM1][NM1], t[NM1][NM1], base[NM1], sq[NM1], cl[NM1];
};
__constant__ LegConstF c_legf;

// once per device (on `stream`); 0 or a CUDA error code
static cudaError_t leg_upload(int device, cudaStream_t stream) {
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> lock(mu);
  if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
  LegConst h = {};
  for (int m = 0; m < NM1; ++m) {
    double df = 1.0, f2 = 1.0;
    for (int t = 1; t < 2 * m; t += 2) df *= t;
    for (int t = 2; t <= 2 * m; ++t) f2 *= t;
    h.base[m] = std::sqrt((2 * m + 1) / (2.0 * f2)) * df;
  }
  for (int l = 0; l < NM1; ++l) {
    h.sq[l] = std::sqrt(l * (l + 1.0));
    h.cl[l] = l > 0 ? 1.0 / std::sqrt(2.0 * l * (l + 1)) : 0.0;
    for (int m = 0; m < NM1; ++m) {
      if (l > m) {
        h.a[l][m] = std::sqrt((4.0 * l * l - 1) / ((double)l * l - (double)m * m));
        h.b[l][m] = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1));
      }
      if (l >= 1 && m <= l) h.t[l][m] = std::sqrt((2.0 * l + 1) * ((double)l * l - (double)m * m) / (2.0 * l - 1));
    }
  }
  LegConstF hf;
  for (int i = 0; i < NM1; ++i) {
    hf.base[i] = (float)h.base[i];
    hf.sq[i] = (float)h.sq[i];
    hf.cl[i] = (float)h.cl[i];
    for (int j = 0; j < NM1; ++j) {
      hf.a[i][j] = (float)h.a[i][j];
      hf.b[i][j] = (float)h.b[i][j];
      hf.t[i][j] = (float)h.t[i][j];
    }
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_leg, &h, sizeof(h), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_legf, &hf, sizeof(hf), 0, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
  return e;
}

static int upload_legendre(tmat_ctx* ctx) {
  TM_CUDA(ctx, leg_upload(ctx->device, ctx->stream));
  return TMAT_OK;
}

// Calls f(flat, vec[3]) for every VSWF Phi_f(k d) (outgoing), far=false, or the
// far-field amplitude F_f(d^), far=true (|d| ignored). Compile-time nmax; the waves are
// produced m-major (the flat index carries the order), so only one Legendre recurrence
// (over l, for the current m) is live at a time; e^{i m phi} by powers of e^{i phi}.
template <int NMAX, typename Fn>
__device__ __forceinline__ void waves_t(double k, double dx, double dy, double dz, bool far, Fn&& f) {
  constexpr int L = NMAX * (NMAX + 2);
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  const double ct = dz / r, st = sqrt(fmax(0.0, 1.0 - ct * ct));
  const double rho = sqrt(dx * dx + dy * dy);
  const double cp = rho > 0 ? dx / rho : 1.0, sp = rho > 0 ? dy / rho : 0.0;
  // radial factors c_l z_l, c_l l(l+1) z_l/(kr), c_l (z_{l-1} - l z_l/(kr)) (far: phases)
  double2 zM[NMAX + 1], zNr[NMAX + 1], zNt[NMAX + 1];
  {
    const double kr = k * r;
    double2 h[NMAX + 1];
    if (!far) {
      double sn, cs;
      sincos(kr, &sn, &cs);
      const double ix = 1.0 / kr;
      h[0] = make_double2(sn * ix, -cs * ix);
      h[1] = make_double2(-ix * cs + ix * ix * sn, -ix * sn - ix * ix * cs);
#pragma unroll
      for (int q = 1; q < NMAX; ++q) {
        const double fq = (2 * q + 1) * ix;
        h[q + 1] = make_double2(fq * h[q].x - h[q - 1].x, fq * h[q].y - h[q - 1].y);
      }
    }
#pragma unroll
    for (int l = 1; l <= NMAX; ++l) {
      const double cl = c_leg.cl[l];
      if (far) {
        const int e = (3 * (l + 1)) & 3;  // (-i)^{l+1} = i^{3(l+1)}
        zM[l] = make_double2(e == 0 ? cl : (e == 2 ? -cl : 0.0), e == 1 ? cl : (e == 3 ? -cl : 0.0));
        const int e2 = (3 * l) & 3;
        zNt[l] = make_double2(e2 == 0 ? cl : (e2 == 2 ? -cl : 0.0), e2 == 1 ? cl : (e2 == 3 ? -cl : 0.0));
        zNr[l] = make_double2(0, 0);
      } else {
        zM[l] = cscale(h[l], cl);
        zNr[l] = cscale(h[l], cl * l * (l + 1.0) / kr);
        zNt[l] = make_double2(cl * (h[l - 1].x - l * h[l].x / kr), cl * (h[l - 1].y - l * h[l].y / kr));
      }
    }
  }
  const double thv[3] = {ct * cp, ct * sp, -st}, phv[3] = {-sp, cp, 0.0}, rhv[3] = {st * cp, st * sp, ct};
  // Pbar_l^1 for tau_l^0 = -sqrt(l(l+1)) Pbar_l^1
  double P1[NMAX + 1];
  {
    double pp = 0.0, pc = c_leg.base[1] * st;
    P1[1] = pc;
#pragma unroll
    for (int l = 2; l <= NMAX; ++l) {
      const double pn = c_leg.a[l][1] * (ct * pc - c_leg.b[l][1] * pp);
      pp = pc;
      pc = pn;
      P1[l] = pn;
    }
  }
  double2 em = make_double2(1.0, 0.0);
  double pw = 1.0, pw1 = 1.0;  // st^m and st^(m-1)
#pragma unroll
  for (int m = 0; m <= NMAX; ++m) {
    const double base = c_leg.base[m];
    double p_prev = 0.0, p_cur = base * pw;                    // Pbar_m^m
    double q_prev = 0.0, q_cur = m >= 1 ? base * pw1 : 0.0;    // pi_m^m
#pragma unroll
    for (int l = (m > 1 ? m : 1); l <= NMAX; ++l) {
      if (l > m) {
        const double a = c_leg.a[l][m], bb = c_leg.b[l][m];
        const double pn = a * (ct * p_cur - bb * p_prev), qn = a * (ct * q_cur - bb * q_prev);
        p_prev = p_cur;
        p_cur = pn;
        q_prev = q_cur;
        q_cur = qn;
      }
      // now p_cur = Pbar_l^m, q_cur = pi_l^m, q_prev = pi_{l-1}^m (0 when l == m)
      const double pb = p_cur;
      const double ta = m == 0 ? -c_leg.sq[l] * P1[l] : l * ct * q_cur - c_leg.t[l][m] * (l > m ? q_prev : 0.0);
#pragma unroll
      for (int sg = 0; sg < (m == 0 ? 1 : 2); ++sg) {
        const int mm = sg == 0 ? m : -m;
        const double mpi = mm * q_cur;
        const double2 e = sg == 0 ? em : cconj(em);
        // M: c z [ i mpi th - ta ph ] e ; N: c [ zNr pb r + zNt (ta th + i mpi ph) ] e
        const double2 aM = cmul(zM[l], e), aNr = cmul(cscale(zNr[l], pb), e), aNt = cmul(zNt[l], e);
        double2 vM[3], vN[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double2 gM = make_double2(-ta * phv[c], mpi * thv[c]);
          const double2 gN = make_double2(ta * thv[c], mpi * phv[c]);
          vM[c] = cmul(aM, gM);
          vN[c] = cadd(cscale(aNr, rhv[c]), cmul(aNt, gN));
        }
        const int n = l * (l + 1) + mm - 1;
        f(n, vM);
        f(L + n, vN);
      }
    }
    pw1 = pw;
    pw *= st;
    em = cmul(em, make_double2(cp, sp));
  }
}

// Mixed-precision near field: the outgoing waves Phi_f(k d) with the distance, k|d| and its
// reduction modulo 2 pi in fp64 (so the phase of a wave hundreds of wavelengths away keeps
// ~1e-7 accuracy), everything else (sin/cos of the reduced phase, the Hankel recurrence, the
// Legendre recurrences, the vector components) in fp32. Same formulas as waves_t.
template <int NMAX, typename Fn>
__device__ __forceinline__ void waves32_near(double k, double dx, double dy, double dz, Fn&& f) {
  constexpr int L = NMAX * (NMAX + 2);
  const double r2 = dx * dx + dy * dy + dz * dz;
  // 1/sqrt(r2): fp32 estimate, one Newton step in fp64 (relative error ~1e-14)
  double y = (double)rsqrtf((float)r2);
  y = y * (1.5 - 0.5 * r2 * y * y);
  const double r = r2 * y;
  const double kr = k * r;
  const double twopi = 6.283185307179586476925286766559;
  const float ang = (float)(kr - twopi * rint(kr * (1.0 / twopi)));
  const float fy = (float)y;
  const float fdx = (float)dx, fdy = (float)dy;
  const float rho = sqrtf(fdx * fdx + fdy * fdy);
  // sin(theta) from the transverse distance, not sqrt(1 - cos^2) (which loses every digit
  // in fp32 for points nearly straight above a scatterer)
  const float ct = (float)dz * fy, st = rho * fy;
  const float cp = rho > 0.f ? fdx / rho : 1.f, sp = rho > 0.f ? fdy / rho : 0.f;
  float2 zM[NMAX + 1], zNr[NMAX + 1], zNt[NMAX + 1];
  {
    float sn, cs;
    sincosf(ang, &sn, &cs);
    const float ix = (float)(1.0 / kr);
    float2 h[NMAX + 1];
    h[0] = make_float2(sn * ix, -cs * ix);
    h[1] = make_float2(-ix * cs + ix * ix * sn, -ix * sn - ix * ix * cs);
#pragma unroll
    for (int q = 1; q < NMAX; ++q) {
      const float fq = (2 * q + 1) * ix;
      h[q + 1] = make_float2(fq * h[q].x - h[q - 1].x, fq * h[q].y - h[q - 1].y);
    }
#pragma unroll
    for (int l = 1; l <= NMAX; ++l) {
      const float cl = c_legf.cl[l];
      zM[l] = cscale(h[l], cl);
      zNr[l] = cscale(h[l], cl * l * (l + 1.f) * ix);
      zNt[l] = make_float2(cl * (h[l - 1].x - l * h[l].x * ix), cl * (h[l - 1].y - l * h[l].y * ix));
    }
  }
  const float thv[3] = {ct * cp, ct * sp, -st}, phv[3] = {-sp, cp, 0.f}, rhv[3] = {st * cp, st * sp, ct};
  float P1[NMAX + 1];
  {
    float pp = 0.f, pc = c_legf.base[1] * st;
    P1[1] = pc;
#pragma unroll
    for (int l = 2; l <= NMAX; ++l) {
      const float pn = c_legf.a[l][1] * (ct * pc - c_legf.b[l][1] * pp);
      pp = pc;
      pc = pn;
      P1[l] = pn;
    }
  }
  float2 em = make_float2(1.f, 0.f);
  float pw = 1.f, pw1 = 1.f;
#pragma unroll
  for (int m = 0; m <= NMAX; ++m) {
    const float base = c_legf.base[m];
    float p_prev = 0.f, p_cur = base * pw;
    float q_prev = 0.f, q_cur = m >= 1 ? base * pw1 : 0.f;
#pragma unroll
    for (int l = (m > 1 ? m : 1); l <= NMAX; ++l) {
      if (l > m) {
        const float a = c_legf.a[l][m], bb = c_legf.b[l][m];
        const float pn = a * (ct * p_cur - bb * p_prev), qn = a * (ct * q_cur - bb * q_prev);
        p_prev = p_cur;
        p_cur = pn;
        q_prev = q_cur;
        q_cur = qn;
      }
      const float pb = p_cur;
      const float ta = m == 0 ? -c_legf.sq[l] * P1[l] : l * ct * q_cur - c_legf.t[l][m] * (l > m ? q_prev : 0.f);
#pragma unroll
      for (int sg = 0; sg < (m == 0 ? 1 : 2); ++sg) {
        const int mm = sg == 0 ? m : -m;
        const float mpi = mm * q_cur;
        const float2 e = sg == 0 ? em : cconj(em);
        const float2 aM = cmul(zM[l], e), aNr = cmul(cscale(zNr[l], pb), e), aNt = cmul(zNt[l], e);
        float2 vM[3], vN[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 gM = make_float2(-ta * phv[c], mpi * thv[c]);
          const float2 gN = make_float2(ta * thv[c], mpi * phv[c]);
          vM[c] = cmul(aM, gM);
          vN[c] = cadd(cscale(aNr, rhv[c]), cmul(aNt, gN));
        }
        const int n = l * (l + 1) + mm - 1;
        f(n, vM);
        f(L + n, vN);
      }
    }
    pw1 = pw;
    pw *= st;
    em = cmul(em, make_float2(cp, sp));
  }
}

// mixed-precision partial near field over a chunk of scatterers (coefficients s32 in
// complex64): fp32 products per scatterer, fp64 sums across scatterers and threads
template <int NMAX>
__global__ void __launch_bounds__(128)
field32_kernel(const double* __restrict__ pos, int64_t N, double k, const float2* __restrict__ s32,
               const double* __restrict__ pts, double2* __restrict__ part) {
  constexpr int P = 2 * NMAX * (NMAX + 2);
  const int64_t a = blockIdx.x;
  __shared__ double2 red[3][128];
  double2 E[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  const double px = pts[3 * a], py = pts[3 * a + 1], pz = pts[3 * a + 2];
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.y * blockDim.x) {
    const float2* si = s32 + i * P;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
    waves32_near<NMAX>(k, px - pos[3 * i], py - pos[3 * i + 1], pz - pos[3 * i + 2], [&](int fidx, const float2* v) {
      const float2 c = si[fidx];
      acc0 = cadd(acc0, cmul(c, v[0]));
      acc1 = cadd(acc1, cmul(c, v[1]));
      acc2 = cadd(acc2, cmul(c, v[2]));
    });
    E[0] = cadd(E[0], to_c128(acc0));
    E[1] = cadd(E[1], to_c128(acc1));
    E[2] = cadd(E[2], to_c128(acc2));
  }
  for (int q = 0; q < 3; ++q) red[q][threadIdx.x] = E[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    double2 t = make_double2(0, 0);
    for (int b = 0; b < blockDim.x; ++b) t = cadd(t, red[threadIdx.x][b]);
    part[(a * gridDim.y + blockIdx.y) * 3 + threadIdx.x] = t;
  }
}

__global__ void to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = to_c64(in[i]);
}

// partial E over a chunk of scatterers: grid (M, chunks); block reduce
template <int NMAX, bool FAR>
__global__ void __launch_bounds__(128)
field_kernel(const double* __restrict__ pos, int64_t N, double k, const double2* __restrict__ s,
             const double* __restrict__ pts, int64_t M, double2* __restrict__ part) {
  constexpr int P = 2 * NMAX * (NMAX + 2);
  const int64_t a = blockIdx.x;
  __shared__ double2 red[3][128];
  double2 E[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  double ux = 0, uy = 0, uz = 0, px = 0, py = 0, pz = 0;
  if (FAR) {  // direction (theta, phi)
    double s_, c_, sp_, cp_;
    sincos(pts[2 * a], &s_, &c_);
    sincos(pts[2 * a + 1], &sp_, &cp_);
    ux = s_ * cp_;
    uy = s_ * sp_;
    uz = c_;
  } else {
    px = pts[3 * a];
    py = pts[3 * a + 1];
    pz = pts[3 * a + 2];
  }
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.y * blockDim.x) {
    const double2* si = s + i * P;
    double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0), acc2 = make_double2(0, 0);
    auto fn = [&](int f, const double2* v) {
      const double2 c = si[f];
      acc0 = cadd(acc0, cmul(c, v[0]));
      acc1 = cadd(acc1, cmul(c, v[1]));
      acc2 = cadd(acc2, cmul(c, v[2]));
    };
    if (FAR) {
      waves_t<NMAX>(k, ux, uy, uz, true, fn);
      const double ph = -k * (ux * pos[3 * i] + uy * pos[3 * i + 1] + uz * pos[3 * i + 2]);
      double sn, cs;
      sincos(ph, &sn, &cs);
      const double2 e = make_double2(cs, sn);
      E[0] = cadd(E[0], cmul(e, acc0));
      E[1] = cadd(E[1], cmul(e, acc1));
      E[2] = cadd(E[2], cmul(e, acc2));
    } else {
      waves_t<NMAX>(k, px - pos[3 * i], py - pos[3 * i + 1], pz - pos[3 * i + 2], false, fn);
      E[0] = cadd(E[0], acc0);
      E[1] = cadd(E[1], acc1);
      E[2] = cadd(E[2], acc2);
    }
  }
  for (int q = 0; q < 3; ++q) red[q][threadIdx.x] = E[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    double2 t = make_double2(0, 0);
    for (int b = 0; b < blockDim.x; ++b) t = cadd(t, red[threadIdx.x][b]);
    part[(a * gridDim.y + blockIdx.y) * 3 + threadIdx.x] = t;
  }
}

template <int NMAX>
static void launch_field(dim3 grid, cudaStream_t st, const double* pos, int64_t N, double k, const double2* s,
                         const double* pts, int64_t M, bool far, double2* part) {
  if (far)
    field_kernel<NMAX, true><<<grid, 128, 0, st>>>(pos, N, k, s, pts, M, part);
  else
    field_kernel<NMAX, false><<<grid, 128, 0, st>>>(pos, N, k, s, pts, M, part);
}

static void launch_field_n(int nmax, dim3 grid, cudaStream_t st, const double* pos, int64_t N, double k,
                           const double2* s, const double* pts, int64_t M, bool far, double2* part) {
  switch (nmax) {
    case 1: launch_field<1>(grid, st, pos, N, k, s, pts, M, far, part); break;
    case 2: launch_field<2>(grid, st, pos, N, k, s, pts, M, far, part); break;
    case 3: launch_field<3>(grid, st, pos, N, k, s, pts, M, far, part); break;
    case 4: launch_field<4>(grid, st, pos, N, k, s, pts, M, far, part); break;
    case 5: launch_field<5>(grid, st, pos, N, k, s, pts, M, far, part); break;
    case 6: launch_field<6>(grid, st, pos, N, k, s, pts, M, far, part); break;
  }
}

__global__ void field_reduce_kernel(const double2* __restrict__ part, int64_t M, int nchunk, double2* __restrict__ E) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * 3) return;
  int64_t a = t / 3;
  int q = (int)(t % 3);
  double2 s = make_double2(0, 0);
  for (int c = 0; c < nchunk; ++c) s = cadd(s, part[(a * nchunk + c) * 3 + q]);
  E[t] = s;
}

// v[i][f] = sum_c conj(E_c) Phi_{f,c}(k(x_f - x_i))
template <int NMAX>
__global__ void adjoint_source_kernel(const double* __restrict__ pos, int64_t N, double k, int nmax,
                                      const double* __restrict__ xf, const double2* __restrict__ Etot,
                                      double2* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int P = num_coeffs(nmax);
  double2 ce[3] = {cconj(Etot[0]), cconj(Etot[1]), cconj(Etot[2])};
  waves_t<NMAX>(k, xf[0] - pos[3 * i], xf[1] - pos[3 * i + 1], xf[2] - pos[3 * i + 2], false,
                [&](int f, const double2* w) {
                  double2 acc = make_double2(0, 0);
                  for (int q = 0; q < 3; ++q) acc = cadd(acc, cmul(ce[q], w[q]));
                  v[i * P + f] = acc;
                });
}

__global__ void add3_kernel(double2* __restrict__ E, const double2* __restrict__ Einc) {
  int q = threadIdx.x;
  if (q < 3) E[q] = cadd(E[q], Einc[q]);
}

int field_dev(tmat_ctx* ctx, const double* pos, int64_t N, double k, int nmax, const double2* s, const double* pts,
              int64_t M, bool far, double2* E) {
  TM_TRY(upload_legendre(ctx));
  if (M == 0) return TMAT_OK;
  int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(N, 128), std::max<int64_t>(1, 16 * ctx->num_sms / std::max<int64_t>(M, 1))));
  if (nchunk > 65535) nchunk = 65535;
  double2* part;
  TM_TRY(scratch(ctx, "fld_part", sizeof(double2) * M * nchunk * 3, (void**)&part));
  cudaEvent_t ev = timing_begin(ctx);
  if (!far && ctx->field_mixed) {
    const int P = num_coeffs(nmax);
    float2* s32;
    TM_TRY(scratch(ctx, "fld_s32", sizeof(float2) * N * P, (void**)&s32));
    to_c64_kernel<<<(unsigned)std::min<int64_t>(cdiv(N * P, 256), 4096), 256, 0, ctx->stream>>>(s, s32, N * P);
    TM_LAUNCHED(ctx);
    const dim3 g((unsigned)M, nchunk);
    switch (nmax) {
#define F32(NM) \
  case NM: field32_kernel<NM><<<g, 128, 0, ctx->stream>>>(pos, N, k, s32, pts, part); break;
      F32(1) F32(2) F32(3) F32(4) F32(5) F32(6)
#undef F32
    }
  } else {
    launch_field_n(nmax, dim3((unsigned)M, nchunk), ctx->stream, pos, N, k, s, pts, M, far, part);
  }
  TM_LAUNCHED(ctx);
  timing_end(ctx, far ? "farfield" : (ctx->field_mixed ? "field32" : "field64"), ev);
  field_reduce_kernel<<<(unsigned)cdiv(M * 3, 128), 128, 0, ctx->stream>>>(part, M, nchunk, E);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

// v[i][f] = sum_c conj(E_c) Phi_{f,c}(k(x_f - x_i)) for a device focal point and field
int adjoint_source_dev(tmat_ctx* ctx, const double* pos, int64_t N, double k, int nmax, const double* xf,
                       const double2* E, double2* v) {
  TM_TRY(upload_legendre(ctx));
  if (N == 0) return TMAT_OK;
  switch (nmax) {
#define AK(NM) \
  case NM: adjoint_source_kernel<NM><<<(unsigned)cdiv(N, 64), 64, 0, ctx->stream>>>(pos, N, k, nmax, xf, E, v); break;
    AK(1) AK(2) AK(3) AK(4) AK(5) AK(6)
#undef AK
    default: return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  }
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

}  // namespace tmat

using namespace tmat;

static int field_entry(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                       const tmat_c128* s, const double* pts, int64_t M, tmat_c128* out, bool far) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || M < 0 || !(wavelength > 0) || !(n_bg > 0) || (M > 0 && (!pts || !out)) || (N > 0 && (!pos || !s)))
    return set_error(ctx, TMAT_EINVAL, "tmat_field: bad arguments");
  if (M > 2147483647LL) return set_error(ctx, TMAT_EINVAL, "tmat_field: too many points");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  Staged sp, ss, st, so;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  TM_TRY(stage_in(ctx, "st_s", s, sizeof(double2) * N * P, &ss));
  TM_TRY(stage_in(ctx, "st_pts", pts, sizeof(double) * (far ? 2 : 3) * M, &st));
  TM_TRY(stage_out(ctx, "st_E", out, sizeof(double2) * 3 * M, &so));
  double k = 2.0 * M_PI * n_bg / wavelength;
  TM_TRY(field_dev(ctx, (const double*)sp.dev, N, k, nmax, (const double2*)ss.dev, (const double*)st.dev, M, far,
                   (double2*)so.dev));
  TM_TRY(finish_out(ctx, &so));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}

extern "C" int tmat_field(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                          const tmat_c128* s, const double* pts, int64_t M, tmat_c128* E_out) {
  return field_entry(ctx, pos, N, wavelength, n_bg, nmax, s, pts, M, E_out, false);
}

extern "C" int tmat_farfield(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                             const tmat_c128* s, const double* dirs, int64_t M, tmat_c128* F_out) {
  return field_entry(ctx, pos, N, wavelength, n_bg, nmax, s, dirs, M, F_out, true);
}

extern "C" int tmat_point_fom(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                              const tmat_c128* s, const double* x_f, const tmat_c128* E_inc_f, double* fom_out,
                              tmat_c128* v_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || !x_f || !E_inc_f || !fom_out || (N > 0 && (!pos || !s)) || !(wavelength > 0) || !(n_bg > 0))
    return set_error(ctx, TMAT_EINVAL, "tmat_point_fom: bad arguments");
  if (nmax < 1 || nmax > TMAT_NMAX_MAX) return set_error(ctx, TMAT_EINVAL, "nmax %d outside 1..%d", nmax, TMAT_NMAX_MAX);
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int P = num_coeffs(nmax);
  Staged sp, ss, sx, se, sv;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  TM_TRY(stage_in(ctx, "st_s", s, sizeof(double2) * N * P, &ss));
  TM_TRY(stage_in(ctx, "st_xf", x_f, sizeof(double) * 3, &sx));
  TM_TRY(stage_in(ctx, "st_einc", E_inc_f, sizeof(double2) * 3, &se));
  TM_TRY(stage_out(ctx, "st_v", v_out, sizeof(double2) * N * P, &sv));
  double k = 2.0 * M_PI * n_bg / wavelength;
  double2* E;
  TM_TRY(scratch(ctx, "fom_E", sizeof(double2) * 3, (void**)&E));
  TM_TRY(field_dev(ctx, (const double*)sp.dev, N, k, nmax, (const double2*)ss.dev, (const double*)sx.dev, 1, false, E));
  add3_kernel<<<1, 32, 0, ctx->stream>>>(E, (const double2*)se.dev);
  TM_LAUNCHED(ctx);
  if (v_out && N > 0) {
    switch (nmax) {
#define AK(NM) case NM: adjoint_source_kernel<NM><<<(unsigned)cdiv(N, 64), 64, 0, ctx->stream>>>((const double*)sp.dev, N, k, nmax, (const double*)sx.dev, E, (double2*)sv.dev); break;
      AK(1) AK(2) AK(3) AK(4) AK(5) AK(6)
#undef AK
    }
    TM_LAUNCHED(ctx);
  }
  double2* pin = (double2*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, E, sizeof(double2) * 3, cudaMemcpyDeviceToHost, ctx->stream));
  TM_TRY(finish_out(ctx, &sv));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double f = 0;
  for (int q = 0; q < 3; ++q) f += pin[q].x * pin[q].x + pin[q].y * pin[q].y;
  *fom_out = f;
  return TMAT_OK;
}

// ---- allocation-free variant ------------------------------------------------------
// The partial sums of field_kernel live in this fixed array instead of context
// scratch. Host code must not pass `g_field_noalloc_part` itself to a kernel
// (on the host it names a stand-in, not the device memory): the device address
// is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

static __device__ __align__(256) double2 g_field_noalloc_part[TMAT_NOALLOC_FIELD_SLOTS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double2* g_noalloc_addr[kMaxDevices] = {nullptr};

// True when p is device memory of device `dev`, or managed memory. A pointer into another
// GPU's memory is refused: this entry point enables no peer access.
bool device_ptr_on(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // the error of this query only (no launch is pending: checked on entry)
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// device address of the scratch array on the current device (one-time set-up)
int noalloc_scratch(int dev, double2** out) {
  if (dev < 0 || dev >= kMaxDevices) return TMAT_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_field_noalloc_part);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return TMAT_ECUDA;
    }
    g_noalloc_addr[dev] = (double2*)p;
  }
  *out = g_noalloc_addr[dev];
  return TMAT_OK;
}
}  // namespace

extern "C" int tmat_field_noalloc(void* cuda_stream, const double* pos, int64_t N, double wavelength, double n_bg,
                                  int nmax, const tmat_c128* s, const double* pts, int64_t M, tmat_c128* E_out) {
  if (N < 0 || M < 0 || M > TMAT_NOALLOC_FIELD_SLOTS / 3 || nmax < 1 || nmax > TMAT_NMAX_MAX ||
      !(wavelength > 0) || !(n_bg > 0))
    return TMAT_EINVAL;
  if (M == 0) return TMAT_OK;
  // an error left pending by earlier work of the caller is reported, not consumed
  if (cudaPeekAtLastError() != cudaSuccess) return TMAT_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TMAT_ECUDA;
  }
  if (!device_ptr_on(pts, dev) || !device_ptr_on(E_out, dev) ||
      (N > 0 && (!device_ptr_on(pos, dev) || !device_ptr_on(s, dev))))
    return TMAT_EINVAL;
  double2* part = nullptr;
  int rc = noalloc_scratch(dev, &part);
  if (rc != TMAT_OK) return rc;
  if (leg_upload(dev, (cudaStream_t)cuda_stream) != cudaSuccess) {
    cudaGetLastError();
    return TMAT_ECUDA;
  }
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t nchunk = std::min<int64_t>(cdiv(N, 128), std::max<int64_t>(1, 4 * sms / M));
  nchunk = std::min<int64_t>(nchunk, TMAT_NOALLOC_FIELD_SLOTS / (3 * M));
  nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, 65535));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double k = 2.0 * M_PI * n_bg / wavelength;
  launch_field_n(nmax, dim3((unsigned)M, (unsigned)nchunk), st, pos, N, k, (const double2*)s, pts, M, false, part);
  if (cudaGetLastError() != cudaSuccess) return TMAT_ECUDA;
  field_reduce_kernel<<<(unsigned)cdiv(M * 3, 128), 128, 0, st>>>(part, M, (int)nchunk, (double2*)E_out);
  if (cudaGetLastError() != cudaSuccess) return TMAT_ECUDA;
  return TMAT_OK;
}
