// Field evaluation (App. I-C, Eq. sca_fld_concise), the far-field amplitude and
// the point figure of merit with its adjoint source (App. IV).
//
//  Phi_{lm0} = c_l z_l(kr) [ i m pi th^ - tau ph^ ] e^{i m ph}
//  Phi_{lm1} = c_l [ l(l+1) z_l/(kr) Pbar r^ + ((kr z_l)'/(kr)) (tau th^ + i m pi ph^) ] e^{i m ph}
//  c_l = 1/sqrt(2 l (l+1)), (kr z_l)'/(kr) = z_{l-1} - l z_l/(kr), z = h^(1).
// Far field: h_l(z) -> (-i)^{l+1} e^{iz}/z, so F_{lm0} = c_l (-i)^{l+1}[..], F_{lm1} = c_l (-i)^l (tau th^ + i m pi ph^) e^{imph}.
#include <cmath>

#include "dev.cuh"
#include "internal.h"

namespace tmat {

constexpr int NM1 = TMAT_NMAX_MAX + 1;

// normalised Legendre tables at cos(theta): P[l][m], pi[l][m] = P/sin, tau[l][m]
__device__ void legendre_tables(int nmax, double ct, double st, double (*P)[NM1], double (*pi)[NM1], double (*tau)[NM1]) {
  for (int l = 0; l <= nmax; ++l)
    for (int m = 0; m <= nmax; ++m) P[l][m] = pi[l][m] = tau[l][m] = 0.0;
  for (int m = 0; m <= nmax; ++m) {
    double df = 1.0, f2 = 1.0;
    for (int t = 1; t < 2 * m; t += 2) df *= t;
    for (int t = 2; t <= 2 * m; ++t) f2 *= t;
    double base = sqrt((2 * m + 1) / (2.0 * f2)) * df;  // Pbar_m^m = base s^m; pi_m^m = base s^(m-1)
    double q_prev = 0.0, q_cur = (m >= 1) ? base * pow(st, (double)(m - 1)) : 0.0;
    double p_prev = 0.0, p_cur = base * pow(st, (double)m);
    P[m][m] = p_cur;
    pi[m][m] = q_cur;
    for (int l = m + 1; l <= nmax; ++l) {
      double a = sqrt((4.0 * l * l - 1) / ((double)l * l - (double)m * m));
      double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1));
      double pn = a * (ct * p_cur - b * p_prev);
      double qn = a * (ct * q_cur - b * q_prev);
      p_prev = p_cur;
      p_cur = pn;
      q_prev = q_cur;
      q_cur = qn;
      P[l][m] = pn;
      pi[l][m] = qn;
    }
  }
  for (int l = 1; l <= nmax; ++l) {
    tau[l][0] = -sqrt(l * (l + 1.0)) * P[l][1 <= nmax ? 1 : 0];
    for (int m = 1; m <= l; ++m) {
      double prev = (l - 1 >= m) ? pi[l - 1][m] : 0.0;
      tau[l][m] = l * ct * pi[l][m] - sqrt((2.0 * l + 1) * ((double)l * l - (double)m * m) / (2.0 * l - 1)) * prev;
    }
  }
}

// Calls f(flat, vec[3]) for every VSWF Phi_f(k d) (outgoing), far=false, or the
// far-field amplitude F_f(d^), far=true (|d| ignored).
template <typename Fn>
__device__ void for_each_wave(int nmax, double k, double dx, double dy, double dz, bool far, Fn f) {
  const int L = nmax * (nmax + 2);
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double ct = dz / r, st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double rho = sqrt(dx * dx + dy * dy);
  double cp = rho > 0 ? dx / rho : 1.0, sp = rho > 0 ? dy / rho : 0.0;
  double P[NM1][NM1], pi[NM1][NM1], tau[NM1][NM1];
  legendre_tables(nmax, ct, st, P, pi, tau);
  double2 h[NM1 + 1];
  double kr = k * r;
  if (!far) {
    double s, c;
    sincos(kr, &s, &c);
    double ix = 1.0 / kr;
    h[0] = make_double2(s * ix, -c * ix);
    h[1] = make_double2(-ix * c + ix * ix * s, -ix * s - ix * ix * c);
    for (int q = 1; q < nmax; ++q) {
      double fq = (2 * q + 1) * ix;
      h[q + 1] = make_double2(fq * h[q].x - h[q - 1].x, fq * h[q].y - h[q - 1].y);
    }
  }
  double3 rh = make_double3(st * cp, st * sp, ct), th = make_double3(ct * cp, ct * sp, -st), ph = make_double3(-sp, cp, 0.0);
  const double ir[4] = {1, 0, -1, 0}, ii[4] = {0, 1, 0, -1};
  for (int l = 1; l <= nmax; ++l) {
    double cl = 1.0 / sqrt(2.0 * l * (l + 1));
    double2 zM, zNr, zNt;  // radial factors of M, of N's radial part, of N's tangential part
    if (far) {
      int e = (3 * (l + 1)) & 3;  // (-i)^{l+1} = i^{3(l+1)}
      zM = make_double2(ir[e], ii[e]);
      int e2 = (3 * l) & 3;
      zNt = make_double2(ir[e2], ii[e2]);
      zNr = make_double2(0, 0);
    } else {
      zM = h[l];
      zNr = cscale(h[l], l * (l + 1.0) / kr);
      zNt = make_double2(h[l - 1].x - l * h[l].x / kr, h[l - 1].y - l * h[l].y / kr);
    }
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double mpi = m * pi[l][am], ta = tau[l][am], pb = P[l][am];
      double sm, cm;
      sincos(m * atan2(sp, cp), &sm, &cm);
      double2 e = make_double2(cm, sm);
      // M: c z [ i mpi th - ta ph ] e ; N: c [ zNr pb r + zNt (ta th + i mpi ph) ] e
      double2 aM = cmul(cscale(zM, cl), e), aNr = cmul(cscale(zNr, cl * pb), e), aNt = cmul(cscale(zNt, cl), e);
      double2 vM[3], vN[3];
      const double thv[3] = {th.x, th.y, th.z}, phv[3] = {ph.x, ph.y, ph.z}, rhv[3] = {rh.x, rh.y, rh.z};
      for (int c = 0; c < 3; ++c) {
        // i*mpi*th_c - ta*ph_c   and   ta*th_c + i*mpi*ph_c
        double2 gM = make_double2(-ta * phv[c], mpi * thv[c]);
        double2 gN = make_double2(ta * thv[c], mpi * phv[c]);
        vM[c] = cmul(aM, gM);
        vN[c] = cadd(cscale(aNr, rhv[c]), cmul(aNt, gN));
      }
      int n = l * (l + 1) + m - 1;
      f(n, vM);
      f(L + n, vN);
    }
  }
}

// partial E over a chunk of scatterers: grid (M, chunks); block reduce
__global__ void field_kernel(const double* __restrict__ pos, int64_t N, double k, int nmax, const double2* __restrict__ s,
                             const double* __restrict__ pts, int64_t M, int far, double2* __restrict__ part) {
  const int64_t a = blockIdx.x;
  const int P = num_coeffs(nmax);
  __shared__ double2 red[3][128];
  double2 E[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  double ux = 0, uy = 0, uz = 0;
  if (far) {  // direction (theta, phi)
    double s_, c_, sp_, cp_;
    sincos(pts[2 * a], &s_, &c_);
    sincos(pts[2 * a + 1], &sp_, &cp_);
    ux = s_ * cp_;
    uy = s_ * sp_;
    uz = c_;
  }
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.y * blockDim.x) {
    const double2* si = s + i * P;
    double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    auto fn = [&](int f, const double2* v) {
      double2 c = si[f];
      for (int q = 0; q < 3; ++q) acc[q] = cadd(acc[q], cmul(c, v[q]));
    };
    if (far) {
      for_each_wave(nmax, k, ux, uy, uz, true, fn);
      double ph = -k * (ux * pos[3 * i] + uy * pos[3 * i + 1] + uz * pos[3 * i + 2]);
      double sn, cs;
      sincos(ph, &sn, &cs);
      for (int q = 0; q < 3; ++q) E[q] = cadd(E[q], cmul(make_double2(cs, sn), acc[q]));
    } else {
      for_each_wave(nmax, k, pts[3 * a] - pos[3 * i], pts[3 * a + 1] - pos[3 * i + 1], pts[3 * a + 2] - pos[3 * i + 2],
                    false, fn);
      for (int q = 0; q < 3; ++q) E[q] = cadd(E[q], acc[q]);
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
__global__ void adjoint_source_kernel(const double* __restrict__ pos, int64_t N, double k, int nmax,
                                      const double* __restrict__ xf, const double2* __restrict__ Etot,
                                      double2* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int P = num_coeffs(nmax);
  double2 ce[3] = {cconj(Etot[0]), cconj(Etot[1]), cconj(Etot[2])};
  for_each_wave(nmax, k, xf[0] - pos[3 * i], xf[1] - pos[3 * i + 1], xf[2] - pos[3 * i + 2], false,
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
  if (M == 0) return TMAT_OK;
  int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(N, 128), std::max<int64_t>(1, 4 * ctx->num_sms / std::max<int64_t>(M, 1))));
  if (nchunk > 65535) nchunk = 65535;
  double2* part;
  TM_TRY(scratch(ctx, "fld_part", sizeof(double2) * M * nchunk * 3, (void**)&part));
  field_kernel<<<dim3((unsigned)M, nchunk), 128, 0, ctx->stream>>>(pos, N, k, nmax, s, pts, M, far ? 1 : 0, part);
  TM_LAUNCHED(ctx);
  field_reduce_kernel<<<(unsigned)cdiv(M * 3, 128), 128, 0, ctx->stream>>>(part, M, nchunk, E);
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
    adjoint_source_kernel<<<(unsigned)cdiv(N, 64), 64, 0, ctx->stream>>>((const double*)sp.dev, N, k, nmax,
                                                                         (const double*)sx.dev, E, (double2*)sv.dev);
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
  if (!is_device_ptr(pts) || !is_device_ptr(E_out) || (N > 0 && (!is_device_ptr(pos) || !is_device_ptr(s))))
    return TMAT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TMAT_ECUDA;
  }
  double2* part = nullptr;
  int rc = noalloc_scratch(dev, &part);
  if (rc != TMAT_OK) return rc;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t nchunk = std::min<int64_t>(cdiv(N, 128), std::max<int64_t>(1, 4 * sms / M));
  nchunk = std::min<int64_t>(nchunk, TMAT_NOALLOC_FIELD_SLOTS / (3 * M));
  nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, 65535));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double k = 2.0 * M_PI * n_bg / wavelength;
  field_kernel<<<dim3((unsigned)M, (unsigned)nchunk), 128, 0, st>>>(pos, N, k, nmax, (const double2*)s, pts, M, 0,
                                                                     part);
  field_reduce_kernel<<<(unsigned)cdiv(M * 3, 128), 128, 0, st>>>(part, M, (int)nchunk, (double2*)E_out);
  if (cudaGetLastError() != cudaSuccess) return TMAT_ECUDA;
  return TMAT_OK;
}
