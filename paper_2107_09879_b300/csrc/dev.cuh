// Device-side helpers: complex arithmetic on float2/double2 and the outgoing
// spherical Hankel functions by upward recurrence.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "../../include/tmat.h"

namespace tmat {

// Programmatic dependent launch: a kernel launched with launch_pdl (below) may become
// resident while its predecessor in the stream drains; it waits here, before its first
// global access, until the predecessor's writes are visible (a no-op for a plain launch).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialisation (the kernel must begin with pdl_wait()):
// the launch latency overlaps the predecessor's last wave instead of following it.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(cudaStream_t stream, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename R> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename R> using C = typename cplx<R>::t;

template <typename R> __host__ __device__ __forceinline__ C<R> mk(R a, R b) { C<R> z; z.x = a; z.y = b; return z; }
template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> __host__ __device__ __forceinline__ T csub(T a, T b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
template <typename T> __host__ __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
template <typename T, typename R> __host__ __device__ __forceinline__ T cscale(T a, R s) { a.x *= s; a.y *= s; return a; }
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }

// h_q^(1)(x), q = 0..Q-1 for real x > 0, by upward recurrence
// h_{q+1} = (2q+1)/x h_q - h_{q-1}, which is stable for the outgoing Hankel
// function (it is dominated by y_q). e^{ix} is taken from an fp64 argument
// reduced modulo 2 pi, so the fp32 version keeps the phase of large k d.
template <typename R, int Q>
__device__ __forceinline__ void hankel_up(double x, C<R> (&h)[Q]) {
  const double twopi = 6.283185307179586476925286766559;
  double xr = x - twopi * rint(x * (1.0 / twopi));
  R s, c;
  if constexpr (sizeof(R) == 4) {
    sincosf((float)xr, &s, &c);
  } else {
    sincos(xr, &s, &c);
  }
  R xf = (R)x;
  R ix = (R)1 / xf;
  // h0 = -i e^{ix}/x ; h1 = -e^{ix}(x + i)/x^2 = e^{ix}(-1/x - i/x^2)
  h[0] = mk<R>(s * ix, -c * ix);
  if (Q > 1) {
    R a = -ix, b = -ix * ix;  // (a + ib) e^{ix}
    h[1] = mk<R>(a * c - b * s, a * s + b * c);
  }
#pragma unroll
  for (int q = 1; q + 1 < Q; ++q) {
    R f = (R)(2 * q + 1) * ix;
    h[q + 1] = mk<R>(f * h[q].x - h[q - 1].x, f * h[q].y - h[q - 1].y);
  }
}

// Interaction weight of a pair at distance d: 1 inside cutoff - taper, a
// raised-cosine fall-off 0.5 (1 + cos(pi (d - (cutoff - taper)) / taper)) over
// the last `taper` before the cutoff, 1 everywhere when taper == 0 (hard
// cutoff) or cutoff <= 0 (every pair). Pairs beyond the cutoff are not coupled.
__host__ __device__ __forceinline__ double taper_weight(double d, double cutoff, double taper) {
  if (!(taper > 0) || !(cutoff > 0)) return 1.0;
  double d0 = cutoff - taper;
  if (d <= d0) return 1.0;
  if (d >= cutoff) return 0.0;
  return 0.5 * (1.0 + cos(3.14159265358979323846 * (d - d0) / taper));
}

// d w / d d of taper_weight (zero outside the taper, where w is constant)
__host__ __device__ __forceinline__ double taper_dweight(double d, double cutoff, double taper) {
  if (!(taper > 0) || !(cutoff > 0)) return 0.0;
  double d0 = cutoff - taper;
  if (d <= d0 || d >= cutoff) return 0.0;
  const double pi = 3.14159265358979323846;
  return -0.5 * (pi / taper) * sin(pi * (d - d0) / taper);
}

// pi_l^m(b) = Pbar_l^m(cos b)/sin b (m >= 1) and tau_l^m(b) = d Pbar_l^m / d b,
// normalised Legendre functions without the Condon-Shortley phase.
__device__ inline void pi_tau(int l, int m, double beta, double* pi_out, double* tau_out) {
  double s, c;
  sincos(beta, &s, &c);
  int mu = m < 1 ? 1 : m;  // m = 0 needs pi^1 for tau
  double df = 1.0, f2 = 1.0;
  for (int t = 1; t < 2 * mu; t += 2) df *= t;
  for (int t = 2; t <= 2 * mu; ++t) f2 *= t;
  double p_prev = 0.0, p_cur = sqrt((2 * mu + 1) / (2.0 * f2)) * df * pow(s, (double)(mu - 1));
  double pis[TMAT_NMAX_MAX + 2];
  for (int t = 0; t < TMAT_NMAX_MAX + 2; ++t) pis[t] = 0.0;
  if (mu <= l) pis[mu] = p_cur;
  for (int ll = mu + 1; ll <= l; ++ll) {
    double a = sqrt((4.0 * ll * ll - 1) / ((double)ll * ll - (double)mu * mu));
    double b = sqrt(((ll - 1.0) * (ll - 1.0) - (double)mu * mu) / (4.0 * (ll - 1.0) * (ll - 1.0) - 1));
    double pn = a * (c * p_cur - b * p_prev);
    p_prev = p_cur;
    p_cur = pn;
    pis[ll] = pn;
  }
  if (m >= 1) {
    *pi_out = (m <= l) ? pis[l] : 0.0;
    double prev = (l - 1 >= m) ? pis[l - 1] : 0.0;
    *tau_out = (m <= l) ? (l * c * pis[l] - sqrt((2.0 * l + 1) * ((double)l * l - (double)m * m) / (2.0 * l - 1)) * prev) : 0.0;
  } else {
    *pi_out = 0.0;
    *tau_out = -sqrt(l * (l + 1.0)) * s * pis[l];  // -sqrt(l(l+1)) Pbar_l^1
  }
}

}  // namespace tmat
