// Restarted GMRES(m) (Saad, Iterative Methods, Alg. 6.9/6.11) for R right-hand
// sides at once, all state resident on the device: the paper solves its system
// with GMRES using only matrix-vector products (App. I, I-D). Arnoldi uses
// classical Gram-Schmidt applied twice (CGS2) with fp64 dot products and fp64
// Hessenberg / Givens / least-squares work; basis vectors are complex64 or
// complex128. Reductions are two-stage with a fixed order (deterministic).
#include <atomic>
#include <chrono>
#include <cstring>
#include <cmath>

#include <cuda_fp16.h>

#include "dev.cuh"
#include "dfloat.cuh"
#include "solver.h"

namespace tmat {

constexpr int DOT_CHUNK = 8;
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double2 shfl_down2(double2 v, int o) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, o);
  v.y = __shfl_down_sync(0xffffffffu, v.y, o);
  return v;
}

// part[(r*maxv + k)*nb + b] = partial sum_i conj(V_k[r][i]) w[r][i], k < nvec
template <typename VR>
__global__ void __launch_bounds__(RED_THREADS)
dots_kernel(const C<VR>* __restrict__ V, int64_t vstride, int nvec, const C<VR>* __restrict__ w, int64_t n,
            int64_t rstride, double2* __restrict__ part, int maxv, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  __shared__ double2 red[RED_THREADS / 32][DOT_CHUNK];
  const int nb = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const C<VR>* wr = w + r * rstride;
  for (int k0 = 0; k0 < nvec; k0 += DOT_CHUNK) {
    double2 acc[DOT_CHUNK];
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c) acc[c] = make_double2(0, 0);
    for (int64_t i = (int64_t)b * blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x) {
      C<VR> wv = wr[i];
      double wx = wv.x, wy = wv.y;
#pragma unroll
      for (int c = 0; c < DOT_CHUNK; ++c) {
        if (k0 + c < nvec) {
          C<VR> v = V[(int64_t)(k0 + c) * vstride + r * rstride + i];
          double vx = v.x, vy = v.y;
          acc[c].x = fma(vx, wx, fma(vy, wy, acc[c].x));   // conj(v) w
          acc[c].y = fma(vx, wy, fma(-vy, wx, acc[c].y));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c) {
      double2 v = acc[c];
      for (int o = 16; o > 0; o >>= 1) {
        double2 t = shfl_down2(v, o);
        v.x += t.x;
        v.y += t.y;
      }
      if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < DOT_CHUNK && k0 + threadIdx.x < nvec) {
      double2 s = make_double2(0, 0);
      for (int q = 0; q < RED_THREADS / 32; ++q) {
        s.x += red[q][threadIdx.x].x;
        s.y += red[q][threadIdx.x].y;
      }
      part[((int64_t)r * maxv + k0 + threadIdx.x) * nb + b] = s;
    }
    __syncthreads();
  }
}


// ---- complex64 vectors: fp32 products, fp64 accumulation across warps/blocks ----
// B300 runs fp64 FMAs at ~1/75 of the fp32 rate, so the per-element products of
// the complex64 Krylov vectors are done in fp32 (a lane sums the products of its
// elements, a warp its 32 lanes), and only the per-warp partials are summed in fp64.
// Work unit = one warp: D32_VPW basis vectors over one contiguous element range; the
// ranges per vector group are chosen so that ~64 warps per SM stream at once, each
// with D32_VPW + 1 independent 512-byte loads per step (the same occupancy-driven
// pattern as the update kernel). w is re-read once per vector group (from L1/L2).
// (measured on a B300 for 2 RHS of 1.92 M values and j = 2..30: two vectors per warp, four
// blocks per SM, the element loop unrolled by two and ~64 warps per SM reach 3.5-5.8 TB/s,
// eight vectors per warp at two blocks per SM 1.8-4.6 TB/s)
constexpr int D32_VPW = 2;
constexpr int D32_NBMAX = 1024;  // element ranges per group (a multiple of 8)
// The ranges of a group come in blocks of eight (one per warp of a CTA): a CTA sums its
// eight warp partials in a fixed order and writes one partial per dot, so a dot has
// ranges / 8 partials, summed by the Hessenberg step in a fixed order.

struct Dots32Plan {
  int groups, ranges, blocks;
};

static inline Dots32Plan dots32_plan(int64_t n, int nvec, int num_sms, int R) {
  Dots32Plan p;
  p.groups = (nvec + D32_VPW - 1) / D32_VPW;
  const int64_t target = (int64_t)num_sms * 64 / std::max(1, R);  // warps per RHS
  int64_t nr = cdiv(target, (int64_t)p.groups);
  nr = std::min<int64_t>(nr, std::max<int64_t>(1, cdiv(n / 2, (int64_t)32 * 16)));
  p.ranges = (int)(cdiv(std::max<int64_t>(1, std::min<int64_t>(nr, D32_NBMAX)), 8) * 8);
  p.blocks = p.groups * (p.ranges / 8);
  return p;
}

// TWO: also dots against a second target w2 into part2 (one read of the basis for both).
template <bool TWO>
__global__ void __launch_bounds__(256, 4)
dots32_kernel(const float2* __restrict__ V, int64_t vstride, int nvec, const float2* __restrict__ w, int64_t n,
              int64_t rstride, float4* __restrict__ part, int maxv, int groups, int ranges,
              const int* __restrict__ active, const float2* __restrict__ w2 = nullptr,
              float4* __restrict__ part2 = nullptr) {
  pdl_wait();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if ((int64_t)blockIdx.x >= (int64_t)groups * (ranges / 8)) return;  // uniform over the CTA
  __shared__ float2 bred[TWO ? 2 : 1][D32_VPW][8];  // warp sums; the last warp to finish adds them
  __shared__ unsigned bdone;
  if (threadIdx.x == 0) bdone = 0;
  __syncthreads();
  const int64_t unit = (int64_t)blockIdx.x * 8 + wid;
  const int g = (int)(unit / ranges), b = (int)(unit % ranges);
  const int kb = g * D32_VPW;
  const int64_t n2 = n >> 1;  // float4 = two complex values (n is even)
  const int64_t per = ((n2 + ranges - 1) / ranges + 31) / 32 * 32;
  const int64_t lo = (int64_t)b * per, hi = lo + per < n2 ? lo + per : n2;
  const float4* w4 = reinterpret_cast<const float4*>(w + r * rstride);
  const float4* v4[D32_VPW];
#pragma unroll
  for (int q = 0; q < D32_VPW; ++q) {
    const int k = kb + q < nvec ? kb + q : kb;  // out-of-range vectors read a valid one, unused
    v4[q] = reinterpret_cast<const float4*>(V + (int64_t)k * vstride + r * rstride);
  }
  const float4* w24 = TWO ? reinterpret_cast<const float4*>(w2 + r * rstride) : nullptr;
  float2 acc[D32_VPW], acc2[TWO ? D32_VPW : 1];
#pragma unroll
  for (int q = 0; q < D32_VPW; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < (TWO ? D32_VPW : 1); ++q) acc2[q] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int64_t i = lo + lane; i < hi; i += 32) {
    const float4 wv = w4[i];
    float4 wv2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TWO) wv2 = w24[i];
    float4 v[D32_VPW];
#pragma unroll
    for (int q = 0; q < D32_VPW; ++q) v[q] = v4[q][i];
#pragma unroll
    for (int q = 0; q < D32_VPW; ++q) {
      // conj(v) w for both complex values
      acc[q].x = fmaf(v[q].x, wv.x, fmaf(v[q].y, wv.y, fmaf(v[q].z, wv.z, fmaf(v[q].w, wv.w, acc[q].x))));
      acc[q].y = fmaf(v[q].x, wv.y, fmaf(-v[q].y, wv.x, fmaf(v[q].z, wv.w, fmaf(-v[q].w, wv.z, acc[q].y))));
      if (TWO) {
        acc2[q].x = fmaf(v[q].x, wv2.x, fmaf(v[q].y, wv2.y, fmaf(v[q].z, wv2.z, fmaf(v[q].w, wv2.w, acc2[q].x))));
        acc2[q].y = fmaf(v[q].x, wv2.y, fmaf(-v[q].y, wv2.x, fmaf(v[q].z, wv2.w, fmaf(-v[q].w, wv2.z, acc2[q].y))));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < D32_VPW; ++q) {
    float2 v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) bred[0][q][wid] = v;
    if (TWO) {
      float2 v2 = acc2[q];
      for (int o = 16; o > 0; o >>= 1) {
        v2.x += __shfl_down_sync(0xffffffffu, v2.x, o);
        v2.y += __shfl_down_sync(0xffffffffu, v2.y, o);
      }
      if (lane == 0) bred[TWO ? 1 : 0][q][wid] = v2;
    }
  }
  // the last warp of the CTA (fence, then a shared counter) sums the eight warp sums in
  // warp order and writes the CTA's partial; the others leave without waiting
  unsigned prev = 0;
  if (lane == 0) {
    __threadfence_block();
    prev = atomicAdd(&bdone, 1u);
  }
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != 7) return;
  __threadfence_block();
  if (lane < (TWO ? 2 : 1) * D32_VPW) {
    const int tg = lane / D32_VPW, q = lane % D32_VPW;
    if (kb + q < nvec) {
      // double-float sum in warp order: (re hi, re lo, im hi, im lo)
      float4 t = make_float4(bred[tg][q][0].x, 0.f, bred[tg][q][0].y, 0.f);
#pragma unroll
      for (int w8 = 1; w8 < 8; ++w8) {
        df_add(t.x, t.y, bred[tg][q][w8].x, 0.f, t.x, t.y);
        df_add(t.z, t.w, bred[tg][q][w8].y, 0.f, t.z, t.w);
      }
      const int RB = ranges / 8;
      (tg ? part2 : part)[((int64_t)r * maxv + kb + q) * RB + (b >> 3)] = t;
    }
  }
}

// out[r*maxv + k] = sum_b part[(r*maxv + k)*nb + b]: one block of RED2_THREADS per
// (r, k); each thread sums a strided subset of the block partials, then a fixed tree
// (deterministic order).
constexpr int RED2_THREADS = 64;
__global__ void __launch_bounds__(RED2_THREADS)
reduce_kernel(const double2* __restrict__ part, int nb, int nvec, int maxv, double2* __restrict__ out,
              const int* __restrict__ active) {
  pdl_wait();
  const int r = blockIdx.x, k = blockIdx.y;
  if (k >= nvec) return;
  if (active && !active[r]) return;
  const double2* pp = part + ((int64_t)r * maxv + k) * nb;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < nb; b += RED2_THREADS) {
    const double2 v = pp[b];
    s.x += v.x;
    s.y += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double2 t = shfl_down2(s, o);
    s.x += t.x;
    s.y += t.y;
  }
  __shared__ double2 w2[RED2_THREADS / 32];
  if ((threadIdx.x & 31) == 0) w2[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = w2[0];
    for (int q = 1; q < RED2_THREADS / 32; ++q) {
      t.x += w2[q].x;
      t.y += w2[q].y;
    }
    out[r * maxv + k] = t;
  }
}

static inline void launch_reduce(tmat_ctx* ctx, const double2* part, int nb, int nvec, int maxv, double2* out,
                                 const int* active, int R) {
  // launched behind its producer's last wave (the launch's result is checked by the caller)
  launch_pdl(ctx->stream, reduce_kernel, dim3(R, nvec), dim3(RED2_THREADS), 0, part, nb, nvec, maxv, out, active);
}

// ||v[r]||^2 block partials of complex64 vectors into part[(r*maxv + 0)*nb + b] (as the
// .x of a double2): float4 loads, four in flight per thread, fp32 per thread, fp64 per block
__global__ void __launch_bounds__(256)
norm32_kernel(const float2* __restrict__ v, int64_t n, int64_t rstride, double2* __restrict__ part, int maxv,
              const int* __restrict__ active) {
  pdl_wait();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int64_t n2 = n >> 1;
  const float4* v4 = reinterpret_cast<const float4*>(v + r * rstride);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.f;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n2; i += 4 * stride) {
    float4 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = v4[i + t * stride];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc += a[t].x * a[t].x + a[t].y * a[t].y + a[t].z * a[t].z + a[t].w * a[t].w;
  }
  for (; i < n2; i += stride) {
    const float4 a = v4[i];
    acc += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
  }
  double d = acc;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ws[q];
    part[(int64_t)r * maxv * gridDim.x + blockIdx.x] = make_double2(t, 0.0);  // slot k = 0
  }
}

// ||v[r]||^2 block partials of complex128 vectors (fp64 throughout), as norm32_kernel: four
// loads in flight per thread, a fixed summation order
__global__ void __launch_bounds__(256)
norm64_kernel(const double2* __restrict__ v, int64_t n, int64_t rstride, double2* __restrict__ part, int maxv,
              const int* __restrict__ active) {
  pdl_wait();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double2* vr = v + r * rstride;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    double2 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = vr[i + t * stride];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = fma(a[t].x, a[t].x, fma(a[t].y, a[t].y, acc));
  }
  for (; i < n; i += stride) {
    const double2 a = vr[i];
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ws[q];
    part[(int64_t)r * maxv * gridDim.x + blockIdx.x] = make_double2(t, 0.0);  // slot k = 0
  }
}

// out[r][i] += sign * sum_k V_k[r][i] coef[r][k]
template <typename VR, typename XR>
__global__ void update_kernel(const C<VR>* __restrict__ V, int64_t vstride, int nvec, const double2* __restrict__ coef,
                              int maxv, double sign, C<XR>* __restrict__ out, int64_t n, int64_t rstride,
                              const int* __restrict__ active, const int* __restrict__ ncols) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int nv = ncols ? min(nvec, ncols[r]) : nvec;  // only the columns this RHS built
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sx = 0, sy = 0;
    for (int k = 0; k < nv; ++k) {
      C<VR> v = V[(int64_t)k * vstride + r * rstride + i];
      double2 c = coef[r * maxv + k];
      sx += (double)v.x * c.x - (double)v.y * c.y;
      sy += (double)v.x * c.y + (double)v.y * c.x;
    }
    C<XR> o = out[r * rstride + i];
    o.x = (XR)((double)o.x + sign * sx);
    o.y = (XR)((double)o.y + sign * sy);
    out[r * rstride + i] = o;
  }
}

// x[r] += sum_{k < ncols[r]} V_k[r] y[r][k] for complex64 bases: the sum in fp32 (the
// coefficients rounded to fp32 once, in shared memory), the addition to x in fp64
__global__ void __launch_bounds__(256)
xupdate32_kernel(const float2* __restrict__ V, int64_t vstride, int nvec, const double2* __restrict__ coef, int maxv,
                 double2* __restrict__ x, int64_t n, int64_t rstride, const int* __restrict__ ncols) {
  const int r = blockIdx.y;
  const int nv = ncols ? min(nvec, ncols[r]) : nvec;
  extern __shared__ float2 xcs[];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const double2 c = coef[r * maxv + k];
    xcs[k] = make_float2((float)c.x, (float)c.y);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f;
    for (int k = 0; k < nv; ++k) {
      const float2 v = V[(int64_t)k * vstride + r * rstride + i];
      const float2 c = xcs[k];
      sx = fmaf(v.x, c.x, fmaf(-v.y, c.y, sx));
      sy = fmaf(v.x, c.y, fmaf(v.y, c.x, sy));
    }
    double2 o = x[r * rstride + i];
    o.x += sx;
    o.y += sy;
    x[r * rstride + i] = o;
  }
}

// y[r] = scale[r] * x[r] (scale from a device vector: 1/norm, or 0 if norm == 0)
template <typename XR, typename YR>
__global__ void scale_kernel(const C<XR>* __restrict__ x, C<YR>* __restrict__ y, int64_t n, int64_t rstride,
                             const double* __restrict__ norm, int inv, const int* __restrict__ active) {
  pdl_wait();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  double s = norm ? norm[r] : 1.0;
  if (inv) s = (s > 0) ? 1.0 / s : 0.0;
  if constexpr (std::is_same_v<YR, float>) {
    // a complex64 result: the product in fp32 (the B300's fp64 rate would bound this pass)
    const float sf = (float)s;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const C<XR> v = x[r * rstride + i];
      y[r * rstride + i] = make_float2((float)v.x * sf, (float)v.y * sf);
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      C<XR> v = x[r * rstride + i];
      C<YR> o;
      o.x = (YR)((double)v.x * s);
      o.y = (YR)((double)v.y * s);
      y[r * rstride + i] = o;
    }
  }
}

// out[r] = b[r] - y[r] in the type of out
template <typename BR, typename YR>
__global__ void residual_kernel(const C<BR>* __restrict__ b, const C<YR>* __restrict__ y, C<BR>* __restrict__ out,
                                int64_t total) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    C<BR> bv = b[i];
    C<YR> yv = y[i];
    if constexpr (std::is_same_v<BR, float> && std::is_same_v<YR, float>)
      out[i] = make_float2(bv.x - yv.x, bv.y - yv.y);  // fp32 throughout: no fp64 round trip
    else
      out[i] = mk<BR>((BR)((double)bv.x - (double)yv.x), (BR)((double)bv.y - (double)yv.y));
  }
}

template <typename XR, typename YR>
__global__ void convert_kernel(const C<XR>* __restrict__ x, C<YR>* __restrict__ y, int64_t total) {
  pdl_wait();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = mk<YR>((YR)x[i].x, (YR)x[i].y);
}

// x[r] += alpha[r] * d[r]
__global__ void axpy_scaled_kernel(double2* __restrict__ x, const double2* __restrict__ d, const double* __restrict__ alpha,
                                   int64_t n, int64_t rstride) {
  pdl_wait();
  const int r = blockIdx.y;
  const double a = alpha[r];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = x[r * rstride + i], w = d[r * rstride + i];
    v.x += a * w.x;
    v.y += a * w.y;
    x[r * rstride + i] = v;
  }
}

// Small per-RHS state of one GMRES run (device)
struct GState {
  double2 *hA, *hB;      // [R][maxv] CGS coefficients of pass 1 and 2
  double2 *H;            // [R][maxv][m] rotated Hessenberg (upper triangle used)
  double2 *cs, *sn, *g;  // rotations [R][m], rhs [R][maxv]
  double2 *y;            // [R][maxv] least-squares solution
  double *nrm;           // [R] norm of the new vector / residual
  double *tol_abs;       // [R]
  int *active, *ncols, *flags;
  // delayed CGS2 (complex64 vectors): unrotated Hessenberg [R][maxv][m] and the update
  // coefficients [R][maxv] with the self-scales [R]
  double2 *Hu;
  float2 *cA, *cB;
  float *selfA, *selfB;
};

__global__ void cycle_init_kernel(GState s, int R, int maxv, const double* __restrict__ rnorm, const int* __restrict__ want) {
  pdl_wait();
  int r = threadIdx.x;
  if (r >= R) return;
  for (int k = 0; k < maxv; ++k) s.g[r * maxv + k] = make_double2(0, 0);
  double rn = rnorm[r];
  s.g[r * maxv] = make_double2(rn, 0);
  s.ncols[r] = 0;
  s.active[r] = (want[r] && rn > 0 && isfinite(rn)) ? 1 : 0;
}

__global__ void norm_from_dots_kernel(const double2* __restrict__ d, int maxv, double* __restrict__ nrm, int R,
                                      const int* __restrict__ active) {
  pdl_wait();
  int r = threadIdx.x;
  if (r >= R) return;
  if (active && !active[r]) return;
  nrm[r] = sqrt(fmax(d[r * maxv].x, 0.0));
}

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Givens step for column j, one block per RHS: the previous rotations and the new
// column are staged in shared memory by the block, then one thread applies the j
// rotations in order (the recurrence is serial) and writes the column back to
// H[r][.][j] in global memory (so the restart length is not bounded by registers).
// Givens step for column j of RHS r by the calling block (gsm: 2 m + maxv double2 of
// shared memory); the caller has checked that r is active.
__device__ void givens_block(GState& s, int r, int j, int m, int maxv, double2* gsm) {
  double2* cs = gsm;          // [j]
  double2* sn = cs + m;       // [j]
  double2* col = sn + m;      // [j + 1]
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs[i] = s.cs[r * m + i];
    sn[i] = s.sn[r * m + i];
  }
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double2 a = s.hA[r * maxv + i], b = s.hB[r * maxv + i];
    col[i] = make_double2(a.x + b.x, a.y + b.y);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = s.nrm[r];
    // rotation G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]]
    double2 t0 = col[0];
    for (int i = 0; i < j; ++i) {
      const double2 c = cs[i], sv = sn[i];
      const double2 t1 = col[i + 1];
      col[i] = make_double2(c.x * t0.x + c.y * t0.y + sv.x * t1.x + sv.y * t1.y,
                            c.x * t0.y - c.y * t0.x + sv.x * t1.y - sv.y * t1.x);
      t0 = make_double2(-(sv.x * t0.x - sv.y * t0.y) + (c.x * t1.x - c.y * t1.y),
                        -(sv.x * t0.y + sv.y * t0.x) + (c.x * t1.y + c.y * t1.x));
    }
    const double2 hjj = t0;
    const double2 hj1 = make_double2(hn, 0);  // H[j+1][j], never stored
    const double den = sqrt(cabs2(hjj) + cabs2(hj1));
    double2 c = make_double2(1, 0), sv = make_double2(0, 0);
    if (den > 0) {
      c = make_double2(hjj.x / den, hjj.y / den);
      sv = make_double2(hj1.x / den, hj1.y / den);
    }
    s.cs[r * m + j] = c;
    s.sn[r * m + j] = sv;
    col[j] = make_double2(den, 0);
    const double2 gj = s.g[r * maxv + j];
    s.g[r * maxv + j + 1] = make_double2(-(sv.x * gj.x - sv.y * gj.y), -(sv.x * gj.y + sv.y * gj.x));
    s.g[r * maxv + j] = make_double2(c.x * gj.x + c.y * gj.y, c.x * gj.y - c.y * gj.x);
    s.ncols[r] = j + 1;
    const double res = sqrt(cabs2(s.g[r * maxv + j + 1]));
    if (!isfinite(res) || !isfinite(hn)) {
      s.flags[r] |= 1;  // NaN / Inf
      s.active[r] = 0;
    } else if (res <= s.tol_abs[r] || hn == 0.0) {
      s.active[r] = 0;
    }
  }
  __syncthreads();
  double2* hcol = s.H + (int64_t)r * maxv * m + j;  // element i at hcol[i * m]
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hcol[(int64_t)i * m] = col[i];
  __syncthreads();
}

__global__ void givens_kernel(GState s, int R, int j, int m, int maxv) {
  const int r = blockIdx.x;
  if (r >= R || !s.active[r]) return;
  extern __shared__ double2 gsm[];
  givens_block(s, r, j, m, maxv, gsm);
}

// ---- delayed CGS2 (Arnoldi with the second projection one step late) ----------------
// Iteration j expands the pending vector u_j (slot j: first projection of A q_{j-1}
// against q_0..q_{j-1}, not normalised; q_0 for j = 0) with w = A u_j. One pass over the
// basis gives D1 = V^H u_j and D2 = V^H w (slots 0..j). With b1 = ||u_j||, s = D1/b1 and
// nu = sqrt(1 - |s|^2):
//   column j-1 (final)  H[0..j-1][j-1] += b1 s,  H[j][j-1] = b1 nu,  q_j = (u_j/b1 - Q s)/nu;
//   column j (first projection, by the Arnoldi relation A Q = Q_{j+1} H applied to A q_j =
//   (w/b1 - A Q s)/nu)  H[0..j][j] = ([z; zeta] - H s)/nu with z = D2/b1 and
//   zeta = (c - s^H z)/nu, c = D2[j]/b1^2;
//   u_{j+1} = (w/b1 - Q (z - (zeta/nu) s) - (zeta/(nu b1)) u_j)/nu.
// One more pass writes q_j into slot j and u_{j+1} into slot j+1 (both from one read of
// the basis): two passes over the basis per iteration instead of four. The Hessenberg
// columns are the classical Gram-Schmidt-twice ones; the reorthogonalisation of u_j uses the
// vector actually stored, so rounding in forming it is corrected as in CGS2.
// The step runs as one block per RHS with its inputs staged in shared memory in one phase:
// the dot partials of the pass (ranges / 8 double-float values per dot, summed here in a
// fixed order), the rotations, column j-1 and, for short cycles, the Hessenberg block the
// product H s needs, so the serial part waits on global memory once instead of once per
// quantity. The fp64 work is kept on few lanes (the B300 issues fp64 at a small fraction of
// its fp32 rate): the partial sums are double-float, the length-j vector steps run on one
// warp with warp reductions, H s takes one thread per row.
constexpr int DCGS2_HB = 48;  // Hessenberg blocks up to (48 + 1) x 48 are staged (j <= 48)
constexpr int DCGS2_THREADS = 256;
static inline size_t dcgs2_step_smem(int m, int maxv) {
  return sizeof(double2) * (4 * (size_t)maxv + 2 * (size_t)m + (size_t)(DCGS2_HB + 1) * DCGS2_HB);
}
__device__ __forceinline__ void dcgs2_cp16(void* dst, const void* src) {  // 16-byte cp.async
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
// the RHS's convergence flag to mapped host memory, then the step's tag (the host reads the
// flag once it sees the tag)
__device__ __forceinline__ void dcgs2_publish(int* hflag, int r, int act, int tag) {
  reinterpret_cast<volatile int*>(hflag)[r] = act;
  __threadfence_system();
  reinterpret_cast<volatile int*>(hflag)[TMAT_MAX_RHS + r] = tag;
}
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(DCGS2_THREADS)
dcgs2_step_kernel(GState s, const float4* __restrict__ part, const float4* __restrict__ part2, int RB, int j, int m,
                  int maxv, int R, int final_only, int stage_p, int* __restrict__ hflag, int tag) {
  pdl_wait();
  const int r = blockIdx.x;
  if (r >= R) return;
  if (j == 0 && final_only) return;
  extern __shared__ double2 dsm[];
  double2* sD1 = dsm;              // [maxv] V^H u_j
  double2* sD2 = sD1 + maxv;       // [maxv] V^H w
  double2* sv = sD2 + maxv;        // [maxv] s = D1 / b1
  double2* col = sv + maxv;        // [maxv] column j-1
  double2* scs = col + maxv;       // [m] rotations
  double2* ssn = scs + m;          // [m]
  double2* Hb = ssn + m;           // [(j + 1) * j] rows 0..j of columns 0..j-1 (j <= DCGS2_HB)
                                   // then (stage_p) the partials [S][RB] as double-float
  __shared__ __align__(16) double2 g_sh;
  __shared__ double2 zeta_sh;
  __shared__ double b1_sh, nu_sh;
  __shared__ int act_sh;
  const int tid = threadIdx.x, lane = tid & 31;
  double2* Hu = s.Hu + (int64_t)r * maxv * m;  // Hu[i * m + c]
  float2* cA = s.cA + (int64_t)r * maxv;
  float2* cB = s.cB + (int64_t)r * maxv;
  const bool stage_h = j <= DCGS2_HB;
  // ---- one phase of copies: dot partials, rotations, column j-1, the Hessenberg block, all
  // in flight at once (cp.async), then the sums from shared memory ----
  {
    const int S = final_only ? j + 1 : 2 * (j + 1);  // sums: D1[0..j] (and D2[0..j])
    float4* pst = reinterpret_cast<float4*>(Hb + (DCGS2_HB + 1) * DCGS2_HB);  // [S][RB] (stage_p)
    if (stage_p)
      for (int e = tid; e < S * RB; e += DCGS2_THREADS) {
        const int si = e / RB, bq = e % RB, k = si % (j + 1);
        dcgs2_cp16(pst + e, (si <= j ? part : part2) + ((int64_t)r * maxv + k) * RB + bq);
      }
    if (j > 0) {
      for (int i = tid; i < j - 1; i += DCGS2_THREADS) {
        dcgs2_cp16(scs + i, s.cs + r * m + i);
        dcgs2_cp16(ssn + i, s.sn + r * m + i);
      }
      for (int k = tid; k < j; k += DCGS2_THREADS) dcgs2_cp16(col + k, Hu + (int64_t)k * m + (j - 1));
      if (tid == 0) dcgs2_cp16(&g_sh, s.g + r * maxv + j - 1);
      if (stage_h && !final_only)
        for (int e = tid; e < (j + 1) * j; e += DCGS2_THREADS) {
          const int i = e / j, c = e % j;
          if (c >= i - 1 && c != j - 1) dcgs2_cp16(Hb + e, Hu + (int64_t)i * m + c);
        }
    }
    const int act0 = s.active[r];  // read while the copies are in flight (an inactive RHS leaves)
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    if (!act0) {
      if (tag && tid == 0) dcgs2_publish(hflag, r, 0, tag);
      return;
    }
    int tps = 32;  // threads per sum (a power of two)
    while (tps > 1 && tps * S > DCGS2_THREADS) tps >>= 1;
    const int per_round = DCGS2_THREADS / tps;
    for (int base = 0; base < S; base += per_round) {  // uniform trip count
      const int si = base + tid / tps, li = tid % tps;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);  // double-float (re hi, re lo, im hi, im lo)
      if (si < S) {
        const int k = si % (j + 1);
        const float4* pp = stage_p ? pst + (int64_t)si * RB : (si <= j ? part : part2) + ((int64_t)r * maxv + k) * RB;
#pragma unroll 4
        for (int bq = li; bq < RB; bq += tps) {
          const float4 v = pp[bq];
          df_add(acc.x, acc.y, v.x, v.y, acc.x, acc.y);
          df_add(acc.z, acc.w, v.z, v.w, acc.z, acc.w);
        }
      }
      for (int o = tps >> 1; o > 0; o >>= 1) {
        const float4 t = make_float4(__shfl_down_sync(0xffffffffu, acc.x, o, tps),
                                     __shfl_down_sync(0xffffffffu, acc.y, o, tps),
                                     __shfl_down_sync(0xffffffffu, acc.z, o, tps),
                                     __shfl_down_sync(0xffffffffu, acc.w, o, tps));
        df_add(acc.x, acc.y, t.x, t.y, acc.x, acc.y);
        df_add(acc.z, acc.w, t.z, t.w, acc.z, acc.w);
      }
      if (si < S && li == 0)
        (si <= j ? sD1 : sD2)[si % (j + 1)] =
            make_double2((double)acc.x + (double)acc.y, (double)acc.z + (double)acc.w);
    }
  }
  __syncthreads();
  if (j == 0) {
    if (tid == 0) {
      const double2 z0 = sD2[0];
      Hu[0] = z0;
      cB[0] = make_float2((float)z0.x, (float)z0.y);
      s.selfB[r] = 1.f;
      s.selfA[r] = 0.f;
    }
    return;
  }
  const int J = j - 1;
  if (tid < 32) {
    // ---- b1 = ||u_j||, s = D1 / b1, nu = sqrt(1 - |s|^2) (warp 0) ----
    const double b1 = sqrt(fmax(sD1[j].x, 0.0));
    const double ib1 = b1 > 0 ? 1.0 / b1 : 0.0;  // divisions by b1 and nu as products with reciprocals
    double ss = 0.0;
    for (int k = lane; k < j; k += 32) {
      const double2 v = make_double2(sD1[k].x * ib1, sD1[k].y * ib1);
      sv[k] = v;
      ss += v.x * v.x + v.y * v.y;
    }
    ss = warp_sum_d(ss);
    const double nu = b1 > 0 ? sqrt(fmax(1.0 - ss, 1e-30)) : 1.0;
    // ---- column j-1 final: H[0..j-1][j-1] += b1 s, H[j][j-1] = b1 nu ----
    for (int k = lane; k < j; k += 32) {
      double2 h = col[k];
      h.x += b1 * sv[k].x;
      h.y += b1 * sv[k].y;
      col[k] = h;
      Hu[(int64_t)k * m + J] = h;
      if (stage_h) Hb[k * j + J] = h;
    }
    const double hn = b1 * nu;  // subdiagonal H[j][j-1]
    __syncwarp();
    if (lane == 0) {
      Hu[(int64_t)j * m + J] = make_double2(hn, 0.0);
      if (stage_h) Hb[j * j + J] = make_double2(hn, 0.0);
      s.nrm[r] = hn;
      b1_sh = b1;
      nu_sh = nu;
      // ---- Givens step of column J (serial; G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]]) ----
      double2 t0 = col[0];
      for (int i = 0; i < J; ++i) {
        const double2 c = scs[i], sn = ssn[i];
        const double2 t1 = col[i + 1];
        col[i] = make_double2(c.x * t0.x + c.y * t0.y + sn.x * t1.x + sn.y * t1.y,
                              c.x * t0.y - c.y * t0.x + sn.x * t1.y - sn.y * t1.x);
        t0 = make_double2(-(sn.x * t0.x - sn.y * t0.y) + (c.x * t1.x - c.y * t1.y),
                          -(sn.x * t0.y + sn.y * t0.x) + (c.x * t1.y + c.y * t1.x));
      }
      const double2 hjj = t0;
      const double den = sqrt(cabs2(hjj) + hn * hn);
      double2 c = make_double2(1, 0), sn = make_double2(0, 0);
      if (den > 0) {
        const double iden = 1.0 / den;
        c = make_double2(hjj.x * iden, hjj.y * iden);
        sn = make_double2(hn * iden, 0.0);
      }
      s.cs[r * m + J] = c;
      s.sn[r * m + J] = sn;
      col[J] = make_double2(den, 0);
      const double2 gj = g_sh;
      const double2 gn = make_double2(-(sn.x * gj.x - sn.y * gj.y), -(sn.x * gj.y + sn.y * gj.x));
      s.g[r * maxv + J + 1] = gn;
      s.g[r * maxv + J] = make_double2(c.x * gj.x + c.y * gj.y, c.x * gj.y - c.y * gj.x);
      s.ncols[r] = J + 1;
      const double res = sqrt(cabs2(gn));
      int act = 1;
      if (!isfinite(res) || !isfinite(hn)) {
        s.flags[r] |= 1;  // NaN / Inf
        act = 0;
      } else if (res <= s.tol_abs[r] || hn == 0.0) {
        act = 0;
      }
      if (!act) s.active[r] = 0;
      act_sh = act;
      if (tag) dcgs2_publish(hflag, r, act, tag);
    }
  }
  __syncthreads();
  {
    double2* hcol = s.H + (int64_t)r * maxv * m + J;  // rotated column J, element i at hcol[i * m]
    for (int i = tid; i <= J; i += DCGS2_THREADS) hcol[(int64_t)i * m] = col[i];
  }
  const double b1 = b1_sh;
  if (final_only || !(b1 > 0) || !act_sh) return;
  const double ib1 = 1.0 / b1, inu = 1.0 / nu_sh;
  if (tid < 32) {
    // ---- zeta = (c - s^H z)/nu with z = D2/b1, c = D2[j]/b1^2 (warp 0) ----
    double zr = 0.0, zi = 0.0;
    for (int k = lane; k < j; k += 32) {
      const double2 z = make_double2(sD2[k].x * ib1, sD2[k].y * ib1);
      zr += sv[k].x * z.x + sv[k].y * z.y;  // conj(s) z
      zi += sv[k].x * z.y - sv[k].y * z.x;
    }
    zr = warp_sum_d(zr);
    zi = warp_sum_d(zi);
    const double ib2 = ib1 * ib1;
    const double2 zeta = make_double2((sD2[j].x * ib2 - zr) * inu, (sD2[j].y * ib2 - zi) * inu);
    if (lane == 0) zeta_sh = zeta;
    // ---- update coefficients ----
    const double zn_r = zeta.x * inu, zn_i = zeta.y * inu;  // zeta / nu
    for (int k = lane; k < j; k += 32) {
      const double2 sk = sv[k];
      const double2 z = make_double2(sD2[k].x * ib1, sD2[k].y * ib1);
      cA[k] = make_float2((float)(sk.x * inu), (float)(sk.y * inu));
      // (z - (zeta/nu) s)/nu
      const double2 t = make_double2(z.x - (zn_r * sk.x - zn_i * sk.y), z.y - (zn_r * sk.y + zn_i * sk.x));
      cB[k] = make_float2((float)(t.x * inu), (float)(t.y * inu));
    }
    if (lane == 0) {
      cB[j] = make_float2((float)(zn_r * inu * ib1), (float)(zn_i * inu * ib1));  // zeta / (nu^2 b1)
      s.selfA[r] = (float)(ib1 * inu);
      s.selfB[r] = (float)(ib1 * inu);
    }
  }
  __syncthreads();
  // ---- column j: H[i][j] = ([z; zeta]_i - (H s)_i)/nu over the final columns 0..j-1, one
  // thread per row (upper Hessenberg: H[i][c] = 0 for c < i - 1) ----
  const double2 zeta = zeta_sh;
  for (int i = tid; i <= j; i += DCGS2_THREADS) {
    double tx = 0.0, ty = 0.0;
    for (int c = i > 0 ? i - 1 : 0; c < j; ++c) {
      const double2 h = stage_h ? Hb[i * j + c] : Hu[(int64_t)i * m + c];
      tx += h.x * sv[c].x - h.y * sv[c].y;
      ty += h.x * sv[c].y + h.y * sv[c].x;
    }
    const double2 zi2 = i < j ? make_double2(sD2[i].x * ib1, sD2[i].y * ib1) : zeta;
    Hu[(int64_t)i * m + j] = make_double2((zi2.x - tx) * inu, (zi2.y - ty) * inu);
  }
}

// slot j <- selfA V_j - sum_{k<j} V_k cA_k  (if j > 0), and
// w      <- selfB w   - sum_{k<=j} V_k cB_k, from one read of V_0..V_j (complex64)
__global__ void __launch_bounds__(256)
dcgs2_update_kernel(float2* __restrict__ V, int64_t vstride, int j, GState s, int maxv, float2* __restrict__ w,
                    int64_t n, int64_t rstride) {
  pdl_wait();
  const int r = blockIdx.y;
  if (!s.active[r]) return;
  extern __shared__ float2 dcs[];  // cA[0..j), cB[0..j]
  float2* cA = dcs;
  float2* cB = dcs + j + 1;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    cA[k] = k < j ? s.cA[(int64_t)r * maxv + k] : make_float2(0.f, 0.f);
    cB[k] = s.cB[(int64_t)r * maxv + k];
  }
  __syncthreads();
  const float sA = s.selfA[r], sB = s.selfB[r];
  const int64_t n2 = n >> 1;
  float4* vj4 = reinterpret_cast<float4*>(V + (int64_t)j * vstride + r * rstride);
  float4* w4 = reinterpret_cast<float4*>(w + r * rstride);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), bsum = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k <= j; ++k) {
      const float4 v = reinterpret_cast<const float4*>(V + (int64_t)k * vstride + r * rstride)[i];
      const float2 cb = cB[k];
      bsum.x = fmaf(v.x, cb.x, fmaf(-v.y, cb.y, bsum.x));
      bsum.y = fmaf(v.x, cb.y, fmaf(v.y, cb.x, bsum.y));
      bsum.z = fmaf(v.z, cb.x, fmaf(-v.w, cb.y, bsum.z));
      bsum.w = fmaf(v.z, cb.y, fmaf(v.w, cb.x, bsum.w));
      const float2 ca = cA[k];
      a.x = fmaf(v.x, ca.x, fmaf(-v.y, ca.y, a.x));
      a.y = fmaf(v.x, ca.y, fmaf(v.y, ca.x, a.y));
      a.z = fmaf(v.z, ca.x, fmaf(-v.w, ca.y, a.z));
      a.w = fmaf(v.z, ca.y, fmaf(v.w, ca.x, a.w));
    }
    const float4 wv = w4[i];
    w4[i] = make_float4(sB * wv.x - bsum.x, sB * wv.y - bsum.y, sB * wv.z - bsum.z, sB * wv.w - bsum.w);
    if (j > 0) {
      const float4 u = vj4[i];
      vj4[i] = make_float4(sA * u.x - a.x, sA * u.y - a.y, sA * u.z - a.z, sA * u.w - a.w);
    }
  }
}


// ---- compressed basis: final vectors stored as scaled fp16 --------------------------
// For loose inner solves (tolerance >= 1e-2; every refinement step is closed by an
// fp64-accurate residual) the final basis vectors v_0..v_{j-1} are stored as fp16 pairs
// of sqrt(n) v (unit vectors: every scaled element stays below sqrt(n) < 65504, the
// rounding is ~5e-4 relative), halving the basis traffic of the Arnoldi passes; the
// pending vector and the operator's output stay in two fp32 slots, the arithmetic in fp32
// (the compressed-basis GMRES of Aliaga, Anzt et al., Concurr. Comput. 2022). The scale
// 1/sqrt(n) is folded into the dot products and into the update coefficients.
__device__ __forceinline__ float4 h16_load2(const uint2* __restrict__ p, int64_t i) {
  const uint2 u = p[i];
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ uint2 h16_pack2(float4 v) {
  const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned*>(&a);
  u.y = *reinterpret_cast<const unsigned*>(&b);
  return u;
}

// Dot-pass shape on the compressed basis (measured on a B300 for 2 RHS of 1.92 M values and
// j = 2..30: two vectors per warp, four blocks per SM, the element loop unrolled by two and
// ~64 warps per SM in all reach 3.2-4.7 TB/s, against 1.3-2.9 TB/s for eight vectors per
// warp at two blocks per SM): short warps with few streams keep more loads in flight.
constexpr int D16_VPW = 2;
struct Dots16Plan {
  int ranges, blocks;
};
static inline Dots16Plan dots16_plan(int64_t n, int gh, int num_sms, int R) {
  Dots16Plan p;
  const int64_t target = (int64_t)num_sms * 64 / std::max(1, R);  // warps per RHS
  int64_t nr = cdiv(target, (int64_t)gh + 1);
  nr = std::min<int64_t>(nr, std::max<int64_t>(1, cdiv(n / 2, (int64_t)32 * 16)));
  p.ranges = (int)(cdiv(std::max<int64_t>(1, std::min<int64_t>(nr, D32_NBMAX)), 8) * 8);
  p.blocks = (gh + 1) * (p.ranges / 8);
  return p;
}

// Dot pass of iteration j on the compressed basis: units of D16_VPW fp16 vectors of
// Vh[0..nh) (groups gh) and one unit group for the pending fp32 vector u (index nh),
// against the targets u and (TWO) w; partials as dots32_kernel, scaled back by inv_sc.
template <bool TWO>
__global__ void __launch_bounds__(256, 4)
dots16_kernel(const uint2* __restrict__ Vh, int64_t hstride, int nh, const float2* __restrict__ u, int64_t n,
              int64_t rstride, float4* __restrict__ part, int maxv, int gh, int ranges, const int* __restrict__ active,
              float inv_sc, const float2* __restrict__ w2 = nullptr, float4* __restrict__ part2 = nullptr) {
  pdl_wait();
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if ((int64_t)blockIdx.x >= (int64_t)(gh + 1) * (ranges / 8)) return;  // uniform over the CTA
  __shared__ float2 bred[TWO ? 2 : 1][D16_VPW][8];  // warp sums; the last warp to finish adds them
  __shared__ unsigned bdone;
  if (threadIdx.x == 0) bdone = 0;
  __syncthreads();
  const int64_t unit = (int64_t)blockIdx.x * 8 + wid;
  const int g = (int)(unit / ranges), b = (int)(unit % ranges);
  const bool pend = g == gh;  // the pending fp32 vector
  const int kb = pend ? nh : g * D16_VPW;
  const int nq = pend ? 1 : min(D16_VPW, nh - kb);
  const int64_t n2 = n >> 1;
  const int64_t per = ((n2 + ranges - 1) / ranges + 31) / 32 * 32;
  const int64_t lo = (int64_t)b * per, hi = lo + per < n2 ? lo + per : n2;
  const float4* u4 = reinterpret_cast<const float4*>(u + r * rstride);
  const float4* w24 = TWO ? reinterpret_cast<const float4*>(w2 + r * rstride) : nullptr;
  const uint2* h4[D16_VPW];
#pragma unroll
  for (int q = 0; q < D16_VPW; ++q) {
    const int k = q < nq ? kb + q : kb;  // unused slots read a valid vector
    h4[q] = reinterpret_cast<const uint2*>(Vh + ((int64_t)(pend ? 0 : k) * hstride + r * rstride) / 2);
  }
  float2 acc[D16_VPW], acc2[TWO ? D16_VPW : 1];
#pragma unroll
  for (int q = 0; q < D16_VPW; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < (TWO ? D16_VPW : 1); ++q) acc2[q] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int64_t i = lo + lane; i < hi; i += 32) {
    const float4 wv = u4[i];
    float4 wv2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TWO) wv2 = w24[i];
    float4 v[D16_VPW];
    if (pend) {
      v[0] = wv;
#pragma unroll
      for (int q = 1; q < D16_VPW; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int q = 0; q < D16_VPW; ++q) v[q] = h16_load2(h4[q], i);
    }
#pragma unroll
    for (int q = 0; q < D16_VPW; ++q) {
      acc[q].x = fmaf(v[q].x, wv.x, fmaf(v[q].y, wv.y, fmaf(v[q].z, wv.z, fmaf(v[q].w, wv.w, acc[q].x))));
      acc[q].y = fmaf(v[q].x, wv.y, fmaf(-v[q].y, wv.x, fmaf(v[q].z, wv.w, fmaf(-v[q].w, wv.z, acc[q].y))));
      if (TWO) {
        acc2[q].x = fmaf(v[q].x, wv2.x, fmaf(v[q].y, wv2.y, fmaf(v[q].z, wv2.z, fmaf(v[q].w, wv2.w, acc2[q].x))));
        acc2[q].y = fmaf(v[q].x, wv2.y, fmaf(-v[q].y, wv2.x, fmaf(v[q].z, wv2.w, fmaf(-v[q].w, wv2.z, acc2[q].y))));
      }
    }
  }
  const float sc = pend ? 1.0f : inv_sc;
#pragma unroll
  for (int q = 0; q < D16_VPW; ++q) {
    float2 v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) bred[0][q][wid] = make_float2(sc * v.x, sc * v.y);
    if (TWO) {
      float2 v2 = acc2[q];
      for (int o = 16; o > 0; o >>= 1) {
        v2.x += __shfl_down_sync(0xffffffffu, v2.x, o);
        v2.y += __shfl_down_sync(0xffffffffu, v2.y, o);
      }
      if (lane == 0) bred[TWO ? 1 : 0][q][wid] = make_float2(sc * v2.x, sc * v2.y);
    }
  }
  // the last warp of the CTA (fence, then a shared counter) sums the eight warp sums in
  // warp order and writes the CTA's partial; the others leave without waiting
  unsigned prev = 0;
  if (lane == 0) {
    __threadfence_block();
    prev = atomicAdd(&bdone, 1u);
  }
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != 7) return;
  __threadfence_block();
  if (lane < (TWO ? 2 : 1) * D16_VPW) {
    const int tg = lane / D16_VPW, q = lane % D16_VPW;
    if (q < nq) {
      // double-float sum in warp order: (re hi, re lo, im hi, im lo)
      float4 t = make_float4(bred[tg][q][0].x, 0.f, bred[tg][q][0].y, 0.f);
#pragma unroll
      for (int w8 = 1; w8 < 8; ++w8) {
        df_add(t.x, t.y, bred[tg][q][w8].x, 0.f, t.x, t.y);
        df_add(t.z, t.w, bred[tg][q][w8].y, 0.f, t.z, t.w);
      }
      const int RB = ranges / 8;
      (tg ? part2 : part)[((int64_t)r * maxv + kb + q) * RB + (b >> 3)] = t;
    }
  }
}

// Update pass of iteration j on the compressed basis (see dcgs2_update_kernel): the final
// v_j = selfA u - sum_{k<j} V_k cA_k (j = 0: v_0 = u) goes to Vh[j] as fp16 of sc v_j, and
// w <- selfB w - sum_{k<j} V_k cB_k - u cB_j, with V_k = Vh_k / sc.
// (measured shape: the k loop unrolled by four, four blocks per SM, 16 blocks per SM per
// RHS: 3.6-4.8 TB/s for j = 2..30 against 3.3-4.2 TB/s with the update kernel's grid)
__global__ void __launch_bounds__(256, 4)
dcgs2_update16_kernel(uint2* __restrict__ Vh, int64_t hstride, int j, GState s, int maxv,
                      const float2* __restrict__ u, float2* __restrict__ w, int64_t n, int64_t rstride, float sc) {
  pdl_wait();
  const int r = blockIdx.y;
  if (!s.active[r]) return;
  extern __shared__ float2 dcs[];  // cA[0..j) / sc, cB[0..j) / sc, cB[j]
  float2* cA = dcs;
  float2* cB = dcs + j + 1;
  const float inv_sc = 1.0f / sc;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    const float2 a = k < j ? s.cA[(int64_t)r * maxv + k] : make_float2(0.f, 0.f);
    const float2 c = s.cB[(int64_t)r * maxv + k];
    const float f = k < j ? inv_sc : 1.0f;
    cA[k] = make_float2(a.x * inv_sc, a.y * inv_sc);
    cB[k] = make_float2(c.x * f, c.y * f);
  }
  __syncthreads();
  const float sA = s.selfA[r], sB = s.selfB[r];
  const int64_t n2 = n >> 1;
  const float4* u4 = reinterpret_cast<const float4*>(u + r * rstride);
  float4* w4 = reinterpret_cast<float4*>(w + r * rstride);
  uint2* vj = Vh + ((int64_t)j * hstride + r * rstride) / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), bsum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < j; ++k) {
      const float4 v = h16_load2(Vh + ((int64_t)k * hstride + r * rstride) / 2, i);
      const float2 cb = cB[k];
      bsum.x = fmaf(v.x, cb.x, fmaf(-v.y, cb.y, bsum.x));
      bsum.y = fmaf(v.x, cb.y, fmaf(v.y, cb.x, bsum.y));
      bsum.z = fmaf(v.z, cb.x, fmaf(-v.w, cb.y, bsum.z));
      bsum.w = fmaf(v.z, cb.y, fmaf(v.w, cb.x, bsum.w));
      const float2 ca = cA[k];
      a.x = fmaf(v.x, ca.x, fmaf(-v.y, ca.y, a.x));
      a.y = fmaf(v.x, ca.y, fmaf(v.y, ca.x, a.y));
      a.z = fmaf(v.z, ca.x, fmaf(-v.w, ca.y, a.z));
      a.w = fmaf(v.z, ca.y, fmaf(v.w, ca.x, a.w));
    }
    const float4 uv = u4[i];
    {
      const float2 cb = cB[j];
      bsum.x = fmaf(uv.x, cb.x, fmaf(-uv.y, cb.y, bsum.x));
      bsum.y = fmaf(uv.x, cb.y, fmaf(uv.y, cb.x, bsum.y));
      bsum.z = fmaf(uv.z, cb.x, fmaf(-uv.w, cb.y, bsum.z));
      bsum.w = fmaf(uv.z, cb.y, fmaf(uv.w, cb.x, bsum.w));
    }
    const float4 wv = w4[i];
    w4[i] = make_float4(sB * wv.x - bsum.x, sB * wv.y - bsum.y, sB * wv.z - bsum.z, sB * wv.w - bsum.w);
    const float4 fin = j > 0 ? make_float4(sA * uv.x - a.x, sA * uv.y - a.y, sA * uv.z - a.z, sA * uv.w - a.w) : uv;
    vj[i] = h16_pack2(make_float4(sc * fin.x, sc * fin.y, sc * fin.z, sc * fin.w));
  }
}

// x[r] += sum_{k < ncols[r]} V_k coef[r][k] on the compressed basis (V_k = Vh_k / sc)
__global__ void __launch_bounds__(256)
xupdate16_kernel(const uint2* __restrict__ Vh, int64_t hstride, int nvec, const double2* __restrict__ coef, int maxv,
                 double2* __restrict__ x, int64_t n, int64_t rstride, const int* __restrict__ ncols, float inv_sc) {
  pdl_wait();
  const int r = blockIdx.y;
  const int nv = ncols ? min(nvec, ncols[r]) : nvec;
  extern __shared__ float2 xcs[];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    const double2 c = coef[r * maxv + k];
    xcs[k] = make_float2((float)c.x * inv_sc, (float)c.y * inv_sc);
  }
  __syncthreads();
  const int64_t n2 = n >> 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < nv; ++k) {
      const float4 v = h16_load2(Vh + ((int64_t)k * hstride + r * rstride) / 2, i);
      const float2 c = xcs[k];
      a.x = fmaf(v.x, c.x, fmaf(-v.y, c.y, a.x));
      a.y = fmaf(v.x, c.y, fmaf(v.y, c.x, a.y));
      a.z = fmaf(v.z, c.x, fmaf(-v.w, c.y, a.z));
      a.w = fmaf(v.z, c.y, fmaf(v.w, c.x, a.w));
    }
    double2* xo = x + r * rstride + 2 * i;
    double2 o0 = xo[0], o1 = xo[1];
    o0.x += a.x;
    o0.y += a.y;
    o1.x += a.z;
    o1.y += a.w;
    xo[0] = o0;
    xo[1] = o1;
  }
}

// back substitution y = H^{-1} g over the first ncols columns
__global__ void lsq_kernel(GState s, int R, int m, int maxv) {
  pdl_wait();
  // one block per RHS, column-oriented back substitution: y_k = b_k / H_kk, then
  // b_i -= H_ik y_k for i < k in parallel
  const int r = blockIdx.x;
  if (r >= R) return;
  extern __shared__ double2 lsb[];  // [maxv]
  __shared__ double2 yk_sh;
  const int nc = s.ncols[r];
  for (int k = threadIdx.x; k < maxv; k += blockDim.x) {
    s.y[r * maxv + k] = make_double2(0, 0);
    lsb[k] = k < nc ? s.g[r * maxv + k] : make_double2(0, 0);
  }
  __syncthreads();
  const double2* H = s.H + (int64_t)r * maxv * m;  // H[i * m + k]
  for (int k = nc - 1; k >= 0; --k) {
    if (threadIdx.x == 0) {
      const double2 d = H[(int64_t)k * m + k], acc = lsb[k];
      const double den = cabs2(d);
      const double2 yk = den > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                                 : make_double2(0, 0);
      s.y[r * maxv + k] = yk;
      yk_sh = yk;
    }
    __syncthreads();
    const double2 yk = yk_sh;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const double2 h = H[(int64_t)i * m + k];
      lsb[i].x -= h.x * yk.x - h.y * yk.y;
      lsb[i].y -= h.x * yk.y + h.y * yk.x;
    }
    __syncthreads();
  }
}

static unsigned grid_for(tmat_ctx* ctx, int64_t n) {
  int64_t g = cdiv(n, 256);
  int64_t cap = (int64_t)ctx->num_sms * 8;
  return (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// norms of R vectors (rstride apart) into nrm[r] (device)
template <typename VR>
static int vec_norms(tmat_ctx* ctx, const C<VR>* v, int64_t n, int64_t rstride, int R, double2* part, int nb,
                     double2* tmp, int maxv, double* nrm, const int* active) {
  if constexpr (sizeof(VR) == 4) {
    if ((n & 1) == 0) {
      const int nbn = (int)std::max<int64_t>(1, std::min<int64_t>(nb, cdiv(n / 2, 256 * 8)));
      TM_CUDA(ctx, launch_pdl(ctx->stream, norm32_kernel, dim3(nbn, R), dim3(256), 0, (const float2*)v, n, rstride,
                              part, maxv, active));
      TM_LAUNCHED(ctx);
      launch_reduce(ctx, part, nbn, 1, maxv, tmp, active, R);
      TM_LAUNCHED(ctx);
      TM_CUDA(ctx, launch_pdl(ctx->stream, norm_from_dots_kernel, dim3(1), dim3(32), 0, (const double2*)tmp, maxv, nrm,
                              R, active));
      TM_LAUNCHED(ctx);
      return TMAT_OK;
    }
  }
  if constexpr (sizeof(VR) == 8) {
    const int nbn = (int)std::max<int64_t>(1, std::min<int64_t>(nb, cdiv(n, 256 * 4)));
    TM_CUDA(ctx, launch_pdl(ctx->stream, norm64_kernel, dim3(nbn, R), dim3(256), 0, (const double2*)v, n, rstride, part,
                            maxv, active));
    TM_LAUNCHED(ctx);
    launch_reduce(ctx, part, nbn, 1, maxv, tmp, active, R);
    TM_LAUNCHED(ctx);
    TM_CUDA(ctx, launch_pdl(ctx->stream, norm_from_dots_kernel, dim3(1), dim3(32), 0, (const double2*)tmp, maxv, nrm, R,
                            active));
    TM_LAUNCHED(ctx);
    return TMAT_OK;
  }
  dots_kernel<VR><<<dim3(nb, R), RED_THREADS, 0, ctx->stream>>>(v, 0, 1, v, n, rstride, part, maxv, active);
  TM_LAUNCHED(ctx);
  launch_reduce(ctx, part, nb, 1, maxv, tmp, active, R);
  TM_LAUNCHED(ctx);
  norm_from_dots_kernel<<<1, 32, 0, ctx->stream>>>(tmp, maxv, nrm, R, active);
  TM_LAUNCHED(ctx);
  return TMAT_OK;
}

// Restarted GMRES on vectors of type VR. b (VR, internal layout, R x n) and the
// solution x (complex128, zero on entry) both device. Convergence when the true
// residual ||b - K x|| <= tol ||b|| per RHS.
// the mapped flag words (allocated once per context)
static int flags_mapped(tmat_ctx* ctx) {
  if (ctx->flag_host) return TMAT_OK;
  void* h = nullptr;
  TM_CUDA(ctx, cudaHostAlloc(&h, sizeof(int) * 2 * TMAT_MAX_RHS, cudaHostAllocMapped));
  std::memset(h, 0, sizeof(int) * 2 * TMAT_MAX_RHS);
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    return set_error(ctx, TMAT_ECUDA, "gmres: no device mapping of the flag words");
  }
  ctx->flag_host = (int*)h;
  ctx->flag_dev = (int*)d;
  return TMAT_OK;
}
// Waits until every RHS's step has published `tag`, then reports whether any is active.
// Bounded: past 10 s it synchronises the stream (which returns a kernel fault as an error)
// and gives up if the tags are still missing.
static int flags_wait(tmat_ctx* ctx, int R, int tag, bool* any) {
  const volatile int* f = ctx->flag_host;
  const auto t0 = std::chrono::steady_clock::now();
  for (uint64_t spin = 0;; ++spin) {
    bool all = true;
    for (int r = 0; r < R; ++r) all = all && f[TMAT_MAX_RHS + r] == tag;
    if (all) break;
    if ((spin & 1023) == 1023 && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10)) {
      TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      all = true;
      for (int r = 0; r < R; ++r) all = all && f[TMAT_MAX_RHS + r] == tag;
      if (!all) return set_error(ctx, TMAT_ECUDA, "gmres: convergence flags were not published");
      break;
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  *any = false;
  for (int r = 0; r < R; ++r) *any = *any || f[r] != 0;
  return TMAT_OK;
}

template <typename VR>
static int gmres_run(tmat_ctx* ctx, const Operator& A, int mode, const C<VR>* b, double2* x, int R, int64_t n,
                     const GmresParams& p, GmresStats* st) {
  const int m = p.restart;
  const int maxv = m + 1;
  const int64_t rs = n;  // RHS stride
  const int nb = (int)std::min<int64_t>(cdiv(n, RED_THREADS), (int64_t)ctx->num_sms * 4);
  // compressed basis (complex64 operator, loose tolerance): two fp32 slots (the pending
  // vector and the operator's output) and maxv fp16 slots for the final vectors
  const bool h16 = sizeof(VR) == 4 && p.compress_basis;
  C<VR>* V;
  TM_TRY(scratch(ctx, sizeof(VR) == 4 ? "g_V32" : "g_V64", sizeof(C<VR>) * (size_t)(h16 ? 2 : maxv) * R * n,
                 (void**)&V));
  uint2* Vh = nullptr;
  if (h16) TM_TRY(scratch(ctx, "g_V16", sizeof(uint2) / 2 * (size_t)maxv * R * n, (void**)&Vh));
  const float h16_sc = (float)std::sqrt((double)n), h16_inv = 1.0f / h16_sc;
  C<VR>* xv;  // x in operator precision (for the true residual)
  TM_TRY(scratch(ctx, sizeof(VR) == 4 ? "g_xv32" : "g_xv64", sizeof(C<VR>) * (size_t)R * n, (void**)&xv));
  double2* part;
  TM_TRY(scratch(ctx, "g_part", sizeof(double2) * (size_t)R * std::max(nb, D32_NBMAX) * maxv, (void**)&part));
  double2* part2 = nullptr;
  if (sizeof(VR) == 4)
    TM_TRY(scratch(ctx, "g_part2", sizeof(double2) * (size_t)R * D32_NBMAX * maxv, (void**)&part2));
  GState s;
  char* small;
  const size_t R_ = R;
  auto rup = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t sz = rup(sizeof(double2) * R_ * maxv) * 6 + rup(sizeof(double2) * R_ * maxv * m) * 2 +
              rup(sizeof(double2) * R_ * m) * 2 + rup(sizeof(double) * R_) * 4 + rup(sizeof(int) * R_) * 4 +
              rup(sizeof(float2) * R_ * maxv) * 2 + rup(sizeof(float) * R_) * 2;
  TM_TRY(scratch(ctx, "g_small", sz, (void**)&small));
  {
    char* q = small;
    auto take = [&](size_t bytes) { char* o = q; q += (bytes + 255) / 256 * 256; return (void*)o; };
    s.hA = (double2*)take(sizeof(double2) * R_ * maxv);
    s.hB = (double2*)take(sizeof(double2) * R_ * maxv);
    s.g = (double2*)take(sizeof(double2) * R_ * maxv);
    s.y = (double2*)take(sizeof(double2) * R_ * maxv);
    s.H = (double2*)take(sizeof(double2) * R_ * maxv * m);
    s.cs = (double2*)take(sizeof(double2) * R_ * m);
    s.sn = (double2*)take(sizeof(double2) * R_ * m);
    s.nrm = (double*)take(sizeof(double) * R_);
    s.tol_abs = (double*)take(sizeof(double) * R_);
    double* bnorm = (double*)take(sizeof(double) * R_);
    double* rnorm = (double*)take(sizeof(double) * R_);
    s.active = (int*)take(sizeof(int) * R_);
    s.ncols = (int*)take(sizeof(int) * R_);
    s.flags = (int*)take(sizeof(int) * R_);
    int* want = (int*)take(sizeof(int) * R_);
    s.Hu = (double2*)take(sizeof(double2) * R_ * maxv * m);
    s.cA = (float2*)take(sizeof(float2) * R_ * maxv);
    s.cB = (float2*)take(sizeof(float2) * R_ * maxv);
    s.selfA = (float*)take(sizeof(float) * R_);
    s.selfB = (float*)take(sizeof(float) * R_);
    if ((size_t)(q - small) > sz) return set_error(ctx, TMAT_ECUDA, "gmres: state layout overflow");
    TM_CUDA(ctx, cudaMemsetAsync(s.flags, 0, sizeof(int) * R_, ctx->stream));
    const unsigned g1 = grid_for(ctx, n);
    // ||b||
    TM_TRY(vec_norms<VR>(ctx, b, n, rs, R, part, nb, s.hA, maxv, bnorm, nullptr));
    double* pin = (double*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, bnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double hb[TMAT_MAX_RHS], tolabs[TMAT_MAX_RHS];
    int hwant[TMAT_MAX_RHS];
    for (int r = 0; r < R; ++r) {
      hb[r] = pin[r];
      tolabs[r] = 0.9 * p.tol * hb[r];
      hwant[r] = hb[r] > 0 ? 1 : 0;
      st->rel_res[r] = hb[r] > 0 ? 1.0 : 0.0;
    }
    TM_CUDA(ctx, cudaMemcpyAsync(s.tol_abs, tolabs, sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    TM_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(double2) * R_ * n, ctx->stream));
    // first residual = b
    TM_CUDA(ctx, cudaMemcpyAsync(rnorm, bnorm, sizeof(double) * R, cudaMemcpyDeviceToDevice, ctx->stream));
    const C<VR>* rsrc = b;
    // Convergence is read on the host every sync_every iterations: small systems are
    // bound by launch and synchronisation latency, and iterations past convergence are
    // skipped per RHS by the kernels (only the operator application still runs).
    const int sync_every = (int64_t)R * n < (1 << 20) ? 8 : 1;
    bool all_done = true;
    for (int r = 0; r < R; ++r) all_done = all_done && !hwant[r];
    st->converged = all_done;
    while (!all_done) {
      TM_CUDA(ctx, cudaMemcpyAsync(want, hwant, sizeof(int) * R, cudaMemcpyHostToDevice, ctx->stream));
      cycle_init_kernel<<<1, 32, 0, ctx->stream>>>(s, R, maxv, rnorm, want);
      TM_LAUNCHED(ctx);
      TM_CUDA(ctx, launch_pdl(ctx->stream, scale_kernel<VR, VR>, dim3(g1, R), dim3(256), 0, rsrc, V, n, rs,
                              (const double*)rnorm, 1, (const int*)nullptr));
      TM_LAUNCHED(ctx);
      int j = 0;
      if constexpr (sizeof(VR) == 4) {
        // delayed CGS2: the Hessenberg column of iteration j is finalised at iteration j + 1
        float2* V32 = reinterpret_cast<float2*>(V);
        const size_t step_bytes = dcgs2_step_smem(m, maxv);
        struct SkipReset {  // the sampling mark never outlives the loop (error returns included)
          tmat_ctx* c;
          ~SkipReset() { c->timing_skip = false; }
        } skip_reset{ctx};
        for (;; ++j) {
          const bool final_only = j == m || st->iterations >= p.max_iter;
          // sampled kernel timing: one iteration in timing_every is timed
          ctx->timing_skip = ctx->timing_every > 1 && (ctx->timing_iter++ % ctx->timing_every) != 0;
          float2* vj = V32 + (int64_t)(h16 ? (j & 1) : j) * R * n;
          float2* w = final_only ? nullptr : V32 + (int64_t)(h16 ? ((j + 1) & 1) : j + 1) * R * n;
          if (!final_only) {
            TM_TRY(op_apply(ctx, A, mode, vj, w, R));
            st->iterations++;
          }
          const int gh = (j + D16_VPW - 1) / D16_VPW;  // fp16 vector groups (compressed basis)
          Dots32Plan dp = dots32_plan(n, j + 1, ctx->num_sms, R);
          if (h16) {
            const Dots16Plan hp = dots16_plan(n, gh, ctx->num_sms, R);
            dp.ranges = hp.ranges;
            dp.blocks = hp.blocks;
          }
          float4* pf4 = reinterpret_cast<float4*>(part);  // double-float partials
          float4* pf4b = reinterpret_cast<float4*>(part2);
          cudaEvent_t ev_d = timing_begin(ctx);
          if (h16) {
            if (final_only)
              TM_CUDA(ctx, launch_pdl(ctx->stream, dots16_kernel<false>, dim3(dp.blocks, R), dim3(256), 0,
                                      (const uint2*)Vh, (int64_t)R * n, j, (const float2*)vj, n, rs, pf4, maxv, gh,
                                      dp.ranges, (const int*)s.active, h16_inv, (const float2*)nullptr,
                                      (float4*)nullptr));
            else
              TM_CUDA(ctx, launch_pdl(ctx->stream, dots16_kernel<true>, dim3(dp.blocks, R), dim3(256), 0,
                                      (const uint2*)Vh, (int64_t)R * n, j, (const float2*)vj, n, rs, pf4, maxv, gh,
                                      dp.ranges, (const int*)s.active, h16_inv, (const float2*)w, pf4b));
          } else if (final_only) {
            TM_CUDA(ctx, launch_pdl(ctx->stream, dots32_kernel<false>, dim3(dp.blocks, R), dim3(256), 0,
                                    (const float2*)V32, (int64_t)R * n, j + 1, (const float2*)vj, n, rs, pf4, maxv,
                                    dp.groups, dp.ranges, (const int*)s.active, (const float2*)nullptr,
                                    (float4*)nullptr));
          } else {
            TM_CUDA(ctx, launch_pdl(ctx->stream, dots32_kernel<true>, dim3(dp.blocks, R), dim3(256), 0,
                                    (const float2*)V32, (int64_t)R * n, j + 1, (const float2*)vj, n, rs, pf4, maxv,
                                    dp.groups, dp.ranges, (const int*)s.active, (const float2*)w, pf4b));
          }
          TM_LAUNCHED(ctx);
          // reads the j + 1 basis slots (the pending vector is slot j) and w
          timing_end(ctx, "arnoldi_dots32", ev_d,
                     h16 ? 4.0 * R * n * j + 8.0 * R * n * (1 + (final_only ? 0 : 1))
                         : 8.0 * R * n * (j + 1 + (final_only ? 0 : 1)));
          // the dot sums (ranges / 8 partials each), column j-1 final, its rotation, column j
          // and the update coefficients. The step publishes its convergence flags to mapped
          // host memory (with a tag) and the host reads them while the update pass runs (it
          // skips every RHS that has converged): no copy or event between the two kernels, so
          // the update launch overlaps the step, and the device does not idle through the
          // host's check before the next operator launch.
          const bool check = j >= 1 && !final_only && j % sync_every == 0;
          int tag = 0;
          if (check) {
            TM_TRY(flags_mapped(ctx));
            if (++ctx->flag_tag <= 0) ctx->flag_tag = 1;
            tag = ctx->flag_tag;
          }
          {
            // the partials go through shared memory with everything else when they fit
            const int RB = dp.ranges / 8, S = final_only ? j + 1 : 2 * (j + 1);
            const size_t pbytes = sizeof(float4) * (size_t)S * RB;
            const int stage_p = step_bytes + pbytes <= 200 * 1024 ? 1 : 0;
            const size_t sm = step_bytes + (stage_p ? pbytes : 0);
            if (sm > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)dcgs2_step_kernel, sm));
            TM_CUDA(ctx, launch_pdl(ctx->stream, dcgs2_step_kernel, dim3(R), dim3(DCGS2_THREADS), sm, s,
                                    (const float4*)pf4, (const float4*)pf4b, RB, j, m, maxv, R, final_only ? 1 : 0,
                                    stage_p, ctx->flag_dev, tag));
          }
          TM_LAUNCHED(ctx);
          if (final_only) break;
          cudaEvent_t ev_u = timing_begin(ctx);
          if (h16) {
            const unsigned gu = (unsigned)std::min<int64_t>(cdiv(n / 2, 256), (int64_t)ctx->num_sms * 16);
            TM_CUDA(ctx, launch_pdl(ctx->stream, dcgs2_update16_kernel, dim3(gu, R), dim3(256),
                                    sizeof(float2) * (2 * (size_t)j + 2), Vh, (int64_t)R * n, j, s, maxv,
                                    (const float2*)vj, w, n, rs, h16_sc));
          } else {
            TM_CUDA(ctx, launch_pdl(ctx->stream, dcgs2_update_kernel, dim3(g1, R), dim3(256),
                                    sizeof(float2) * (2 * (size_t)j + 2), V32, (int64_t)R * n, j, s, maxv, w, n, rs));
          }
          TM_LAUNCHED(ctx);
          // reads slots 0..j and w, writes slot j (j > 0) and w (compressed: fp16 slots 0..j-1,
          // the fp32 pending vector and w; writes fp16 slot j and w)
          timing_end(ctx, "arnoldi_update32", ev_u,
                     h16 ? 4.0 * R * n * (j + 1) + 8.0 * R * n * 3 : 8.0 * R * n * (j + 2 + (j > 0 ? 1 : 0) + 1));
          if (check) {
            bool any = false;
            TM_TRY(flags_wait(ctx, R, tag, &any));
            if (!any) break;
          }
        }
        // columns 0..j-1 are final
      } else
      for (; j < m && st->iterations < p.max_iter; ++j) {
        C<VR>* vj = V + (int64_t)j * R * n;
        C<VR>* w = V + (int64_t)(j + 1) * R * n;
        TM_TRY(op_apply(ctx, A, mode, vj, w, R));
        for (int pass = 0; pass < 2; ++pass) {
          double2* hc = pass == 0 ? s.hA : s.hB;
          // (complex128 vectors: complex64 ones take the delayed CGS2 above)
          dots_kernel<VR><<<dim3(nb, R), RED_THREADS, 0, ctx->stream>>>(V, (int64_t)R * n, j + 1, w, n, rs, part, maxv,
                                                                         s.active);
          TM_LAUNCHED(ctx);
          launch_reduce(ctx, part, nb, j + 1, maxv, hc, s.active, R);
          TM_LAUNCHED(ctx);
          update_kernel<VR, VR><<<dim3(g1, R), 256, 0, ctx->stream>>>(V, (int64_t)R * n, j + 1, hc, maxv, -1.0, w, n, rs,
                                                                      s.active, nullptr);
          TM_LAUNCHED(ctx);
        }
        TM_TRY(vec_norms<VR>(ctx, w, n, rs, R, part, nb, s.y, maxv, s.nrm, s.active));
        scale_kernel<VR, VR><<<dim3(g1, R), 256, 0, ctx->stream>>>(w, w, n, rs, s.nrm, 1, s.active);
        TM_LAUNCHED(ctx);
        const size_t gsm_bytes = sizeof(double2) * (2 * (size_t)m + maxv);
        if (gsm_bytes > 48 * 1024)
          TM_TRY(set_smem_limit(ctx, (const void*)givens_kernel, gsm_bytes));
        givens_kernel<<<R, 64, gsm_bytes, ctx->stream>>>(s, R, j, m, maxv);
        TM_LAUNCHED(ctx);
        st->iterations++;
        if ((j + 1) % sync_every != 0 && j + 1 < m && st->iterations < p.max_iter) continue;
        int* ipin = (int*)ctx->pinned;
        TM_CUDA(ctx, cudaMemcpyAsync(ipin, s.active, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->stream));
        TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || ipin[r];
        if (!any) {
          ++j;
          break;
        }
      }
      // x += V y over the columns each RHS built in this cycle (ncols[r] <= j)
      TM_CUDA(ctx, launch_pdl(ctx->stream, lsq_kernel, dim3(R), dim3(128), sizeof(double2) * maxv, s, R, m, maxv));
      TM_LAUNCHED(ctx);
      if constexpr (sizeof(VR) == 4) {
        if (h16)  // the update pass's grid (16 blocks per SM per RHS)
          TM_CUDA(ctx, launch_pdl(ctx->stream, xupdate16_kernel,
                                  dim3((unsigned)std::min<int64_t>(cdiv(n / 2, 256), (int64_t)ctx->num_sms * 16), R),
                                  dim3(256), sizeof(float2) * std::max(j, 1), (const uint2*)Vh, (int64_t)R * n, j,
                                  (const double2*)s.y, maxv, x, n, rs, (const int*)s.ncols, h16_inv));
        else
          xupdate32_kernel<<<dim3(g1, R), 256, sizeof(float2) * std::max(j, 1), ctx->stream>>>(
              reinterpret_cast<const float2*>(V), (int64_t)R * n, j, s.y, maxv, x, n, rs, s.ncols);
      } else {
        update_kernel<VR, double><<<dim3(g1, R), 256, 0, ctx->stream>>>(V, (int64_t)R * n, j, s.y, maxv, 1.0, x, n, rs,
                                                                        nullptr, s.ncols);
      }
      TM_LAUNCHED(ctx);
      // true residual r = b - K x (in the operator precision)
      convert_kernel<double, VR><<<g1, 256, 0, ctx->stream>>>(x, xv, (int64_t)R * n);
      TM_LAUNCHED(ctx);
      C<VR>* w = V + (int64_t)R * n;  // V[1] as scratch, V[0] receives the new start vector
      TM_TRY(op_apply(ctx, A, mode, xv, w, R));
      residual_kernel<VR, VR><<<g1, 256, 0, ctx->stream>>>(b, w, w, (int64_t)R * n);
      TM_LAUNCHED(ctx);
      TM_TRY(vec_norms<VR>(ctx, w, n, rs, R, part, nb, s.y, maxv, rnorm, nullptr));
      TM_CUDA(ctx, cudaMemcpyAsync(pin, rnorm, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
      int* fl = (int*)(pin + TMAT_MAX_RHS);
      TM_CUDA(ctx, cudaMemcpyAsync(fl, s.flags, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->stream));
      TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      all_done = true;
      bool conv = true;
      for (int r = 0; r < R; ++r) {
        double rel = hb[r] > 0 ? pin[r] / hb[r] : 0.0;
        st->rel_res[r] = rel;
        bool ok = hb[r] == 0 || rel <= p.tol;
        if (fl[r] & 1) st->breakdown = true;
        hwant[r] = (!ok && !(fl[r] & 1)) ? 1 : 0;
        conv = conv && ok;
        all_done = all_done && !hwant[r];
      }
      st->converged = conv;
      if (st->iterations >= p.max_iter) break;
      rsrc = w;
      // the new start vector goes to V[0] = w / ||w|| (scale reads w = V[1], writes V[0])
    }
  }
  return TMAT_OK;
}

static unsigned g_for(tmat_ctx* ctx, int64_t n) { return grid_for(ctx, n); }

// Relative error of a complex64 residual b - K x (x rounded to complex64, K applied in
// fp32/3xTF32 arithmetic), as a fraction of ||b||.
constexpr double kFastResidualFloor = 1e-7;

int solve_system(tmat_ctx* ctx, const Operator& A64, const Operator* A32, int mode, const double2* b, double2* x, int R,
                 const SolveParams& p, SolveStats* st, const Operator* res64) {
  const Operator& Ares = res64 ? *res64 : A64;
  const int64_t n = A64.N() * num_coeffs(A64.nmax());
  GmresParams gp;
  gp.restart = std::max(2, std::min(p.restart, 1024));
  gp.max_iter = p.max_iter;
  if (p.precision == TMAT_PREC_FP64 || !A32) {
    gp.tol = p.tol;
    GmresStats gs;
    TM_TRY(gmres_run<double>(ctx, A64, mode, b, x, R, n, gp, &gs));
    st->iterations = gs.iterations;
    st->converged = gs.converged;
    for (int r = 0; r < R; ++r) st->rel_res[r] = gs.rel_res[r];
    if (gs.breakdown && !gs.converged) return set_error(ctx, TMAT_EBREAKDOWN, "GMRES produced a non-finite value");
    return TMAT_OK;
  }
  // mixed: iterative refinement with an fp64 residual around fp32 inner GMRES
  double2 *r64, *d64, *y64;
  float2* r32;
  TM_TRY(scratch(ctx, "mx_r64", sizeof(double2) * R * n, (void**)&r64));
  TM_TRY(scratch(ctx, "mx_d64", sizeof(double2) * R * n, (void**)&d64));
  TM_TRY(scratch(ctx, "mx_y64", sizeof(double2) * R * n, (void**)&y64));
  TM_TRY(scratch(ctx, "mx_r32", sizeof(float2) * R * n, (void**)&r32));
  float2* y32;
  TM_TRY(scratch(ctx, "mx_y32", sizeof(float2) * R * n, (void**)&y32));
  const int nb = (int)std::min<int64_t>(cdiv(n, RED_THREADS), (int64_t)ctx->num_sms * 4);
  double2 *part, *tmp;
  double *rn, *bn, *alpha;
  TM_TRY(scratch(ctx, "mx_part", sizeof(double2) * R * nb, (void**)&part));
  TM_TRY(scratch(ctx, "mx_tmp", sizeof(double2) * R + sizeof(double) * 3 * R + 1024, (void**)&tmp));
  rn = (double*)(tmp + R);
  bn = rn + R;
  alpha = bn + R;
  const unsigned g1 = g_for(ctx, n);
  TM_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(double2) * R * n, ctx->stream));
  TM_TRY(vec_norms<double>(ctx, b, n, n, R, part, nb, tmp, 1, bn, nullptr));
  TM_CUDA(ctx, cudaMemcpyAsync(r64, b, sizeof(double2) * R * n, cudaMemcpyDeviceToDevice, ctx->stream));
  double* pin = (double*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, bn, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double hb[TMAT_MAX_RHS], hr[TMAT_MAX_RHS];
  for (int r = 0; r < R; ++r) hb[r] = hr[r] = pin[r];
  st->iterations = 0;
  st->refinements = 0;
  for (int outer = 0; outer < 50; ++outer) {
    bool done = true;
    double halpha[TMAT_MAX_RHS];
    for (int r = 0; r < R; ++r) {
      double rel = hb[r] > 0 ? hr[r] / hb[r] : 0.0;
      st->rel_res[r] = rel;
      bool ok = hb[r] == 0 || rel <= p.tol;
      done = done && ok;
      halpha[r] = ok ? 0.0 : hr[r];  // scale of the correction; 0 freezes a converged RHS
    }
    st->converged = done;
    if (done || st->iterations >= p.max_iter) break;
    // r32 = r64 / ||r|| (zero for converged RHS)
    TM_CUDA(ctx, cudaMemcpyAsync(alpha, halpha, sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    scale_kernel<double, float><<<dim3(g1, R), 256, 0, ctx->stream>>>(r64, r32, n, n, alpha, 1, nullptr);
    TM_LAUNCHED(ctx);
    GmresParams ip = gp;
    // Do not oversolve: a correction that reduces ||r|| by rho leaves ~rho ||r||, so when
    // the remaining factor to the tolerance is milder than inner_tol the inner solve stops
    // at half of it (the most demanding of the RHS still refined decides).
    double need = 1.0;
    for (int r = 0; r < R; ++r)
      if (halpha[r] != 0.0 && hr[r] > 0) need = std::min(need, 0.5 * p.tol * hb[r] / hr[r]);
    ip.tol = std::max(p.inner_tol, need);
    ip.max_iter = p.max_iter - st->iterations;
    // loose inner solves keep their final basis vectors in fp16 (the fp64-accurate outer
    // residual closes every step); tight ones in fp32
    ip.compress_basis = ctx->compress_basis && ip.tol >= 1e-2;
    GmresStats gs;
    TM_TRY(gmres_run<float>(ctx, *A32, mode, r32, d64, R, n, ip, &gs));
    st->iterations += gs.iterations;
    // x += ||r|| d
    TM_CUDA(ctx, launch_pdl(ctx->stream, axpy_scaled_kernel, dim3(g1, R), dim3(256), 0, x, (const double2*)d64,
                            (const double*)alpha, n, n));
    TM_LAUNCHED(ctx);
    // Fast check first while the residual is large: r = b - K x with K applied in
    // complex64 to x rounded to complex64 has an absolute error of about
    // kFastResidualFloor ||b||, so it stands in for the fp64 residual only while it is far
    // above that floor and above the tolerance (the next correction cannot push the true
    // residual below its error), and only while it keeps falling (no stagnation on the
    // error of the complex64 product); near the tolerance the fp64 residual decides, and
    // only the fp64 residual can declare convergence. It is tried when this step is
    // expected to leave the residual far above that threshold.
    const double fast_thr = std::max(10.0 * p.tol, 100.0 * kFastResidualFloor);
    bool try_fast = true;
    for (int r = 0; r < R; ++r)
      if (hb[r] != 0 && halpha[r] != 0.0) try_fast = try_fast && ip.tol * hr[r] > 10.0 * fast_thr * hb[r];
    if (try_fast) {
      TM_CUDA(ctx, launch_pdl(ctx->stream, convert_kernel<double, float>, dim3(g1), dim3(256), 0, (const double2*)x,
                              r32, (int64_t)R * n));
      TM_LAUNCHED(ctx);
      TM_TRY(op_apply(ctx, *A32, mode, r32, y32, R));
      TM_CUDA(ctx, launch_pdl(ctx->stream, residual_kernel<double, float>, dim3(g1), dim3(256), 0, (const double2*)b,
                              (const float2*)y32, r64, (int64_t)R * n));
      TM_LAUNCHED(ctx);
      TM_TRY(vec_norms<double>(ctx, r64, n, n, R, part, nb, tmp, 1, rn, nullptr));
      TM_CUDA(ctx, cudaMemcpyAsync(pin, rn, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
      TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      bool far = true;
      for (int r = 0; r < R; ++r) {
        if (!std::isfinite(pin[r])) return set_error(ctx, TMAT_EBREAKDOWN, "refinement residual is not finite");
        if (hb[r] == 0 || halpha[r] == 0.0) continue;  // converged or zero RHS: frozen
        far = far && pin[r] > fast_thr * hb[r] && pin[r] < 0.5 * hr[r];
      }
      if (far) {
        for (int r = 0; r < R; ++r)
          if (hb[r] != 0 && halpha[r] != 0.0) hr[r] = pin[r];
        st->refinements++;
        continue;
      }
    }
    // r = b - K x, fp64-accurate
    TM_TRY(op_apply(ctx, Ares, mode, x, y64, R));
    TM_CUDA(ctx, launch_pdl(ctx->stream, residual_kernel<double, double>, dim3(g1), dim3(256), 0, (const double2*)b,
                            (const double2*)y64, r64, (int64_t)R * n));
    TM_LAUNCHED(ctx);
    TM_TRY(vec_norms<double>(ctx, r64, n, n, R, part, nb, tmp, 1, rn, nullptr));
    TM_CUDA(ctx, cudaMemcpyAsync(pin, rn, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < R; ++r) {
      if (!std::isfinite(pin[r])) return set_error(ctx, TMAT_EBREAKDOWN, "refinement residual is not finite");
      hr[r] = pin[r];
    }
    st->refinements++;
  }
  for (int r = 0; r < R; ++r) st->rel_res[r] = hb[r] > 0 ? hr[r] / hb[r] : 0.0;
  return TMAT_OK;
}

}  // namespace tmat
