// Lattice operator apply with fp64-class accuracy on the tcgen05 tensor cores.
//
// The refinement residual of the mixed solver (and the TMAT_PREC_FP64_TC precision)
// needs A x to about 1e-12 relative; the fp64 CUDA-core kernel gets there at the
// FP64 pipe's rate. Here the product runs as exact integer arithmetic on the bf16
// tensor cores (the splitting idea of Ozaki et al., "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)):
//
//   x[k] / d_k (per RHS and class) = sigma 2^-8 sum_i X'_i,  X'_i = X_i 2^-8i,
//   W[n][k] d_k (per class, column n) = tau_n 2^-8 sum_j W'_j,  W'_j = W_j 2^-8j,
//
// with d_k, sigma, tau_n powers of two, |X_0|, |W_0| <= 256 and X_i, W_j integers
// (OZ_S = 6 slices of 8 bits, every slice exact in bf16). The per-coefficient scale
// d_k (the largest |x[k]| over positions and RHS) matches the operand scales along
// the contraction: the sources of the solve carry the T-matrix's decay over the
// multipole order while the blocks grow with it, and a single scale per row would
// lose that many bits. d depends on x, so the W slices are cut per apply (K blocks,
// a few tens of MB). A product X'_i W'_j is an integer times 2^-8(i+j), so
// the products of one level l = i + j summed over k and over a group of offsets are
// exact in an fp32 accumulator as long as the sum of their magnitudes stays below
// 2^24; the groups are cut on the device from bounds of the W slices (a single
// offset always fits). Levels 0, 1 and 2 get exact accumulators, levels 3..OZ_LMAX share a
// fourth one (its fp32 rounding is 2^-24 of a 2^-24-scaled quantity). Every group
// is drained into double-float (fp32 pair) registers with error-free additions,
// and the epilogue forms y in fp64. Dropped levels and slices cost ~2^-48 of the
// operand scales.
//
// Layout and roles follow the window-view kernel (lattice_tc2.cu): sources split
// once per apply into zero-padded k-chunk planes (now one set per slice), one
// window per dy, shifted descriptors per dx; the W slices of one offset stream in
// by cp.async.bulk; two ping-pong sets of four TMEM accumulators; all waits bounded.
#include <cstdint>

#include "dev.cuh"
#include "solver.h"

namespace tmat {

constexpr int OZ_THREADS = 256;
constexpr int OZ_S = 6;      // slices per operand
constexpr int OZ_LMAX = 5;   // highest level kept
constexpr int OZ_NACC = 4;   // accumulators: levels 0, 1, 2 exact; 3..OZ_LMAX
constexpr int OZ_WSTAGES = 2;
constexpr int OZ_ACC_STRIDE = 256;  // TMEM columns between the two accumulator sets
constexpr uint32_t OZ_WAIT_LIMIT = 1u << 22;
constexpr double OZ_GROUP_LIMIT = 16777216.0;  // 2^24

template <int NMAX> struct OzShape {
  static constexpr int L = NMAX * (NMAX + 2);
  static constexpr int LP2 = (L + 7) / 8 * 8;
  static constexpr int KR = 2 * LP2;               // real K (and N) extent
  static constexpr int KC = KR / 8;                // 16-byte chunks of 8 bf16 along K
  static constexpr int W_SLICE = KR * KR * 2;      // bytes of one W slice
  static constexpr int W_STAGE = OZ_S * W_SLICE;   // bytes of one offset's W slices
  static_assert(OZ_NACC * KR <= OZ_ACC_STRIDE, "accumulators do not fit");
};

// bf16 bit pattern of a float that is exactly representable in bf16
__host__ __device__ __forceinline__ uint32_t bf16_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f) >> 16;
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u >> 16;
#endif
}

// byte offset of element (row, k) in the no-swizzle K-major core layout of a
// bf16 operand with KC chunks along K
__host__ __device__ __forceinline__ int oz_core_off(int row, int k, int KC) {
  return (((row >> 3) * KC + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// Real-ified block entry W[n][k] of offset o, class c: forward blocks
// G_o[u][u'] = BT[o][c][u'][u]; adjoint G[u][u'] = BT[neg(o)][c][u][u'].
template <int L>
__device__ __forceinline__ double oz_w_entry(const double2* __restrict__ BT, int LP, const int* __restrict__ neg, int o,
                                             int c, int n, int k, int mode) {
  const int u = n >> 1, t = n & 1, up = k >> 1, s = k & 1;
  if (u >= L || up >= L) return 0.0;
  const double2 z = mode == 0 ? BT[(((size_t)o * 2 + c) * L + up) * LP + u] : BT[(((size_t)neg[o] * 2 + c) * L + u) * LP + up];
  return (t == s) ? z.x : (t == 1 ? z.y : -z.y);
}

// exponent e with |v| <= 2^e for the largest |v| (0 for v = 0)
__host__ __device__ __forceinline__ int oz_scale_exp(double m) {
  if (!(m > 0)) return 0;
  int e;
  frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// colexp[c][n] = scale exponent of column n of W[n][k] d_k over all offsets and k
template <int NMAX>
__global__ void oz_wscale_kernel(const double2* __restrict__ BT, int LP, const int* __restrict__ neg, int K, int mode,
                                 const int* __restrict__ dexp, int* __restrict__ colexp) {
  using S = OzShape<NMAX>;
  const int c = blockIdx.x / S::KR, n = blockIdx.x % S::KR;
  double m = 0.0;
  for (int e = threadIdx.x; e < K * S::KR; e += blockDim.x) {
    const int o = e / S::KR, k = e % S::KR;
    const int u = k >> 1;
    const double w = oz_w_entry<S::L>(BT, LP, neg, o, c, n, k, mode);
    m = fmax(m, fabs(u < S::L ? ldexp(w, dexp[c * S::L + u]) : 0.0));
  }
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) colexp[c * S::KR + n] = oz_scale_exp(red[0]);
}

// W slices of every (offset, class) in the core layout, W[((o*2 + c)*OZ_S + j)][KR x KR]
// bf16, and the per-level magnitude bounds bound[(o*2 + c)*3 + l] = max_n sum_k
// sum_{i+j=l} Xmax_i |W_j[n][k]| (integers; Xmax_0 = 256, Xmax_i = 128).
template <int NMAX>
__global__ void oz_wtables_kernel(const double2* __restrict__ BT, int LP, const int* __restrict__ neg, int K, int mode,
                                  const int* __restrict__ dexp, const int* __restrict__ colexp,
                                  unsigned char* __restrict__ W, double* __restrict__ bound) {
  using S = OzShape<NMAX>;
  const int oc = blockIdx.x;
  if (oc >= 2 * K) return;
  const int o = oc >> 1, c = oc & 1;
  __shared__ unsigned long long colsum[3][S::KR];
  for (int e = threadIdx.x; e < 3 * S::KR; e += blockDim.x) (&colsum[0][0])[e] = 0ull;
  __syncthreads();
  unsigned char* Wo = W + (size_t)oc * S::W_STAGE;
  for (int e = threadIdx.x; e < S::KR * S::KR; e += blockDim.x) {
    const int n = e / S::KR, k = e % S::KR;
    const int u = k >> 1;
    const double w = u < S::L ? ldexp(oz_w_entry<S::L>(BT, LP, neg, o, c, n, k, mode),
                                      dexp[c * S::L + u] - colexp[c * S::KR + n])
                              : 0.0;
    double t = w * 256.0;
    int dig[OZ_S];
#pragma unroll
    for (int j = 0; j < OZ_S; ++j) {
      const double d = rint(t);
      dig[j] = (int)d;
      t = (t - d) * 256.0;
    }
    const int off = oz_core_off(n, k, S::KC);
#pragma unroll
    for (int j = 0; j < OZ_S; ++j) {
      const float f = ldexpf((float)dig[j], -8 * j);
      *reinterpret_cast<uint16_t*>(Wo + (size_t)j * S::W_SLICE + off) = (uint16_t)bf16_bits(f);
    }
    const unsigned long long a0 = (unsigned long long)abs(dig[0]), a1 = (unsigned long long)abs(dig[1]),
                             a2 = (unsigned long long)abs(dig[2]);
    atomicAdd(&colsum[0][n], 256ull * a0);
    atomicAdd(&colsum[1][n], 256ull * a1 + 128ull * a0);
    atomicAdd(&colsum[2][n], 256ull * a2 + 128ull * a1 + 128ull * a0);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long m = 0;
    for (int n = 0; n < S::KR; ++n) m = colsum[threadIdx.x][n] > m ? colsum[threadIdx.x][n] : m;
    bound[(size_t)oc * 3 + threadIdx.x] = (double)m;
  }
}

// Scales of the sources x~ (x, or T x for the adjoint), by two reductions over
// positions (non-negative doubles order like their bit patterns):
//   dmax[c][u] = max over RHS, positions of |Re|, |Im| of x~[u] (class c), then
//   smax[r][c] = max over positions and u of |x~_r[u]| / d_u with d_u = 2^dexp[c][u].
template <int NMAX, int MODE, bool SECOND>
__global__ void oz_xscale_kernel(const double2* __restrict__ x, const double2* __restrict__ T, int64_t N, int R,
                                 const int* __restrict__ dexp, unsigned long long* __restrict__ out) {
  constexpr int L = NMAX * (NMAX + 2), P = 2 * L;
  constexpr int PER = 256 / P;  // sites per block step
  __shared__ unsigned long long red[2 * TMAT_MAX_RHS > P ? 2 * TMAT_MAX_RHS : P];
  for (int e = threadIdx.x; e < (int)(sizeof(red) / sizeof(red[0])); e += blockDim.x) red[e] = 0ull;
  __syncthreads();
  if (threadIdx.x < PER * P) {
    const int u = threadIdx.x % P, s0 = threadIdx.x / P;
    const int c = u >= L ? 1 : 0, uc = u - c * L;
    const double dinv = SECOND ? ldexp(1.0, -dexp[c * L + uc]) : 1.0;
    double m[TMAT_MAX_RHS];
    for (int r = 0; r < R; ++r) m[r] = 0.0;
    for (int64_t site = (int64_t)blockIdx.x * PER + s0; site < N; site += (int64_t)gridDim.x * PER) {
      const double2 t = MODE == 1 ? T[site * P + u] : make_double2(1.0, 0.0);
      for (int r = 0; r < R; ++r) {
        double2 v = x[((int64_t)r * N + site) * P + u];
        if (MODE == 1) v = cmul(t, v);
        m[r] = fmax(m[r], fmax(fabs(v.x), fabs(v.y)) * dinv);
      }
    }
    if (SECOND) {
      for (int r = 0; r < R; ++r)
        if (m[r] > 0) atomicMax(&red[r * 2 + c], (unsigned long long)__double_as_longlong(m[r]));
    } else {
      double mm = 0.0;
      for (int r = 0; r < R; ++r) mm = fmax(mm, m[r]);
      if (mm > 0) atomicMax(&red[u], (unsigned long long)__double_as_longlong(mm));
    }
  }
  __syncthreads();
  const int nout = SECOND ? 2 * R : P;
  for (int e = threadIdx.x; e < nout; e += blockDim.x)
    if (red[e]) atomicMax(&out[e], red[e]);
}

// dexp[c*L + u] = scale exponent of dmax (P values in class-split order = [c][u])
__global__ void oz_dexp_kernel(const unsigned long long* __restrict__ dmax, int P, int* __restrict__ dexp) {
  for (int e = threadIdx.x; e < P; e += blockDim.x) dexp[e] = oz_scale_exp(__longlong_as_double((long long)dmax[e]));
}

// Groups of consecutive offsets whose level sums stay below 2^24 in both classes:
// group_end[g] = one past the last offset of group g, *ngroups = count.
__global__ void oz_groups_kernel(const double* __restrict__ bound, int K, int* __restrict__ group_end,
                                 int* __restrict__ ngroups) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc[3] = {0.0, 0.0, 0.0};
  int g = 0;
  for (int o = 0; o < K; ++o) {
    double b[3];
    bool fits = true;
    for (int l = 0; l < 3; ++l) {
      b[l] = fmax(bound[((size_t)o * 2 + 0) * 3 + l], bound[((size_t)o * 2 + 1) * 3 + l]);
      fits = fits && acc[l] + b[l] < OZ_GROUP_LIMIT;
    }
    if (!fits && o > 0) {
      group_end[g++] = o;
      for (int l = 0; l < 3; ++l) acc[l] = 0.0;
    }
    for (int l = 0; l < 3; ++l) acc[l] += b[l];
  }
  group_end[g++] = K;
  *ngroups = g;
}

// Source slices: Xs[plane][PL] 16-byte records (8 bf16 along K), plane =
// ((r*2 + c)*OZ_S + i)*KC + kc, stored index = padded position + CX; zeros off the lattice.
template <int NMAX, int MODE>
__global__ void oz_split_kernel(const double2* __restrict__ x, const double2* __restrict__ T, int nx, int ny, int CX,
                                int CY, int64_t PL, int R, int64_t rstride, const int* __restrict__ dexp,
                                const unsigned long long* __restrict__ smax, uint4* __restrict__ Xs) {
  using S = OzShape<NMAX>;
  constexpr int L = S::L, P = 2 * L, KC = S::KC;
  const int W = nx + 2 * CX;
  const int64_t total = (int64_t)R * 2 * KC * PL;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = t % PL;
    const int64_t rest = t / PL;
    const int kc = (int)(rest % KC);
    const int c = (int)((rest / KC) % 2);
    const int r = (int)(rest / (2 * KC));
    const int ex = oz_scale_exp(__longlong_as_double((long long)smax[r * 2 + c]));
    double v[8];
    int vexp[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = 0.0;
      const int u = 4 * kc + (e >> 1);
      vexp[e] = u < L ? dexp[c * L + u] : 0;
    }
    const int64_t pp = idx - CX;
    if (pp >= 0) {
      const int64_t iy = pp / W - CY, ix = pp % W - CX;
      if (iy >= 0 && iy < ny && ix >= 0 && ix < nx) {
        const int64_t site = iy * nx + ix;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int u = 4 * kc + h;
          if (u < L) {
            double2 z = x[r * rstride + site * P + c * L + u];
            if (MODE == 1) z = cmul(T[site * P + c * L + u], z);
            v[2 * h] = z.x;
            v[2 * h + 1] = z.y;
          }
        }
      }
    }
    uint32_t word[OZ_S][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      double tt = ldexp(v[e], 8 - ex - vexp[e]);  // x / (d sigma) * 256, |.| <= 256
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        const double d = rint(tt);
        tt = (tt - d) * 256.0;
        const uint32_t b = bf16_bits(ldexpf((float)d, -8 * i));
        if (e & 1)
          word[i][e >> 1] |= b << 16;
        else
          word[i][e >> 1] = b;
      }
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      const int64_t plane = ((int64_t)(r * 2 + c) * OZ_S + i) * KC + kc;
      Xs[plane * PL + idx] = make_uint4(word[i][0], word[i][1], word[i][2], word[i][3]);
    }
  }
}

__device__ __forceinline__ uint32_t oz_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < OZ_WAIT_LIMIT; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// error-free a + b = s + e (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int NMAX, int MODE>
__global__ void __launch_bounds__(OZ_THREADS, 1)
lattice_oz_kernel(const int2* __restrict__ off, int K, const int* __restrict__ dy_start, int ndy,
                  const int* __restrict__ group_end, const int* __restrict__ ngroups_dev, int CX, int CY, int nx,
                  int ny, int64_t PL, const uint4* __restrict__ Xs, const unsigned char* __restrict__ Wt,
                  const int* __restrict__ colexp, const unsigned long long* __restrict__ smax,
                  const double2* __restrict__ T,
                  const double2* __restrict__ x, double2* __restrict__ y, int64_t rstride, int* __restrict__ err) {
  using S = OzShape<NMAX>;
  constexpr int L = S::L, P = 2 * L, KR = S::KR, KC = S::KC;
  const int W = nx + 2 * CX;
  const int WL = 128 + 2 * CX;
  const int tile = blockIdx.x, c = blockIdx.y, r = blockIdx.z;
  const int64_t p0 = (int64_t)CY * W + (int64_t)tile * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sWin = smem;                                          // [OZ_S][KC][WL] x 16 B
  unsigned char* sW = smem + (size_t)OZ_S * KC * WL * 16;              // W ring
  __shared__ uint64_t bars[2 * OZ_WSTAGES + 6];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  constexpr int WFULL = 0, WEMPTY = OZ_WSTAGES, WINFULL = 2 * OZ_WSTAGES, WINEMPTY = WINFULL + 1;
  constexpr int ACCFULL = WINEMPTY + 1, ACCEMPTY = ACCFULL + 2;
  auto bar = [&](int i) { return oz_smem_u32(&bars[i]); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngroups = *ngroups_dev;

  if (tid == 0) {
    for (int b = 0; b < OZ_WSTAGES; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WFULL + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WEMPTY + b)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WINFULL)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WINEMPTY)));
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(ACCFULL + a)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(bar(ACCEMPTY + a)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(oz_smem_u32(&tmem_slot)), "n"(2 * OZ_ACC_STRIDE));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------- window loads + MMA issue ----------------
    if (lane == 0) {
      // kind::f16 with bf16 A and B, fp32 accumulate, K-major, M = 128, N = KR
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(KR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t winbase = oz_smem_u32(sWin);
      const uint32_t plane_bytes = (uint32_t)WL * 16;
      int kk = 0, committed = 0, issued_win = 0;
      int g = 0, gstart = 0;  // current group and its first offset
      for (int d = 0; d < ndy && !*(volatile int*)&abort_flag; ++d) {
        if (d > 0 && !oz_wait(bar(WINEMPTY), (d - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        const int gs = dy_start[d], ge = dy_start[d + 1];
        const int2 o0 = off[gs];
        const int64_t start = p0 + (int64_t)o0.y * W;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar(WINFULL)), "r"((uint32_t)(OZ_S * KC) * plane_bytes) : "memory");
        for (int i = 0; i < OZ_S; ++i)
          for (int kc = 0; kc < KC; ++kc) {
            const int64_t plane = ((int64_t)(r * 2 + c) * OZ_S + i) * KC + kc;
            const uint4* src = Xs + plane * PL + start;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(winbase + (uint32_t)(i * KC + kc) * plane_bytes), "l"(src), "r"(plane_bytes),
                            "r"(bar(WINFULL)) : "memory");
          }
        issued_win = d + 1;
        if (!oz_wait(bar(WINFULL), d & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        for (; kk < ge; ++kk) {
          const int wb = kk % OZ_WSTAGES;
          if (kk == group_end[g]) {  // the previous offset closed group g
            gstart = kk;
            ++g;
          }
          const int a = g & 1;
          const bool first_in_group = kk == gstart;
          if (first_in_group && g >= 2 && !oz_wait(bar(ACCEMPTY + a), ((g - 2) >> 1) & 1)) {
            atomicOr(&abort_flag, 1);
            break;
          }
          if (!oz_wait(bar(WFULL + wb), (kk / OZ_WSTAGES) & 1)) {
            atomicOr(&abort_flag, 1);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int dx = o0.x + (kk - gs);
          const uint32_t ashift = (uint32_t)(CX + dx) * 16;
          const uint32_t wbase = oz_smem_u32(sW + wb * S::W_STAGE);
          const uint32_t dset = tmem + (uint32_t)(a * OZ_ACC_STRIDE);
#pragma unroll
          for (int l = 0; l <= OZ_LMAX; ++l) {
            const int q = l < OZ_NACC - 1 ? l : OZ_NACC - 1;
            const uint32_t dacc = dset + (uint32_t)(q * KR);
#pragma unroll
            for (int i = 0; i <= l; ++i) {
              const int j = l - i;
              if (i >= OZ_S || j >= OZ_S) continue;
#pragma unroll
              for (int s = 0; s < KR / 16; ++s) {
                const uint32_t aaddr = winbase + (uint32_t)(i * KC + 2 * s) * plane_bytes + ashift;
                const uint32_t baddr = wbase + (uint32_t)(j * S::W_SLICE + s * 256);
                const uint64_t dA = oz_desc(aaddr, plane_bytes, 128), dB = oz_desc(baddr, 128, KC * 128);
                const uint32_t acc0 = (first_in_group && i == 0 && s == 0 && l <= OZ_NACC - 1) ? 0u : 1u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             :: "r"(dacc), "l"(dA), "l"(dB), "r"(idesc), "r"(acc0));
              }
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(bar(WEMPTY + wb)) : "memory");
          if (kk + 1 == group_end[g])
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar(ACCFULL + a)) : "memory");
          committed = kk + 1;
        }
        if (*(volatile int*)&abort_flag) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(bar(WINEMPTY)) : "memory");
      }
      if (committed > 0) {
        const int kl = committed - 1;
        if (!oz_wait(bar(WEMPTY + kl % OZ_WSTAGES), (kl / OZ_WSTAGES) & 1)) atomicOr(&abort_flag, 1);
      }
      if (issued_win > 0 && !oz_wait(bar(WINFULL), (issued_win - 1) & 1)) atomicOr(&abort_flag, 1);
      if (committed != K) atomicOr(&abort_flag, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- W loader ----------------
    if (lane == 0) {
      int issued = 0;
      for (int kk = 0; kk < K; ++kk) {
        if (*(volatile int*)&abort_flag) break;
        const int wb = kk % OZ_WSTAGES, use = kk / OZ_WSTAGES;
        if (kk >= OZ_WSTAGES && !oz_wait(bar(WEMPTY + wb), (use - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar(WFULL + wb)), "r"((uint32_t)S::W_STAGE) : "memory");
        const unsigned char* src = Wt + ((size_t)kk * 2 + c) * S::W_STAGE;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(oz_smem_u32(sW + wb * S::W_STAGE)), "l"(src), "r"((uint32_t)S::W_STAGE),
                        "r"(bar(WFULL + wb)) : "memory");
        issued = kk + 1;
      }
      for (int kl = issued > OZ_WSTAGES ? issued - OZ_WSTAGES : 0; kl < issued; ++kl)
        if (!oz_wait(bar(WFULL + kl % OZ_WSTAGES), (kl / OZ_WSTAGES) & 1)) atomicOr(&abort_flag, 1);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---------------- readers: exact group sums into double-float ----------------
    const int q4 = warp & 3;
    const int m = q4 * 32 + lane;
    const int64_t pp = p0 + m;
    const int64_t iy = pp / W - CY, ix = pp % W - CX;
    const bool live = iy >= 0 && iy < ny && ix >= 0 && ix < nx;
    float hi[KR], lo[KR];
#pragma unroll
    for (int e = 0; e < KR; ++e) hi[e] = lo[e] = 0.f;
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      const int a = g & 1;
      const bool seen = __any_sync(0xffffffffu, oz_wait(bar(ACCFULL + a), (g >> 1) & 1));
      if (!seen) {
        ok = false;
        atomicOr(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c0 = 0; c0 < KR; c0 += 16) {
#pragma unroll
        for (int q = 0; q < OZ_NACC; ++q) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * OZ_ACC_STRIDE + q * KR + c0);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                       : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                         "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float s, er;
            two_sum(hi[c0 + e], __uint_as_float(v[e]), s, er);
            hi[c0 + e] = s;
            lo[c0 + e] += er;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar(ACCEMPTY + a)) : "memory");
    }
    __syncwarp();
    if (ok && live) {
      const int ex = oz_scale_exp(__longlong_as_double((long long)smax[r * 2 + c]));
      const int64_t orow = (iy * nx + ix) * P + c * L;
#pragma unroll
      for (int u = 0; u < L; ++u) {
        const double2 av = make_double2(
            ldexp((double)hi[2 * u] + (double)lo[2 * u], ex + colexp[c * KR + 2 * u] - 16),
            ldexp((double)hi[2 * u + 1] + (double)lo[2 * u + 1], ex + colexp[c * KR + 2 * u + 1] - 16));
        double2 out;
        if (MODE == 2) {
          out = av;
        } else {
          const double2 xv = x[r * rstride + orow + u];
          if (MODE == 0) {
            const double2 t = cmul(T[orow + u], av);
            out = make_double2(xv.x - t.x, xv.y - t.y);
          } else {
            out = make_double2(xv.x - av.x, xv.y - av.y);
          }
        }
        y[r * rstride + orow + u] = out;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && abort_flag) atomicAdd(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(2 * OZ_ACC_STRIDE));
}

template <int NMAX>
static size_t oz_smem(int CX) {
  using S = OzShape<NMAX>;
  return (size_t)OZ_S * S::KC * (128 + 2 * CX) * 16 + (size_t)OZ_WSTAGES * S::W_STAGE;
}

bool lattice_oz_fits(int nmax, int CX) {
  size_t need = 0;
  switch (nmax) {
    case 1: need = oz_smem<1>(CX); break;
    case 2: need = oz_smem<2>(CX); break;
    case 3: need = oz_smem<3>(CX); break;
    case 4: need = oz_smem<4>(CX); break;
    default: return false;
  }
  return need + 1024 <= 227 * 1024;
}

int lattice_oz_prepare(tmat_ctx* ctx, LatOp* a, const double2* BT64) {
  (void)BT64;  // the slices depend on the sources and are cut per apply
  if (a->K == 0) return TMAT_OK;
  if (a->nmax < 1 || a->nmax > 4) return set_error(ctx, TMAT_ENOTSUP, "tensor-core fp64 apply supports nmax 1..4");
  int* err;
  TM_TRY(scratch(ctx, "oz_err", sizeof(int), (void**)&err));
  TM_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  a->oz_err = err;
  return TMAT_OK;
}

template <int NMAX, int MODE>
static int run_oz(tmat_ctx* ctx, const LatOp& a, const void* x, void* y, int R_) {
  using S = OzShape<NMAX>;
  constexpr int L = S::L, P = 2 * L;
  const int K = a.K;
  const int CY = a.CY;
  const int Wd = a.nx + 2 * a.CX;
  const int64_t PP = (int64_t)(a.ny + 2 * CY) * Wd;
  const int64_t PL = PP + 2 * a.CX + 256;
  const int64_t rs = a.N * a.P;
  const int tmode = MODE == 1 ? 1 : 0;  // W direction
  uint4* Xs;
  unsigned long long *dmax, *smax;
  int *dexp, *colexp, *gend, *ngroups;
  unsigned char* W;
  double* bound;
  TM_TRY(scratch(ctx, "oz_Xs", sizeof(uint4) * (size_t)R_ * 2 * OZ_S * S::KC * PL, (void**)&Xs));
  TM_TRY(scratch(ctx, "oz_W", (size_t)K * 2 * S::W_STAGE, (void**)&W));
  TM_TRY(scratch(ctx, "oz_bound", sizeof(double) * (size_t)K * 2 * 3, (void**)&bound));
  TM_TRY(scratch(ctx, "oz_gend", sizeof(int) * (size_t)(K + 1), (void**)&gend));
  char* small;
  const size_t nsmall = sizeof(unsigned long long) * (P + 2 * TMAT_MAX_RHS) + sizeof(int) * (P + 2 * S::KR + 1);
  TM_TRY(scratch(ctx, "oz_small", nsmall, (void**)&small));
  dmax = (unsigned long long*)small;
  smax = dmax + P;
  dexp = (int*)(smax + 2 * TMAT_MAX_RHS);
  colexp = dexp + P;
  ngroups = colexp + 2 * S::KR;
  TM_CUDA(ctx, cudaMemsetAsync(small, 0, sizeof(unsigned long long) * (P + 2 * TMAT_MAX_RHS), ctx->stream));
  const unsigned gsc = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(a.N, 256 / P), (int64_t)ctx->num_sms * 4));
  const double2* xd = (const double2*)x;
  const double2* Td = (const double2*)a.T;
  oz_xscale_kernel<NMAX, MODE, false><<<gsc, 256, 0, ctx->stream>>>(xd, Td, a.N, R_, nullptr, dmax);
  TM_LAUNCHED(ctx);
  oz_dexp_kernel<<<1, 64, 0, ctx->stream>>>(dmax, P, dexp);
  TM_LAUNCHED(ctx);
  oz_xscale_kernel<NMAX, MODE, true><<<gsc, 256, 0, ctx->stream>>>(xd, Td, a.N, R_, dexp, smax);
  TM_LAUNCHED(ctx);
  const double2* BT64 = (const double2*)a.BT;
  oz_wscale_kernel<NMAX><<<2 * S::KR, 256, 0, ctx->stream>>>(BT64, a.LP, a.neg, K, tmode, dexp, colexp);
  TM_LAUNCHED(ctx);
  oz_wtables_kernel<NMAX><<<2 * K, 256, 0, ctx->stream>>>(BT64, a.LP, a.neg, K, tmode, dexp, colexp, W, bound);
  TM_LAUNCHED(ctx);
  oz_groups_kernel<<<1, 32, 0, ctx->stream>>>(bound, K, gend, ngroups);
  TM_LAUNCHED(ctx);
  {
    const int64_t total = (int64_t)R_ * 2 * S::KC * PL;
    oz_split_kernel<NMAX, MODE><<<(unsigned)std::min<int64_t>(cdiv(total, 256), (int64_t)ctx->num_sms * 16), 256, 0,
                                  ctx->stream>>>(xd, Td, a.nx, a.ny, a.CX, CY, PL, R_, rs, dexp, smax, Xs);
    TM_LAUNCHED(ctx);
  }
  auto kern = lattice_oz_kernel<NMAX, MODE>;
  const size_t smem = oz_smem<NMAX>(a.CX);
  TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
  const int64_t rows = (int64_t)a.ny * Wd;
  dim3 grid((unsigned)cdiv(rows, 128), 2, (unsigned)R_);
  cudaEvent_t ev = timing_begin(ctx);
  kern<<<grid, OZ_THREADS, smem, ctx->stream>>>(a.off, K, a.dy_start, a.ndy, gend, ngroups, a.CX, CY, a.nx, a.ny, PL,
                                                Xs, W, colexp, smax, Td, xd, (double2*)y, rs, a.oz_err);
  TM_LAUNCHED(ctx);
  timing_end(ctx, "lattice_apply_oz", ev);
  return TMAT_OK;
}

template <int NMAX>
static int oz_dispatch(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  if (mode == TMAT_OP_FORWARD) return run_oz<NMAX, 0>(ctx, a, x, y, R_);
  if (mode == TMAT_OP_ADJOINT) return run_oz<NMAX, 1>(ctx, a, x, y, R_);
  return run_oz<NMAX, 2>(ctx, a, x, y, R_);
}

int lattice_oz_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  switch (a.nmax) {
    case 1: return oz_dispatch<1>(ctx, a, mode, x, y, R_);
    case 2: return oz_dispatch<2>(ctx, a, mode, x, y, R_);
    case 3: return oz_dispatch<3>(ctx, a, mode, x, y, R_);
    case 4: return oz_dispatch<4>(ctx, a, mode, x, y, R_);
  }
  return set_error(ctx, TMAT_ENOTSUP, "tensor-core fp64 apply supports nmax 1..4");
}

}  // namespace tmat
