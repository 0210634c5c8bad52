// Lattice operator apply on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For one class c and one lattice offset o the apply is a dense contraction
//     Y[m, u] += sum_u' X[m + o, u'] G_o[u, u']      (m = target site, per RHS)
// of complex numbers. Written with real and imaginary parts interleaved
// (k = 2u' + s, n = 2u + t) it is the real GEMM D[m, n] += sum_k A[m, k] W_o[n, k]
// with W = [[Re, -Im], [Im, Re]] per complex entry, K = N = 2L (padded to LP2).
// A CTA owns one class and 128 rows m (sites x RHS) and sums all offsets in a
// TMEM accumulator (M = 128, N = 2 LP2, fp32). Precision: 3xTF32 -- every
// operand is split into a TF32 head and a TF32 tail and the product is
// A_hi W_hi + A_hi W_lo + A_lo W_hi, which keeps the fp32-level accuracy of the
// CUDA-core kernel at tensor-core throughput.
//
// Pipeline (2 stages): an elected thread fetches the offset's pre-split W tiles
// (already in the MMA core-matrix layout) with one cp.async.bulk per tile onto a
// "full" mbarrier; all threads gather the shifted source rows (zero outside the
// lattice), split them and store them in core-matrix layout; the elected thread
// then issues the 3 x (2 LP2 / 8) MMAs and commits them to the stage's "empty"
// mbarrier, which gates the next overwrite of that stage. Every wait is bounded:
// on expiry the CTA records an error, drains its own work with bounded waits,
// frees its TMEM and returns.
#include <cstdint>

#include "dev.cuh"
#include "solver.h"

namespace tmat {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

template <int NMAX> struct TcShape {
  static constexpr int L = NMAX * (NMAX + 2);
  static constexpr int LP2 = (L + 7) / 8 * 8;    // padded complex width: 2 LP2 is a multiple of 16
  static constexpr int KR = 2 * LP2;             // real K = real N
  static constexpr int KC = KR / 4;              // 16-byte core columns along K
  static constexpr int A_BYTES = TC_M * KR * 4;  // one A tile (hi or lo)
  static constexpr int W_BYTES = KR * KR * 4;    // one W tile (hi or lo)
  static constexpr int STAGE = 2 * A_BYTES + 2 * W_BYTES;
  static constexpr int TMEM_COLS = KR <= 32 ? 32 : (KR <= 64 ? 64 : 128);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element (row, k) of a K-major, no-swizzle tile with KC 16-byte cores along K:
// 8 x 16-byte core matrices, LBO = 128 B (next core along K), SBO = KC * 128 B (next 8 rows)
__host__ __device__ __forceinline__ int core_off(int row, int k, int KC) {
  return ((row >> 3) * KC + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version 0b001; base offset 0; no swizzle
  return d;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TF32 head of an fp32 value with integer ops: adding half of the dropped 13-bit unit to the
// sign-magnitude pattern and masking rounds the magnitude to nearest, ties away from zero
// (the rounding of cvt.rna.tf32.f32) for finite inputs.
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// W tiles for every offset and class, in the MMA core-matrix layout, split into
// TF32 head and tail: W[((o*2 + c)*2 + h)][core layout of KR x KR]. mode 0:
// forward blocks G_o[u][u'] = BT[o][c][u'][u]; mode 1: adjoint blocks
// G[u][u'] = BT[neg(o)][c][u][u'].
template <int NMAX>
__global__ void tc_wtables_kernel(const double2* __restrict__ BT, int LP, const int* __restrict__ neg, int K, int mode,
                                  float* __restrict__ W) {
  using S = TcShape<NMAX>;
  const int oc = blockIdx.x;  // o*2 + c
  if (oc >= 2 * K) return;
  const int o = oc >> 1, c = oc & 1;
  float* Wh = W + (size_t)oc * 2 * (S::KR * S::KR);
  float* Wl = Wh + S::KR * S::KR;
  for (int e = threadIdx.x; e < S::KR * S::KR; e += blockDim.x) {
    const int n = e / S::KR, k = e % S::KR;
    const int u = n >> 1, t = n & 1, up = k >> 1, s = k & 1;
    double w = 0.0;
    if (u < S::L && up < S::L) {
      double2 z = mode == 0 ? BT[(((size_t)o * 2 + c) * S::L + up) * LP + u]
                            : BT[(((size_t)neg[o] * 2 + c) * S::L + u) * LP + up];
      w = (t == s) ? z.x : (t == 1 ? z.y : -z.y);
    }
    const float hi = tf32_rna((float)w);
    const float lo = tf32_rna((float)(w - (double)hi));
    const int off = core_off(n, k, S::KC) >> 2;
    Wh[off] = hi;
    Wl[off] = lo;
  }
}

// MODE 0: y = x - T (A x); 1: y = x - A^T (T x) (xsrc = T x); 2: y = A x. NR right-hand
// sides share each tile (rows m = r * (128/NR) + site offset).
//
// Warp roles (320 threads):
//   warps 0-3  producers: row m = tid. Offsets come sorted by dy, then dx (contiguous dx per
//              dy). For one dy the sources of the tile's sites form one window of
//              WS = SITES + 2 CX consecutive sites per RHS, staged raw in shared memory with
//              cp.async (double-buffered: the next dy's window loads while this one is used).
//              For each offset a producer reads its source row from the window, splits it
//              into TF32 head/tail and stores both in the A stage (core-matrix layout).
//   warp 4     MMA issuer (one lane): 3 x KR/8 MMAs per offset into one of two TMEM
//              accumulators; the accumulator changes every TC_GROUP offsets.
//   warp 5     W loader (one lane): one cp.async.bulk per offset into a TC_WSTAGES-deep ring,
//              running ahead of the MMAs as far as the ring allows.
//   warps 6-9  readers: drain a finished accumulator into fp32 registers (round to nearest),
//              keeping every tensor-core accumulation chain short, then write the outputs.
constexpr int TC_ASTAGES = 2;
constexpr int TC_WSTAGES = 3;
constexpr int TC_GROUP = 8;
constexpr int TC_ALL_THREADS = 320;

template <int L> struct TcWin { static constexpr int LW = L | 1; };  // odd stride: conflict-free 8-byte reads

template <int NMAX, int NR, int MODE>
__global__ void __launch_bounds__(TC_ALL_THREADS, 1)
lattice_tc_kernel(const int2* __restrict__ off, int K, const int* __restrict__ dy_start, int ndy, int CX, int nx,
                  int ny, int64_t N, const float* __restrict__ W, const float2* __restrict__ T,
                  const float2* __restrict__ xsrc, const float2* __restrict__ x, float2* __restrict__ y,
                  int64_t rstride, int* __restrict__ err) {
  using S = TcShape<NMAX>;
  constexpr int L = S::L, P = 2 * L, KR = S::KR, KC = S::KC, LW = TcWin<L>::LW;
  constexpr int SITES = TC_M / NR;
  constexpr int ACC_COLS = S::TMEM_COLS;
  constexpr int A_STAGE = 2 * S::A_BYTES, W_STAGE = 2 * S::W_BYTES;
  extern __shared__ __align__(1024) unsigned char smem[];
  // afull[2], aempty[2], wfull[3], wempty[3], accfull[2], accempty[2]
  __shared__ uint64_t bars[2 * TC_ASTAGES + 2 * TC_WSTAGES + 4];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.y;
  const int64_t site0 = (int64_t)blockIdx.x * SITES;
  const int ngroups = (K + TC_GROUP - 1) / TC_GROUP;
  constexpr int AFULL = 0, AEMPTY = TC_ASTAGES, WFULL = 2 * TC_ASTAGES, WEMPTY = 2 * TC_ASTAGES + TC_WSTAGES;
  constexpr int ACCFULL = 2 * TC_ASTAGES + 2 * TC_WSTAGES, ACCEMPTY = ACCFULL + 2;
  auto bar = [&](int idx) { return smem_u32(&bars[idx]); };
  unsigned char* sA = smem;                                 // A ring: [stage][hi | lo]
  unsigned char* sW = smem + TC_ASTAGES * A_STAGE;          // W ring: [stage][hi | lo]
  float2* win0 = reinterpret_cast<float2*>(sW + TC_WSTAGES * W_STAGE);

  if (tid == 0) {
    for (int b = 0; b < TC_ASTAGES; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(bar(AFULL + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(AEMPTY + b)));
    }
    for (int b = 0; b < TC_WSTAGES; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WFULL + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(WEMPTY + b)));
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar(ACCFULL + a)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(bar(ACCEMPTY + a)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "n"(2 * S::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp < 4) {
    // ---------------- producers ----------------
    const int WS = SITES + 2 * CX;
    const int m = tid;
    const int r = m / SITES;
    const int sm_ = m % SITES;
    const int64_t i = site0 + sm_;
    const bool live = i < N;
    const int ix = live ? (int)(i % nx) : 0, iy = live ? (int)(i / nx) : 0;
    const int win_elems = NR * WS * LW;
    auto load_window = [&](int d, float2* dst) {
      const int dy = off[dy_start[d]].y;
      const int64_t first = site0 + (int64_t)dy * nx - CX;  // site index of window position 0
      for (int e = tid; e < NR * WS * L; e += 128) {
        const int rr = e / (WS * L), rem = e % (WS * L), p = rem / L, cc = rem % L;
        const int64_t site = first + p;
        float2* d2 = dst + ((size_t)rr * WS + p) * LW + cc;
        if (site >= 0 && site < N) {
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                       :: "r"(smem_u32(d2)), "l"(xsrc + rr * rstride + site * P + c * L + cc) : "memory");
        } else {
          *d2 = make_float2(0.f, 0.f);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (ndy > 0) load_window(0, win0);
    int kk = 0;
    // every producer passes every named barrier: after an abort the work is skipped, the
    // loop structure (and so the barrier count) is not
    for (int d = 0; d < ndy; ++d) {
      asm volatile("bar.sync 1, 128;" ::: "memory");  // all producers are done with window d-1
      if (d + 1 < ndy) {
        load_window(d + 1, win0 + (size_t)((d + 1) & 1) * win_elems);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");  // window d complete and visible
      const float2* win = win0 + (size_t)(d & 1) * win_elems;
      const int gs = dy_start[d], ge = dy_start[d + 1];
      const int2 o0 = off[gs];  // dx is contiguous inside a dy group
      const int sy = iy + o0.y;
      for (; kk < ge; ++kk) {
        if (*(volatile int*)&abort_flag) continue;
        const int b = kk % TC_ASTAGES, use = kk / TC_ASTAGES;
        if (kk >= TC_ASTAGES && !mbar_wait(bar(AEMPTY + b), (use - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          continue;
        }
        unsigned char* sAh = sA + b * A_STAGE;
        unsigned char* sAl = sAh + S::A_BYTES;
        const int dx = o0.x + (kk - gs);
        const int sx = ix + dx;
        const bool valid = live && sx >= 0 && sx < nx && sy >= 0 && sy < ny;
        const float2* src2 = win + ((size_t)r * WS + (sm_ + CX + dx)) * LW;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (valid && 2 * q < L) {
            const float2 h0 = src2[2 * q];
            const float2 h1 = (2 * q + 1 < L) ? src2[2 * q + 1] : make_float2(0.f, 0.f);
            v = make_float4(h0.x, h0.y, h1.x, h1.y);
          }
          // head rounded to TF32; the tail v - h is exact in fp32 and the MMA reads only its
          // top 19 bits (error <= 2^-22 |v|)
          float4 h, l;
          h.x = tf32_head(v.x); h.y = tf32_head(v.y); h.z = tf32_head(v.z); h.w = tf32_head(v.w);
          l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
          const int co = core_off(m, 4 * q, KC);
          *reinterpret_cast<float4*>(sAh + co) = h;
          *reinterpret_cast<float4*>(sAl + co) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar(AFULL + b)) : "memory");
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else if (warp == 4) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KR >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    const uint32_t LBO = 128, SBO = KC * 128;
    if (lane == 0) {
      int committed = 0;
      for (int kk = 0; kk < K; ++kk) {
        if (*(volatile int*)&abort_flag) break;
        const int b = kk % TC_ASTAGES, wb = kk % TC_WSTAGES;
        const int g = kk / TC_GROUP, a = g & 1;
        const bool first_in_group = (kk % TC_GROUP) == 0;
        if (first_in_group && g >= 2 && !mbar_wait(bar(ACCEMPTY + a), ((g - 2) >> 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        if (!mbar_wait(bar(AFULL + b), (kk / TC_ASTAGES) & 1) || !mbar_wait(bar(WFULL + wb), (kk / TC_WSTAGES) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ah = smem_u32(sA + b * A_STAGE), al = ah + S::A_BYTES;
        const uint32_t wh = smem_u32(sW + wb * W_STAGE), wl = wh + S::W_BYTES;
        const uint32_t dacc = tmem + (uint32_t)(a * ACC_COLS);
#pragma unroll
        for (int s = 0; s < KR / 8; ++s) {
          const uint32_t ko = s * 256;  // two 16-byte core columns per K = 8 step
          const uint64_t dAh = umma_desc(ah + ko, LBO, SBO), dAl = umma_desc(al + ko, LBO, SBO);
          const uint64_t dWh = umma_desc(wh + ko, LBO, SBO), dWl = umma_desc(wl + ko, LBO, SBO);
          const uint32_t acc0 = (!first_in_group || s > 0) ? 1u : 0u;
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                       :: "r"(dacc), "l"(dAh), "l"(dWh), "r"(idesc), "r"(acc0));
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                       :: "r"(dacc), "l"(dAh), "l"(dWl), "r"(idesc));
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                       :: "r"(dacc), "l"(dAl), "l"(dWh), "r"(idesc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(bar(AEMPTY + b)) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(bar(WEMPTY + wb)) : "memory");
        if ((kk % TC_GROUP) == TC_GROUP - 1 || kk == K - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(bar(ACCFULL + a)) : "memory");
        committed = kk + 1;
      }
      // drain: the last commit covers every MMA this thread issued
      if (committed > 0) {
        const int kl = committed - 1;
        if (!mbar_wait(bar(AEMPTY + kl % TC_ASTAGES), (kl / TC_ASTAGES) & 1)) atomicOr(&abort_flag, 1);
      }
      if (committed != K) atomicOr(&abort_flag, 1);
    }
    __syncwarp();
  } else if (warp == 5) {
    // ---------------- W loader ----------------
    if (lane == 0) {
      int issued = 0;
      for (int kk = 0; kk < K; ++kk) {
        if (*(volatile int*)&abort_flag) break;
        const int wb = kk % TC_WSTAGES, use = kk / TC_WSTAGES;
        if (kk >= TC_WSTAGES && !mbar_wait(bar(WEMPTY + wb), (use - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar(WFULL + wb)), "r"(W_STAGE) : "memory");
        const float* src = W + ((size_t)kk * 2 + c) * 2 * (KR * KR);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sW + wb * W_STAGE)), "l"(src), "r"(W_STAGE), "r"(bar(WFULL + wb)) : "memory");
        issued = kk + 1;
      }
      // let the last copy land before the CTA's shared memory can be released
      if (issued > 0) {
        const int kl = issued - 1;
        if (!mbar_wait(bar(WFULL + kl % TC_WSTAGES), (kl / TC_WSTAGES) & 1)) atomicOr(&abort_flag, 1);
      }
    }
    __syncwarp();
  } else {
    // ---------------- readers ----------------
    const int q4 = warp & 3;  // TMEM lane quarter this warp may access
    const int m = q4 * 32 + lane;
    const int r = m / SITES;
    const int64_t i = site0 + (m % SITES);
    const bool live = i < N;
    float accr[KR];
#pragma unroll
    for (int e = 0; e < KR; ++e) accr[e] = 0.f;
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      const int a = g & 1;
      // warp-uniform outcome (the tcgen05.ld below is .sync.aligned): if any lane saw the
      // phase complete, it is complete for all
      const bool seen = __any_sync(0xffffffffu, mbar_wait(bar(ACCFULL + a), (g >> 1) & 1));
      if (!seen) {
        ok = false;
        atomicOr(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c0 = 0; c0 < KR; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * ACC_COLS + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                       "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int e = 0; e < 16; ++e) accr[c0 + e] += __uint_as_float(v[e]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar(ACCEMPTY + a)) : "memory");
    }
    __syncwarp();
    if (ok && live) {
      const int64_t orow = i * P + c * L;
#pragma unroll
      for (int u = 0; u < L; ++u) {
        const float2 av = make_float2(accr[2 * u], accr[2 * u + 1]);
        float2 out;
        if (MODE == 2) {
          out = av;
        } else {
          const float2 xv = x[r * rstride + orow + u];
          if (MODE == 0) {
            const float2 t = T[orow + u];
            out = make_float2(xv.x - (t.x * av.x - t.y * av.y), xv.y - (t.x * av.y + t.y * av.x));
          } else {
            out = make_float2(xv.x - av.x, xv.y - av.y);
          }
        }
        y[r * rstride + orow + u] = out;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && abort_flag) atomicAdd(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(2 * S::TMEM_COLS));
}

template <int NMAX>
static size_t tc_smem(int NR, int CX) {
  using S = TcShape<NMAX>;
  const int WS = TC_M / NR + 2 * CX;
  return (size_t)TC_ASTAGES * 2 * S::A_BYTES + (size_t)TC_WSTAGES * 2 * S::W_BYTES +
         2 * sizeof(float2) * (size_t)NR * WS * TcWin<S::L>::LW;
}

template <int NMAX, int NR, int MODE>
static int launch_tc(tmat_ctx* ctx, const LatOp& a, const float* W, const void* xsrc, const void* x, void* y,
                     int64_t rs, int* err) {
  auto kern = lattice_tc_kernel<NMAX, NR, MODE>;
  const size_t smem = tc_smem<NMAX>(NR, a.CX);
  TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
  constexpr int SITES = TC_M / NR;
  dim3 grid((unsigned)cdiv(a.N, SITES), 2);
  cudaEvent_t ev = timing_begin(ctx);
  kern<<<grid, TC_ALL_THREADS, smem, ctx->stream>>>(a.off, a.K, a.dy_start, a.ndy, a.CX, a.nx, a.ny, a.N, W,
                                                    (const float2*)a.T, (const float2*)xsrc, (const float2*)x,
                                                    (float2*)y, rs, err);
  TM_LAUNCHED(ctx);
  timing_end(ctx, "lattice_apply_tc", ev);
  return TMAT_OK;
}

// tx[r][i][u] = T[i][u] x[r][i][u] (the adjoint applies T to the sources first)
__global__ void tmul32_kernel(const float2* __restrict__ T, const float2* __restrict__ x, float2* __restrict__ tx,
                              int64_t NP, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = T[t % NP], b = x[t];
    tx[t] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
}

template <int NMAX>
static int tc_dispatch(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  const int64_t rs = a.N * a.P;
  const float* W = (const float*)(mode == TMAT_OP_ADJOINT ? a.Wtc_adj : a.Wtc_fwd);
  const void* xsrc = x;
  if (mode == TMAT_OP_ADJOINT) {
    float2* tx;
    TM_TRY(scratch(ctx, "tc_tx", sizeof(float2) * (size_t)R_ * rs, (void**)&tx));
    const int64_t total = (int64_t)R_ * rs;
    tmul32_kernel<<<(unsigned)std::min<int64_t>(cdiv(total, 256), 65535), 256, 0, ctx->stream>>>(
        (const float2*)a.T, (const float2*)x, tx, rs, total);
    TM_LAUNCHED(ctx);
    xsrc = tx;
  }
  for (int r0 = 0; r0 < R_; r0 += 2) {
    const int nr = (R_ - r0) >= 2 ? 2 : 1;
    const size_t o = sizeof(float2) * rs * r0;
    const char* sp = (const char*)xsrc + o;
    const char* xp = (const char*)x + o;
    char* yp = (char*)y + o;
    int rc;
    if (nr == 2) {
      rc = mode == TMAT_OP_FORWARD ? launch_tc<NMAX, 2, 0>(ctx, a, W, sp, xp, yp, rs, a.tc_err)
           : mode == TMAT_OP_ADJOINT ? launch_tc<NMAX, 2, 1>(ctx, a, W, sp, xp, yp, rs, a.tc_err)
                                     : launch_tc<NMAX, 2, 2>(ctx, a, W, sp, xp, yp, rs, a.tc_err);
    } else {
      rc = mode == TMAT_OP_FORWARD ? launch_tc<NMAX, 1, 0>(ctx, a, W, sp, xp, yp, rs, a.tc_err)
           : mode == TMAT_OP_ADJOINT ? launch_tc<NMAX, 1, 1>(ctx, a, W, sp, xp, yp, rs, a.tc_err)
                                     : launch_tc<NMAX, 1, 2>(ctx, a, W, sp, xp, yp, rs, a.tc_err);
    }
    if (rc) return rc;
  }
  return TMAT_OK;
}

bool lattice_tc_supported(int nmax) { return nmax >= 1 && nmax <= 4; }

// the source windows must fit next to the pipeline stages (227 KB per block)
bool lattice_tc_fits(int nmax, int CX) {
  size_t need = 0;
  switch (nmax) {
    case 1: need = tc_smem<1>(1, CX); break;
    case 2: need = tc_smem<2>(1, CX); break;
    case 3: need = tc_smem<3>(1, CX); break;
    case 4: need = tc_smem<4>(1, CX); break;
    default: return false;
  }
  size_t need2 = need;
  switch (nmax) {
    case 1: need2 = tc_smem<1>(2, CX); break;
    case 2: need2 = tc_smem<2>(2, CX); break;
    case 3: need2 = tc_smem<3>(2, CX); break;
    case 4: need2 = tc_smem<4>(2, CX); break;
  }
  return std::max(need, need2) + 1024 <= 227 * 1024;
}

int lattice_tc_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  switch (a.nmax) {
    case 1: return tc_dispatch<1>(ctx, a, mode, x, y, R_);
    case 2: return tc_dispatch<2>(ctx, a, mode, x, y, R_);
    case 3: return tc_dispatch<3>(ctx, a, mode, x, y, R_);
    case 4: return tc_dispatch<4>(ctx, a, mode, x, y, R_);
  }
  return set_error(ctx, TMAT_ENOTSUP, "tensor-core lattice apply supports nmax 1..4");
}

// Build the split W tables of both modes from the fp64 block table.
int lattice_tc_prepare(tmat_ctx* ctx, LatOp* a, const double2* BT64) {
  if (!lattice_tc_supported(a->nmax) || a->K == 0) return TMAT_OK;
  int KR = 0;
  switch (a->nmax) {
    case 1: KR = TcShape<1>::KR; break;
    case 2: KR = TcShape<2>::KR; break;
    case 3: KR = TcShape<3>::KR; break;
    case 4: KR = TcShape<4>::KR; break;
  }
  const size_t per = (size_t)a->K * 2 * 2 * KR * KR;
  float *Wf, *Wa;
  int* err;
  TM_TRY(scratch(ctx, "tc_Wfwd", sizeof(float) * per, (void**)&Wf));
  TM_TRY(scratch(ctx, "tc_Wadj", sizeof(float) * per, (void**)&Wa));
  TM_TRY(scratch(ctx, "tc_err", sizeof(int), (void**)&err));
  TM_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  for (int mode = 0; mode < 2; ++mode) {
    float* W = mode == 0 ? Wf : Wa;
    switch (a->nmax) {
#define TW(NM) case NM: tc_wtables_kernel<NM><<<2 * a->K, 256, 0, ctx->stream>>>(BT64, a->LP, a->neg, a->K, mode, W); break;
      TW(1) TW(2) TW(3) TW(4)
#undef TW
    }
    TM_LAUNCHED(ctx);
  }
  a->Wtc_fwd = Wf;
  a->Wtc_adj = Wa;
  a->tc_err = err;
  return TMAT_OK;
}

}  // namespace tmat
