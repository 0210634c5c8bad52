// Lattice operator apply on tcgen05 tensor cores, "window view" variant.
//
// The complex64 source vector is split once per apply (TF32 head + tail) into a
// zero-padded, k-chunk-major layout: for each (RHS, class, head/tail, 16-byte
// k-chunk) one plane over the padded lattice positions pp = (iy + CY) W + ix + CX,
// W = nx + 2 CX, 16 bytes per position. Eight consecutive positions of a plane are
// one 8 x 16-byte core matrix of the no-swizzle K-major MMA layout, so for a tile
// of 128 consecutive positions the A operand of lattice offset (dx, dy) is the
// plane window starting dy W + dx positions further: the descriptor points into a
// staged window at a 16-byte offset (SBO = 128 B, LBO = window plane length).
// The zero pads (CX columns, CY rows) make every shifted source outside the
// lattice read zeros, so no per-offset masking or copying is needed.
//
// Per CTA: one class, one RHS, 128 positions. Warp 0 lane 0 issues the window
// bulk copies (once per dy) and the MMAs; warp 1 lane 0 streams the offsets' W
// tiles (cp.async.bulk, 2-deep ring); warps 4-7 drain two ping-pong TMEM
// accumulators every TC2_GROUP offsets into fp32 registers and write the outputs.
// All waits are bounded (see lattice_tc.cu).
#include <cstdint>

#include "dev.cuh"
#include "solver.h"

namespace tmat {

constexpr int TC2_THREADS = 256;
constexpr int TC2_GROUP = 8;
constexpr int TC2_WSTAGES = 2;
constexpr uint32_t TC2_WAIT_LIMIT = 1u << 22;

template <int NMAX> struct Tc2Shape {
  static constexpr int L = NMAX * (NMAX + 2);
  static constexpr int LP2 = (L + 7) / 8 * 8;
  static constexpr int KR = 2 * LP2;
  static constexpr int KC = KR / 4;
  static constexpr int W_BYTES = KR * KR * 4;
  // one accumulator set: columns [0, KR) collect A_hi W_hi + A_lo W_hi, [KR, 2 KR) A_hi W_lo
  static constexpr int TMEM_COLS = 2 * KR <= 32 ? 32 : (2 * KR <= 64 ? 64 : 128);
};

__device__ __forceinline__ uint32_t smem_u32_2(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool mbar_wait2(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < TC2_WAIT_LIMIT; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ float tf32_head2(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Split pass: Xs[plane][PL] float4 with plane = ((r*2 + c)*2 + h)*KC + kc, stored index
// pp + CX (so window starts never go negative); zeros outside the lattice.
template <int NMAX, int MODE>
__global__ void tc2_split_kernel(const float2* __restrict__ x, const float2* __restrict__ T, int nx, int ny, int CX,
                                 int CY, int64_t PL, int R, int64_t rstride, float4* __restrict__ Xs) {
  using S = Tc2Shape<NMAX>;
  constexpr int L = S::L, P = 2 * L, KC = S::KC;
  const int W = nx + 2 * CX;
  const int64_t total = (int64_t)R * 2 * KC * PL;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = t % PL;
    const int64_t rest = t / PL;
    const int kc = (int)(rest % KC);
    const int c = (int)((rest / KC) % 2);
    const int r = (int)(rest / (2 * KC));
    const int64_t pp = idx - CX;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pp >= 0) {
      const int64_t iy = pp / W - CY, ix = pp % W - CX;
      if (iy >= 0 && iy < ny && ix >= 0 && ix < nx && 2 * kc < L) {
        const int64_t site = iy * nx + ix;
        const float2* src = x + r * rstride + site * P + c * L + 2 * kc;
        float2 a = src[0], b = (2 * kc + 1 < L) ? src[1] : make_float2(0.f, 0.f);
        if (MODE == 1) {
          const float2* tp = T + site * P + c * L + 2 * kc;
          const float2 t0 = tp[0], t1 = (2 * kc + 1 < L) ? tp[1] : make_float2(0.f, 0.f);
          a = make_float2(t0.x * a.x - t0.y * a.y, t0.x * a.y + t0.y * a.x);
          b = make_float2(t1.x * b.x - t1.y * b.y, t1.x * b.y + t1.y * b.x);
        }
        v = make_float4(a.x, a.y, b.x, b.y);
      }
    }
    float4 h = make_float4(tf32_head2(v.x), tf32_head2(v.y), tf32_head2(v.z), tf32_head2(v.w));
    float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    const int64_t plane_h = ((int64_t)(r * 2 + c) * 2 + 0) * KC + kc;
    const int64_t plane_l = ((int64_t)(r * 2 + c) * 2 + 1) * KC + kc;
    Xs[plane_h * PL + idx] = h;
    Xs[plane_l * PL + idx] = l;
  }
}

template <int NMAX, int MODE>
__global__ void __launch_bounds__(TC2_THREADS, 2)
lattice_tc2_kernel(const int2* __restrict__ off, int K, const int* __restrict__ dy_start, int ndy, int CX, int CY,
                   int nx, int ny, int64_t PL, const float4* __restrict__ Xs, const float* __restrict__ Wt,
                   const float2* __restrict__ T, const float2* __restrict__ x, float2* __restrict__ y,
                   int64_t rstride, int* __restrict__ err) {
  using S = Tc2Shape<NMAX>;
  constexpr int L = S::L, P = 2 * L, KR = S::KR, KC = S::KC;
  constexpr int ACC_COLS = S::TMEM_COLS;
  constexpr int W_STAGE = 2 * S::W_BYTES;
  const int W = nx + 2 * CX;
  const int WL = 128 + 2 * CX;  // window positions
  const int tile = blockIdx.x, c = blockIdx.y, r = blockIdx.z;
  const int64_t p0 = (int64_t)CY * W + (int64_t)tile * 128;  // first padded position of the tile
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sWin = smem;                                        // [2 (h)][KC][WL] x 16 B
  unsigned char* sW = smem + (size_t)2 * KC * WL * 16;               // W ring
  // bars: wfull[2], wempty[2], winfull, winempty, accfull[2], accempty[2]
  __shared__ uint64_t bars[2 * TC2_WSTAGES + 6];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  constexpr int WFULL = 0, WEMPTY = TC2_WSTAGES, WINFULL = 2 * TC2_WSTAGES, WINEMPTY = WINFULL + 1;
  constexpr int ACCFULL = WINEMPTY + 1, ACCEMPTY = ACCFULL + 2;
  auto bar = [&](int i) { return smem_u32_2(&bars[i]); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngroups = (K + TC2_GROUP - 1) / TC2_GROUP;

  if (tid == 0) {
    for (int b = 0; b < TC2_WSTAGES; ++b) {
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
                 :: "r"(smem_u32_2(&tmem_slot)), "n"(2 * S::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------- window loads + MMA issue ----------------
    if (lane == 0) {
      // kind::tf32, fp32 accumulate, K-major A and B, M = 128; N = 2 KR (the W head and
      // tail tiles are consecutive row groups, so one B descriptor covers both) or KR
      const uint32_t idesc_hl = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * KR) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t idesc_h = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      const uint32_t winbase = smem_u32_2(sWin);
      const uint32_t plane_bytes = (uint32_t)WL * 16;
      int kk = 0, committed = 0, issued_win = 0;
      for (int d = 0; d < ndy && !*(volatile int*)&abort_flag; ++d) {
        // the window buffer is free once the MMAs of the previous group are done
        if (d > 0 && !mbar_wait2(bar(WINEMPTY), (d - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        const int gs = dy_start[d], ge = dy_start[d + 1];
        const int2 o0 = off[gs];
        const int64_t start = p0 + (int64_t)o0.y * W;  // stored index of window position 0 (= pp - CX)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar(WINFULL)), "r"((uint32_t)(2 * KC) * plane_bytes) : "memory");
        for (int h = 0; h < 2; ++h)
          for (int kc = 0; kc < KC; ++kc) {
            const int64_t plane = ((int64_t)(r * 2 + c) * 2 + h) * KC + kc;
            const float4* src = Xs + plane * PL + start;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(winbase + (uint32_t)(h * KC + kc) * plane_bytes), "l"(src), "r"(plane_bytes),
                            "r"(bar(WINFULL)) : "memory");
          }
        issued_win = d + 1;
        if (!mbar_wait2(bar(WINFULL), d & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        for (; kk < ge; ++kk) {
          const int wb = kk % TC2_WSTAGES;
          const int g = kk / TC2_GROUP, a = g & 1;
          const bool first_in_group = (kk % TC2_GROUP) == 0;
          if (first_in_group && g >= 2 && !mbar_wait2(bar(ACCEMPTY + a), ((g - 2) >> 1) & 1)) {
            atomicOr(&abort_flag, 1);
            break;
          }
          if (!mbar_wait2(bar(WFULL + wb), (kk / TC2_WSTAGES) & 1)) {
            atomicOr(&abort_flag, 1);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int dx = o0.x + (kk - gs);
          const uint32_t ashift = (uint32_t)(CX + dx) * 16;
          const uint32_t wh = smem_u32_2(sW + wb * W_STAGE);
          const uint32_t dacc = tmem + (uint32_t)(a * ACC_COLS);
#pragma unroll
          for (int s = 0; s < KR / 8; ++s) {
            const uint32_t ah = winbase + (uint32_t)(0 * KC + 2 * s) * plane_bytes + ashift;
            const uint32_t al = winbase + (uint32_t)(1 * KC + 2 * s) * plane_bytes + ashift;
            const uint64_t dAh = umma_desc2(ah, plane_bytes, 128), dAl = umma_desc2(al, plane_bytes, 128);
            const uint64_t dWh = umma_desc2(wh + s * 256, 128, KC * 128);
            const uint32_t acc0 = (!first_in_group || s > 0) ? 1u : 0u;
            // A_hi [W_hi; W_lo] (N = 2 KR), then A_lo W_hi into the first KR columns
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                         :: "r"(dacc), "l"(dAh), "l"(dWh), "r"(idesc_hl), "r"(acc0));
            asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                         :: "r"(dacc), "l"(dAl), "l"(dWh), "r"(idesc_h));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(bar(WEMPTY + wb)) : "memory");
          if ((kk % TC2_GROUP) == TC2_GROUP - 1 || kk == K - 1)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar(ACCFULL + a)) : "memory");
          committed = kk + 1;
        }
        if (*(volatile int*)&abort_flag) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(bar(WINEMPTY)) : "memory");
      }
      // drain: every MMA of this thread, and the last window copy
      if (committed > 0) {
        const int kl = committed - 1;
        if (!mbar_wait2(bar(WEMPTY + kl % TC2_WSTAGES), (kl / TC2_WSTAGES) & 1)) atomicOr(&abort_flag, 1);
      }
      if (issued_win > 0 && !mbar_wait2(bar(WINFULL), (issued_win - 1) & 1)) atomicOr(&abort_flag, 1);
      if (committed != K) atomicOr(&abort_flag, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- W loader ----------------
    if (lane == 0) {
      int issued = 0;
      for (int kk = 0; kk < K; ++kk) {
        if (*(volatile int*)&abort_flag) break;
        const int wb = kk % TC2_WSTAGES, use = kk / TC2_WSTAGES;
        if (kk >= TC2_WSTAGES && !mbar_wait2(bar(WEMPTY + wb), (use - 1) & 1)) {
          atomicOr(&abort_flag, 1);
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar(WFULL + wb)), "r"(W_STAGE) : "memory");
        const float* src = Wt + ((size_t)kk * 2 + c) * 2 * (KR * KR);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32_2(sW + wb * W_STAGE)), "l"(src), "r"(W_STAGE), "r"(bar(WFULL + wb)) : "memory");
        issued = kk + 1;
      }
      // the last copy into every stage has landed before the CTA may exit
      for (int kl = issued > TC2_WSTAGES ? issued - TC2_WSTAGES : 0; kl < issued; ++kl)
        if (!mbar_wait2(bar(WFULL + kl % TC2_WSTAGES), (kl / TC2_WSTAGES) & 1)) atomicOr(&abort_flag, 1);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---------------- readers ----------------
    const int q4 = warp & 3;
    const int m = q4 * 32 + lane;
    const int64_t pp = p0 + m;
    const int64_t iy = pp / W - CY, ix = pp % W - CX;
    const bool live = iy >= 0 && iy < ny && ix >= 0 && ix < nx;
    float accr[KR];
#pragma unroll
    for (int e = 0; e < KR; ++e) accr[e] = 0.f;
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      const int a = g & 1;
      const bool seen = __any_sync(0xffffffffu, mbar_wait2(bar(ACCFULL + a), (g >> 1) & 1));
      if (!seen) {
        ok = false;
        atomicOr(&abort_flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c0 = 0; c0 < 2 * KR; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * ACC_COLS + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                       "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int cb = c0 < KR ? c0 : c0 - KR;  // the W-tail columns add onto the same outputs
#pragma unroll
        for (int e = 0; e < 16; ++e) accr[cb + e] += __uint_as_float(v[e]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar(ACCEMPTY + a)) : "memory");
    }
    __syncwarp();
    if (ok && live) {
      const int64_t orow = (iy * nx + ix) * P + c * L;
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
static size_t tc2_smem(int CX) {
  using S = Tc2Shape<NMAX>;
  return (size_t)2 * S::KC * (128 + 2 * CX) * 16 + (size_t)TC2_WSTAGES * 2 * S::W_BYTES;
}

bool lattice_tc2_fits(int nmax, int CX) {
  size_t need = 0;
  switch (nmax) {
    case 1: need = tc2_smem<1>(CX); break;
    case 2: need = tc2_smem<2>(CX); break;
    case 3: need = tc2_smem<3>(CX); break;
    case 4: need = tc2_smem<4>(CX); break;
    default: return false;
  }
  return need + 1024 <= 227 * 1024;
}

template <int NMAX, int MODE>
static int run_tc2(tmat_ctx* ctx, const LatOp& a, const float* W, const void* x, void* y, int R_) {
  using S = Tc2Shape<NMAX>;
  const int CY = a.CY;
  const int Wd = a.nx + 2 * a.CX;
  const int64_t PP = (int64_t)(a.ny + 2 * CY) * Wd;
  const int64_t PL = PP + 2 * a.CX + 256;
  const int64_t rs = a.N * a.P;
  float4* Xs;
  TM_TRY(scratch(ctx, "tc2_Xs", sizeof(float4) * (size_t)R_ * 2 * 2 * S::KC * PL, (void**)&Xs));
  {
    const int64_t total = (int64_t)R_ * 2 * S::KC * PL;
    tc2_split_kernel<NMAX, MODE><<<(unsigned)std::min<int64_t>(cdiv(total, 256), (int64_t)ctx->num_sms * 16), 256, 0,
                                   ctx->stream>>>((const float2*)x, (const float2*)a.T, a.nx, a.ny, a.CX, CY, PL, R_,
                                                  rs, Xs);
    TM_LAUNCHED(ctx);
  }
  auto kern = lattice_tc2_kernel<NMAX, MODE>;
  const size_t smem = tc2_smem<NMAX>(a.CX);
  TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
  const int64_t rows = (int64_t)a.ny * Wd;
  dim3 grid((unsigned)cdiv(rows, 128), 2, (unsigned)R_);
  cudaEvent_t ev = timing_begin(ctx);
  kern<<<grid, TC2_THREADS, smem, ctx->stream>>>(a.off, a.K, a.dy_start, a.ndy, a.CX, CY, a.nx, a.ny, PL, Xs, W,
                                                 (const float2*)a.T, (const float2*)x, (float2*)y, rs, a.tc_err);
  TM_LAUNCHED(ctx);
  timing_end(ctx, "lattice_apply_tcv", ev);
  return TMAT_OK;
}

template <int NMAX>
static int tc2_dispatch(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  const float* W = (const float*)(mode == TMAT_OP_ADJOINT ? a.Wtc_adj : a.Wtc_fwd);
  if (mode == TMAT_OP_FORWARD) return run_tc2<NMAX, 0>(ctx, a, W, x, y, R_);
  if (mode == TMAT_OP_ADJOINT) return run_tc2<NMAX, 1>(ctx, a, W, x, y, R_);
  return run_tc2<NMAX, 2>(ctx, a, W, x, y, R_);
}

int lattice_tc2_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  switch (a.nmax) {
    case 1: return tc2_dispatch<1>(ctx, a, mode, x, y, R_);
    case 2: return tc2_dispatch<2>(ctx, a, mode, x, y, R_);
    case 3: return tc2_dispatch<3>(ctx, a, mode, x, y, R_);
    case 4: return tc2_dispatch<4>(ctx, a, mode, x, y, R_);
  }
  return set_error(ctx, TMAT_ENOTSUP, "tensor-core lattice apply supports nmax 1..4");
}

}  // namespace tmat
