// Lattice operator apply by FFT convolution.
//
// On a row-major nx x ny lattice the coupling sum y_i = sum_o B_o x_{i+o} (one block B_o
// per lattice offset o inside the cutoff, the same blocks the direct kernels use) is a
// 2-D correlation of the source field with the offset blocks. With b(p) = B(-p) it is the
// circular convolution y = b (*) x on an Mx x My grid, exact (no wrap-around) for
// Mx >= nx + CX and My >= ny + CY, CX/CY the largest |dx|/|dy| of the offsets, and the
// zero-padded sources. In Fourier space it is one L x L block product per frequency and
// class: Y(f) = B^(f) X(f). The work is O(Mx My L^2) for the products plus FFTs of the
// 2 L components of every RHS, against O(N K L^2) for the direct sum (K offsets).
//
// Data flow (every array component-major, rows contiguous):
//   embed   x[r][site][u] (times T for the adjoint)  -> Xc[r*P+u][iy][ix]      (ny x nx)
//   F1      FFT along ix (zero-padded to Mx), write transposed -> T1[.][kx][iy]  (Mx x ny)
//   F2      FFT along iy (zero-padded to My)               -> X^[.][kx][ky]   (Mx x My)
//   mul     per frequency and class: Y^[u] = sum_u' B^[c][u][u'] X^[u']   (adjoint: the
//           transposed blocks at -f, since A^T has blocks B_{-o}^T)
//   I2      inverse FFT along ky, keep iy < ny, write transposed -> T3[.][iy][kx]
//   I1      inverse FFT along kx, keep ix < nx               -> Yc[.][iy][ix]
//   extract y[r][site][u] = x - T (Yc / (Mx My)), x - Yc / (Mx My) or Yc / (Mx My)
// B^ is built once per operator by the same F1/F2 passes from the blocks scattered to a
// compact (2 CY + 1) x (2 CX + 1) grid at (CX - dx, CY - dy), i.e. position -o shifted (the
// shift is a phase factor, removed after the transform); only the rows that hold offsets
// are transformed along x. The FFT is an iterative decimation in time in shared memory
// (Cooley and Tukey, Math. Comp. 19 (1965)): radix-16 register passes, then radix 4 (one
// radix-2 stage first for odd powers of two), fp64 twiddles (cast for complex64).
#include <cmath>
#include <type_traits>
#include <string>
#include <vector>

#include "dev.cuh"
#include "dfloat.cuh"
#include "solver.h"

namespace tmat {

constexpr int FFT_MAXLEN = 1024;     // longest row transform
constexpr int FFT_THREADS = 256;
constexpr int FFT_SMEM_POINTS = 8192;  // complex points staged per block
constexpr int FFT_LOAD_BATCH = 8;

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
static int pow2_at_least(int v) { return 1 << ilog2(std::max(1, v)); }

// tw[k] = exp(-2 pi i k / FFT_MAXLEN), k < FFT_MAXLEN / 2, in fp64
static int fft_twiddles(tmat_ctx* ctx, const double2** out) {
  double2* tw;
  bool fresh = ctx->bufs.find("fft_tw") == ctx->bufs.end();
  TM_TRY(scratch(ctx, "fft_tw", sizeof(double2) * (FFT_MAXLEN / 2), (void**)&tw));
  if (fresh) {
    std::vector<double2> h(FFT_MAXLEN / 2);
    for (int k = 0; k < FFT_MAXLEN / 2; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)FFT_MAXLEN;
      h[k] = make_double2(cos(a), -sin(a));
    }
    TM_CUDA(ctx, cudaMemcpyAsync(tw, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  *out = tw;
  return TMAT_OK;
}

// Row transforms. Data [batch][rows][cols], cols contiguous with pitch in_pitch, cin
// valid columns (zero beyond, up to the length len = 2^lg). Rows [0, nrows) of every
// batch. Output: natural out[b][row][k] (pitch out_pitch, k < cout), or transposed
// out[b][k][row] (pitch out_pitch over rows, k < cout). dir = -1 forward, +1 inverse
// (unnormalised). One block handles rb = 2^lgrb rows of one batch; the rows sit in
// shared memory padded (one slot per 16 values, plus one per row) so that the transposed read-out, where
// consecutive threads take consecutive rows, spreads over the banks; the twiddles of
// this length are staged in shared memory too.
// shared-memory position of element i of a row: one pad slot after every 16 values, so
// the power-of-two strides of the butterflies and of the bit-reversed stores fall on
// different banks
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// Twiddle table by stage: wt[2^t - 1 + j] = W_{2^(t+1)}^j (j < 2^t, t < lg; W = e^{-+2 pi i/n}
// for dir -/+), len - 1 entries, so that the threads of one stage read consecutive entries.
template <typename R>
__device__ __forceinline__ void fft_stage_twiddles(C<R>* wt, int lg, int dir, const double2* __restrict__ tw) {
  for (int e = threadIdx.x; e < (1 << lg) - 1; e += blockDim.x) {
    const int t = 31 - __clz(e + 1), j = e + 1 - (1 << t);
    const double2 w64 = tw[j << (9 - t)];  // exp(-2 pi i j / 2^(t+1)); FFT_MAXLEN = 2^10
    wt[e] = cfrom64<R>(w64.x, dir < 0 ? w64.y : -w64.y);
  }
}

// The butterfly passes of a decimation-in-time transform of nrows rows of length 2^lg
// held in shared memory in bit-reversed order (row stride pitch, element i at fpad(i)),
// stage twiddles wt of the direction dir. Stages go four at a time through registers
// (radix 16: each thread loads 16 elements i0 + j 2^s, runs stages s..s+3 among them and
// stores them back), then two at a time (radix 4), with one radix-2 stage first for odd
// lg: a length-256 row makes two round trips through shared memory instead of four.
// Ends with a block barrier.
template <typename R>
__device__ __forceinline__ void fft_smem_passes(C<R>* a, int pitch, int nrows, int lg, const C<R>* wt, int dir) {
  const int len = 1 << lg;
  int s = 0;
  if (lg & 1) {  // one radix-2 stage (twiddle 1) when the length is an odd power of two
    for (int e = threadIdx.x; e < (nrows << (lg - 1)); e += blockDim.x) {
      const int rr = e >> (lg - 1), p = e & ((len >> 1) - 1);
      C<R>* row = a + rr * pitch;
      const int q0 = fpad(2 * p), q1 = fpad(2 * p + 1);
      const C<R> u = row[q0], t = row[q1];
      row[q0] = cadd(u, t);
      row[q1] = csub(u, t);
    }
    __syncthreads();
    s = 1;
  }
  for (; s + 3 < lg; s += 4) {
    const int lgg = lg - 4;  // groups of 16 per row
    for (int e = threadIdx.x; e < (nrows << lgg); e += blockDim.x) {
      const int rr = e >> lgg, g = e & ((1 << lgg) - 1);
      const int lo = g & ((1 << s) - 1);
      const int i0 = ((g >> s) << (s + 4)) + lo;
      C<R>* row = a + rr * pitch;
      C<R> v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = row[fpad(i0 + (j << s))];
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int h = 1 << tt;
        // stage t = s + tt: element i0 + (j << s) pairs with j + h; twiddle W_{2^(t+1)}^(i mod 2^t)
        const C<R>* wst = wt + ((1 << (s + tt)) - 1) + lo;
#pragma unroll
        for (int m = 0; m < h; ++m) {
          const C<R> w = wst[m << s];
#pragma unroll
          for (int blk = 0; blk < 16; blk += 2 * h) {
            const C<R> t = cmul(w, v[blk + m + h]);
            v[blk + m + h] = csub(v[blk + m], t);
            v[blk + m] = cadd(v[blk + m], t);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) row[fpad(i0 + (j << s))] = v[j];
    }
    __syncthreads();
  }
  // radix-4: the radix-2 stages s and s + 1 fused in registers (twiddles W_{2h}^j for the
  // first, W_{4h}^j and W_{4h}^{j+h} = W_{4h}^j (-/+ i) for the second)
  for (; s + 1 < lg; s += 2) {
    const int half = 1 << s;
    for (int e = threadIdx.x; e < (nrows << (lg - 2)); e += blockDim.x) {
      const int rr = e >> (lg - 2), p = e & ((len >> 2) - 1);
      const int j = p & (half - 1);
      const int i0 = ((p >> s) << (s + 2)) + j;
      C<R>* row = a + rr * pitch;
      const int q0 = fpad(i0), q1 = fpad(i0 + half), q2 = fpad(i0 + 2 * half), q3 = fpad(i0 + 3 * half);
      const C<R> w1 = wt[half - 1 + j], w2 = wt[2 * half - 1 + j];
      const C<R> a0 = row[q0], a1 = cmul(w1, row[q1]);
      const C<R> a2 = row[q2], a3 = cmul(w1, row[q3]);
      const C<R> b0 = cadd(a0, a1), b1 = csub(a0, a1), b2 = cadd(a2, a3), b3 = csub(a2, a3);
      const C<R> t2 = cmul(w2, b2);
      C<R> t3 = cmul(w2, b3);
      t3 = crot<R>(t3, dir);  // times -i (forward) or +i (inverse)
      row[q0] = cadd(b0, t2);
      row[q2] = csub(b0, t2);
      row[q1] = cadd(b1, t3);
      row[q3] = csub(b1, t3);
    }
    __syncthreads();
  }
}

// Element formats of a transform's global arrays: complex64 transforms read and write
// float2; double-float ones read complex128 (double2, split on load) or double-float pairs
// (dfc, the format of their intermediates and spectra: no conversion) and write either.
template <typename R, typename GT> struct FftIo;
template <> struct FftIo<float, float2> {
  static __device__ __forceinline__ float2 ld(float2 v) { return v; }
  static __device__ __forceinline__ float2 st(float2 v) { return v; }
};
template <> struct FftIo<DF, double2> {
  static __device__ __forceinline__ dfc ld(double2 v) { return gload<DF>(v); }
  static __device__ __forceinline__ double2 st(dfc v) { return gstore<DF>(v); }
};
template <> struct FftIo<DF, dfc> {
  static __device__ __forceinline__ dfc ld(dfc v) { return v; }
  static __device__ __forceinline__ dfc st(dfc v) { return v; }
};
// the double-float storage format of a compute type (complex64 transforms: float2)
template <typename R> struct fft_store { using t = C<R>; };

template <typename T> __device__ __forceinline__ T cneg(T a) { a.x = -a.x; a.y = -a.y; return a; }
__device__ __forceinline__ dfc cneg(dfc a) { return dfc{-a.rh, -a.rl, -a.ih, -a.il}; }

template <typename R, bool TOUT, bool TIN, typename GI = G<R>, typename GO = G<R>>
__global__ void __launch_bounds__(FFT_THREADS, sizeof(C<R>) == 8 ? 4 : 2)
fft_rows_kernel(const GI* __restrict__ in, int64_t in_batch_stride, int in_pitch, int cin, int nrows,
                GO* __restrict__ out, int64_t out_batch_stride, int out_pitch, int cout, int lg, int lgrb, int dir,
                const double2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int len = 1 << lg, rb = 1 << lgrb, pitch = len + (len >> 4) + 1;
  C<R>* a = reinterpret_cast<C<R>*>(fsm);
  C<R>* ws = a + (size_t)rb * pitch;  // [len - 1] stage twiddles
  const int b = blockIdx.y;
  const int row0 = blockIdx.x << lgrb;
  const int nr = min(rb, nrows - row0);
  fft_stage_twiddles<R>(ws, lg, dir, tw);
  // load with bit reversal (zero-padded)
  // FFT_LOAD_BATCH independent loads per thread are issued before their shared-memory
  // stores, so the load latency is paid once per batch rather than once per element
  if (TIN) {
    // in[k][row0 + rr] (transposed input): consecutive threads take consecutive rows of one k
    const GI* src = in + (int64_t)b * in_batch_stride + row0;
    const int rr = threadIdx.x & (rb - 1), step = blockDim.x >> lgrb;
    for (int c0 = threadIdx.x >> lgrb; c0 < len; c0 += step * FFT_LOAD_BATCH) {
      C<R> v[FFT_LOAD_BATCH];
#pragma unroll
      for (int t = 0; t < FFT_LOAD_BATCH; ++t) {
        const int cc = c0 + t * step;
        v[t] = (rr < nr && cc < cin) ? FftIo<R, GI>::ld(src[(int64_t)cc * in_pitch + rr]) : czero<R>();
      }
#pragma unroll
      for (int t = 0; t < FFT_LOAD_BATCH; ++t) {
        const int cc = c0 + t * step;
        if (cc < len) a[rr * pitch + fpad(lg ? (int)(__brev((unsigned)cc) >> (32 - lg)) : 0)] = v[t];
      }
    }
  } else {
    const GI* src = in + (int64_t)b * in_batch_stride + (int64_t)row0 * in_pitch;
    const int total = rb << lg;
    for (int e0 = threadIdx.x; e0 < total; e0 += blockDim.x * FFT_LOAD_BATCH) {
      C<R> v[FFT_LOAD_BATCH];
#pragma unroll
      for (int t = 0; t < FFT_LOAD_BATCH; ++t) {
        const int e = e0 + t * (int)blockDim.x;
        const int rr = e >> lg, cc = e & (len - 1);
        v[t] = (e < total && rr < nr && cc < cin) ? FftIo<R, GI>::ld(src[(int64_t)rr * in_pitch + cc]) : czero<R>();
      }
#pragma unroll
      for (int t = 0; t < FFT_LOAD_BATCH; ++t) {
        const int e = e0 + t * (int)blockDim.x;
        const int rr = e >> lg, cc = e & (len - 1);
        if (e < total) a[rr * pitch + fpad(lg ? (int)(__brev((unsigned)cc) >> (32 - lg)) : 0)] = v[t];
      }
    }
  }
  __syncthreads();
  fft_smem_passes<R>(a, pitch, rb, lg, ws, dir);
  GO* dst = out + (int64_t)b * out_batch_stride;
  if (TOUT) {
    // out[k][row0 + rr]: consecutive threads take consecutive rows of one k
    const int rr = threadIdx.x & (rb - 1);
    for (int k = threadIdx.x >> lgrb; k < cout; k += blockDim.x >> lgrb)
      if (rr < nr) dst[(int64_t)k * out_pitch + row0 + rr] = FftIo<R, GO>::st(a[rr * pitch + fpad(k)]);
  } else {
    for (int rr = 0; rr < nr; ++rr)
      for (int k = threadIdx.x; k < cout; k += blockDim.x)
        dst[(int64_t)(row0 + rr) * out_pitch + k] = FftIo<R, GO>::st(a[rr * pitch + fpad(k)]);
  }
}


// ---- 256-point rows of the complex64 operators: four-step 16 x 16 ------------------------
// X[k1 + 16 k2] = sum_a W256^(a k1) W16^(a k2) [sum_b x[a + 16 b] W16^(b k1)]: the 16 threads
// of a row hold x[a + 16 b] (thread a, b = 0..15), take a 16-point DFT in registers,
// multiply by W256^(a k1), exchange through shared memory within their half-warp and take
// the second 16-point DFT; thread k1 ends with X[k1 + 16 k2]. One global load and one
// store per value, no bit reversal, one shared-memory round trip (the generic kernel
// makes three). 16 rows per block of 256 threads. W[m] = W256^m of the direction (forward
// e^{-2 pi i m / 256}, inverse its conjugate).
// radix-4 butterfly and 16-point DFT in registers, for complex64 (CR = float) and
// double-float (CR = DF) values
template <typename CR>
__device__ __forceinline__ void fft_dft4(C<CR>& a, C<CR>& b, C<CR>& c, C<CR>& d, int dir) {
  const C<CR> t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = crot<CR>(csub(b, d), dir);
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}
template <typename CR>
__device__ __forceinline__ void fft_dft16(C<CR> (&v)[16], const C<CR>* W, int dir) {
  // n = n1 + 4 n2: DFT4 over n2 for each n1 (outputs k' = 0..3 in place of n2)
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) fft_dft4<CR>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12], dir);
  // twiddles W16^(n1 k')
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int kp = 1; kp < 4; ++kp) v[n1 + 4 * kp] = cmul(v[n1 + 4 * kp], W[16 * n1 * kp]);
  // DFT4 over n1 for each k': X[k' + 4 k2] lands at position 4 k' + k2
#pragma unroll
  for (int kp = 0; kp < 4; ++kp) fft_dft4<CR>(v[4 * kp], v[4 * kp + 1], v[4 * kp + 2], v[4 * kp + 3], dir);
  // reorder position 4 k' + k2 -> index k' + 4 k2 (a fixed permutation of registers)
  C<CR> o[16];
#pragma unroll
  for (int kp = 0; kp < 4; ++kp)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) o[kp + 4 * k2] = v[4 * kp + k2];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = o[k];
}


constexpr int F256_RS = 16 * 17;  // exchange stride of a row (k1 blocks of 17)
constexpr int F256_OS = 257;      // staging stride of a row for transposed stores

// CR = float: complex64; CR = DF: double-float arithmetic with complex128 (G) or double-float
// storage (IN_S / OUT_S) in global memory, as in the passes below.
template <typename CR> struct F256RowsSmem {
  static constexpr size_t BYTES = sizeof(C<CR>) * (256 + 16 * F256_RS);
};
template <typename CR, bool TOUT, bool IN_S, bool OUT_S>
__global__ void __launch_bounds__(256, std::is_same_v<CR, float> ? 4 : 2)
fft256_rows_kernel(const std::conditional_t<IN_S, C<CR>, G<CR>>* __restrict__ in, int64_t in_batch_stride,
                   int in_pitch, int cin, int nrows, std::conditional_t<OUT_S, C<CR>, G<CR>>* __restrict__ out,
                   int64_t out_batch_stride, int out_pitch, int cout, int dir, const double2* __restrict__ tw) {
  using CT = C<CR>;
  extern __shared__ __align__(16) unsigned char f256r_sm[];
  CT* W = reinterpret_cast<CT*>(f256r_sm);
  CT* ex = W + 256;  // exchange, then (TOUT) the output staging [16][257]
  static_assert(16 * F256_OS <= 16 * F256_RS, "staging fits the exchange buffer");
  const int b = blockIdx.y;
  const int row0 = blockIdx.x * 16;
  const int rr = threadIdx.x >> 4, a = threadIdx.x & 15;
  for (int m = threadIdx.x; m < 256; m += blockDim.x) {
    // W256^m = tw[4 m] (m < 128), -tw[4 (m - 128)] (m >= 128), tw = e^{-2 pi i k / 1024}
    const double2 t = tw[4 * (m & 127)];
    if constexpr (std::is_same_v<CR, float>) {
      const float sg = m < 128 ? 1.f : -1.f;
      W[m] = make_float2(sg * (float)t.x, sg * (dir < 0 ? (float)t.y : -(float)t.y));
    } else {
      const CT w = cfrom64<CR>(t.x, dir < 0 ? t.y : -t.y);
      W[m] = m < 128 ? w : cneg(w);
    }
  }
  const int row = row0 + rr;
  const bool live = row < nrows;
  CT v[16];
  const auto* src = in + (int64_t)b * in_batch_stride + (int64_t)row * in_pitch;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int c = a + 16 * q;
    if (live && c < cin) {
      if constexpr (IN_S) v[q] = src[c];
      else v[q] = gload<CR>(src[c]);
    } else {
      v[q] = czero<CR>();
    }
  }
  __syncthreads();  // W
  fft_dft16<CR>(v, W, dir);  // v[k1] = Y[a][k1]
  CT* exr = ex + rr * F256_RS;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) exr[k1 * 17 + a] = k1 ? cmul(v[k1], W[(a * k1) & 255]) : v[k1];
  __syncwarp();
  const int k1 = a;  // this thread now owns column k1: Y[a'][k1] for a' = 0..15
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = exr[k1 * 17 + q];
  fft_dft16<CR>(v, W, dir);  // v[k2] = X[k1 + 16 k2]
  auto* dst = out + (int64_t)b * out_batch_stride;
  auto put = [&](int64_t o, const CT& z) {
    if constexpr (OUT_S) dst[o] = z;
    else dst[o] = gstore<CR>(z);
  };
  if (TOUT) {
    __syncthreads();  // every row's exchange reads are done before the staging overwrites
    CT* st = ex + rr * F256_OS;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) st[k1 + 16 * k2] = v[k2];
    __syncthreads();
    // out[k][row0 + r]: consecutive threads take consecutive rows of one k
    const int r = threadIdx.x & 15, nr = min(16, nrows - row0);
    for (int k = threadIdx.x >> 4; k < cout; k += 16)
      if (r < nr) put((int64_t)k * out_pitch + row0 + r, ex[r * F256_OS + k]);
  } else if (live) {
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      const int k = k1 + 16 * k2;
      if (k < cout) put((int64_t)row * out_pitch + k, v[k2]);
    }
  }
}


// ---- 256 x 256 transforms without transposes -------------------------------------------
// Every pass takes blocks of 16 consecutive components c of one right-hand side r and one
// line: a row of the pass is (r, c, line) with elements at
//   r rstride + c cstride + line lstride + col estride,
// and its outputs go to the same form of the output array. Layouts whose components are
// innermost (cstride 1: x, y and the intermediates [r][line][col][P]) are read and written
// with consecutive threads on consecutive components; component-major ones (the spectra
// [r P + c][kx][ky]) with consecutive threads along a row. The first forward pass reads x
// (T x for the adjoint) in place and the last inverse pass writes y = x - T s (or x - s, s)
// in place, so the operator needs no embed or extract kernels. CR = float: complex64
// throughout; CR = DF: x, y and T complex128, the intermediates and spectra double-float
// pairs (IN_S / OUT_S: the input / output is in that storage form), arithmetic in
// double-float.
struct F256Lay {
  int64_t rstride, cstride, lstride, estride;
};
constexpr int F256_RS2 = 16 * 17 + 1;  // exchange stride of a row (odd: conflict-free in both mappings)

// The complex64 EXT 0 pass stages its x and T elements in shared memory with cp.async before
// the transform (x into a buffer of 16 x 256 values at the start, T into the exchange buffer
// once it is free), so the epilogue does not wait on global loads; slot k2 * 256 + thread of
// either buffer is read by the thread that copied it.
__device__ __forceinline__ void f256_cp8(float2* dst, const float2* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
template <typename CR, int EXT> struct F256Smem {
  static constexpr bool PF = EXT == 0 && std::is_same_v<CR, float>;
  static constexpr size_t W_BYTES = 256 * sizeof(C<CR>);
  static constexpr size_t EX_BYTES = 16 * F256_RS2 * sizeof(C<CR>);
  static constexpr size_t BYTES = W_BYTES + EX_BYTES + (PF ? sizeof(float2) * 16 * 256 : 0);
  static constexpr int MIN_BLOCKS = std::is_same_v<CR, float> ? (EXT == 0 ? 3 : 4) : 2;
};
template <typename CR> __device__ __forceinline__ C<CR> f256_scale(C<CR> v, float s) { return cscale(v, s); }
template <> __device__ __forceinline__ dfc f256_scale<DF>(dfc v, float s) { return cscale_df(v, s, 0.f); }

// EMB: 0 plain input, 2 input times T (same layout, T's RHS stride tstride); EXT: -1 plain
// output, 0 y = x - T s, 1 y = x - s, 2 y = s with s = scale * value (x, T in the output's layout)
template <typename CR, bool IN_CI, bool OUT_CI, int EMB, int EXT, bool IN_S, bool OUT_S>
__global__ void __launch_bounds__(256, F256Smem<CR, EXT>::MIN_BLOCKS)
fft256_ci_kernel(const std::conditional_t<IN_S, C<CR>, G<CR>>* __restrict__ in, F256Lay li, int cin,
                 std::conditional_t<OUT_S, C<CR>, G<CR>>* __restrict__ out, F256Lay lo, int cout, int P, int dir,
                 const double2* __restrict__ tw, const G<CR>* __restrict__ T, int64_t tstride,
                 const G<CR>* __restrict__ xs, float scale) {
  pdl_wait();
  using CT = C<CR>;
  using SM = F256Smem<CR, EXT>;
  static_assert(EXT != 0 || OUT_CI, "the staged epilogue assumes the component-innermost output mapping");
  extern __shared__ __align__(16) unsigned char f256_sm[];
  CT* W = reinterpret_cast<CT*>(f256_sm);
  CT* ex = reinterpret_cast<CT*>(f256_sm + SM::W_BYTES);
  float2* pf = reinterpret_cast<float2*>(f256_sm + SM::W_BYTES + SM::EX_BYTES);  // x (staged pass)
  const int line = blockIdx.x;
  const int r = blockIdx.z;
  const int c0 = blockIdx.y * 16;
  // output-side indexing of the second half (thread: row rr, column k1)
  const int rr_o = OUT_CI ? (threadIdx.x & 15) : (threadIdx.x >> 4);
  const int k1_o = OUT_CI ? (threadIdx.x >> 4) : (threadIdx.x & 15);
  const int64_t obase =
      (int64_t)r * lo.rstride + (int64_t)(c0 + rr_o) * lo.cstride + (int64_t)line * lo.lstride;
  if constexpr (SM::PF) {
    if (c0 + rr_o < P) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int k = k1_o + 16 * k2;
        if (k < cout)
          f256_cp8(pf + k2 * 256 + threadIdx.x, reinterpret_cast<const float2*>(xs) + obase + (int64_t)k * lo.estride);
      }
    }
  }
  for (int m = threadIdx.x; m < 256; m += blockDim.x) {
    const double2 t = tw[4 * (m & 127)];
    if constexpr (std::is_same_v<CR, float>) {  // no fp64 arithmetic in the complex64 passes
      const float sg = m < 128 ? 1.f : -1.f;
      W[m] = make_float2(sg * (float)t.x, sg * (dir < 0 ? (float)t.y : -(float)t.y));
    } else {
      const C<CR> w = cfrom64<CR>(t.x, dir < 0 ? t.y : -t.y);  // exact negation below
      W[m] = m < 128 ? w : cneg(w);
    }
  }
  // first half: thread (row rr, column a) holds x[a + 16 b]
  {
    const int rr = IN_CI ? (threadIdx.x & 15) : (threadIdx.x >> 4);
    const int a = IN_CI ? (threadIdx.x >> 4) : (threadIdx.x & 15);
    const int c = c0 + rr;
    const bool live = c < P;
    const int64_t base = (int64_t)r * li.rstride + (int64_t)c * li.cstride + (int64_t)line * li.lstride;
    CT v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = a + 16 * q;
      CT e = czero<CR>();
      if (live && col < cin) {
        const int64_t o = base + (int64_t)col * li.estride;
        if constexpr (IN_S) e = in[o];
        else e = gload<CR>(in[o]);
        if (EMB == 2) e = cmul(gload<CR>(T[(int64_t)r * tstride + o - (int64_t)r * li.rstride]), e);
      }
      v[q] = e;
    }
    __syncthreads();  // W
    fft_dft16<CR>(v, W, dir);
    CT* exr = ex + rr * F256_RS2;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) exr[k1 * 17 + a] = k1 ? cmul(v[k1], W[(a * k1) & 255]) : v[k1];
  }
  __syncthreads();
  // second half: thread (row rr, k1) owns X[k1 + 16 k2]
  const int rr = rr_o;
  const int k1 = k1_o;
  CT v[16];
  const CT* exr = ex + rr * F256_RS2;
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = exr[k1 * 17 + q];
  const int c = c0 + rr;
  if constexpr (SM::PF) {
    __syncthreads();  // every row has left the exchange buffer
    if (c < P) {
      const float2* Tr = reinterpret_cast<const float2*>(T) + (int64_t)r * tstride - (int64_t)r * lo.rstride;
      float2* ts = reinterpret_cast<float2*>(ex);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int k = k1 + 16 * k2;
        if (k < cout) f256_cp8(ts + k2 * 256 + threadIdx.x, Tr + obase + (int64_t)k * lo.estride);
      }
    }
  }
  fft_dft16<CR>(v, W, dir);
  if (c >= P) return;
  if constexpr (SM::PF) asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const int k = k1 + 16 * k2;
    if (k >= cout) continue;
    const int64_t o = obase + (int64_t)k * lo.estride;
    CT res;
    if constexpr (EXT < 0) {
      res = v[k2];
    } else {
      const CT s = f256_scale<CR>(v[k2], scale);
      if constexpr (EXT == 2) {
        res = s;
      } else if constexpr (EXT == 1) {
        res = csub(gload<CR>(xs[o]), s);
      } else if constexpr (SM::PF) {
        const float2* ts = reinterpret_cast<const float2*>(ex);
        res = csub(pf[k2 * 256 + threadIdx.x], cmul(ts[k2 * 256 + threadIdx.x], s));
      } else {
        res = csub(gload<CR>(xs[o]), cmul(gload<CR>(T[(int64_t)r * tstride + o - (int64_t)r * lo.rstride]), s));
      }
    }
    if constexpr (OUT_S) out[o] = res;
    else out[o] = gstore<CR>(res);
  }
}

// complex64 transforms compute in fp32; complex128 ones in double-float (see above)
template <typename R> struct fft_compute { using t = R; };
template <> struct fft_compute<double> { using t = DF; };

// IN_S / OUT_S: the input / output is in the transform's storage format (double-float pairs
// for complex128 transforms; complex64 ones use float2 either way)
template <typename R, bool TOUT, bool TIN = false, bool IN_S = false, bool OUT_S = false>
static int fft_rows(tmat_ctx* ctx, const C<R>* in, int64_t in_bs, int in_pitch, int cin, int nrows, C<R>* out,
                    int64_t out_bs, int out_pitch, int cout, int len, int64_t nbatch, int dir, const double2* tw) {
  using CR = typename fft_compute<R>::t;
  using GI = std::conditional_t<IN_S, C<CR>, G<CR>>;
  using GO = std::conditional_t<OUT_S, C<CR>, G<CR>>;
  static_assert(sizeof(G<CR>) == sizeof(C<R>) && sizeof(C<CR>) == sizeof(C<R>), "global element type");
  if constexpr (!TIN) {
    if (len == 256) {  // 256-point rows: the four-step kernel (complex64 or double-float)
      auto kern = fft256_rows_kernel<CR, TOUT, IN_S, OUT_S>;
      const size_t sm = F256RowsSmem<CR>::BYTES;
      if (sm > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, sm));
      for (int64_t b0 = 0; b0 < nbatch; b0 += 65535) {
        const int nb = (int)std::min<int64_t>(65535, nbatch - b0);
        dim3 grid((unsigned)cdiv(nrows, 16), (unsigned)nb);
        kern<<<grid, 256, sm, ctx->stream>>>((const GI*)(in + b0 * in_bs), in_bs, in_pitch, cin, nrows,
                                             (GO*)(out + b0 * out_bs), out_bs, out_pitch, cout, dir, tw);
        TM_LAUNCHED(ctx);
      }
      return TMAT_OK;
    }
  }
  const int lg = ilog2(len);
  int lgrb = ilog2(std::max(1, std::min((TOUT || TIN) ? 16 : 8, FFT_SMEM_POINTS / len)));
  const int rb = 1 << lgrb;
  const size_t smem = sizeof(C<CR>) * ((size_t)rb * (len + (len >> 4) + 1) + len);
  auto kern = fft_rows_kernel<CR, TOUT, TIN, GI, GO>;
  if (smem > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
  for (int64_t b0 = 0; b0 < nbatch; b0 += 65535) {
    const int nb = (int)std::min<int64_t>(65535, nbatch - b0);
    dim3 grid((unsigned)cdiv(nrows, rb), (unsigned)nb);
    kern<<<grid, FFT_THREADS, smem, ctx->stream>>>((const GI*)(in + b0 * in_bs), in_bs, in_pitch, cin, nrows,
                                                   (GO*)(out + b0 * out_bs), out_bs, out_pitch, cout, lg, lgrb, dir,
                                                   tw);
    TM_LAUNCHED(ctx);
  }
  return TMAT_OK;
}

// Xc[r*P + u][iy][ix] = x[r][iy*nx + ix][u] (MODE 1: times T[site][u]); a 32 x 32 tile
// transpose through shared memory (sites along ix x components).
template <typename R, int MODE>
__global__ void fft_embed_kernel(const C<R>* __restrict__ x, const C<R>* __restrict__ T, int nx, int ny, int P, int R_,
                                 C<R>* __restrict__ Xc, int64_t tstride) {
  __shared__ C<R> tile[32][33];
  const int ix0 = blockIdx.x * 32, iy = blockIdx.y;
  const int r = blockIdx.z / ((P + 31) / 32), u0 = (blockIdx.z % ((P + 31) / 32)) * 32;
  const int64_t N = (int64_t)nx * ny;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int ix = ix0 + q, u = u0 + threadIdx.x;
    C<R> v = mk<R>((R)0, (R)0);
    if (ix < nx && u < P) {
      const int64_t site = (int64_t)iy * nx + ix;
      v = x[((int64_t)r * N + site) * P + u];
      if (MODE == 1) v = cmul(T[r * tstride + site * P + u], v);
    }
    tile[q][threadIdx.x] = v;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int u = u0 + q, ix = ix0 + threadIdx.x;
    if (u < P && ix < nx) Xc[(((int64_t)r * P + u) * ny + iy) * nx + ix] = tile[threadIdx.x][q];
  }
}

// y[r][site][u] from Yc[r*P + u][iy][ix] scaled by 1/(Mx My): MODE 0 y = x - T Yc',
// MODE 1 y = x - Yc', MODE 2 y = Yc'
template <typename R, int MODE>
__global__ void fft_extract_kernel(const C<R>* __restrict__ Yc, const C<R>* __restrict__ x, const C<R>* __restrict__ T,
                                   int nx, int ny, int P, R scale, C<R>* __restrict__ y, int64_t tstride) {
  __shared__ C<R> tile[32][33];
  const int ix0 = blockIdx.x * 32, iy = blockIdx.y;
  const int r = blockIdx.z / ((P + 31) / 32), u0 = (blockIdx.z % ((P + 31) / 32)) * 32;
  const int64_t N = (int64_t)nx * ny;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int u = u0 + q, ix = ix0 + threadIdx.x;
    C<R> v = mk<R>((R)0, (R)0);
    if (u < P && ix < nx) v = Yc[(((int64_t)r * P + u) * ny + iy) * nx + ix];
    tile[q][threadIdx.x] = v;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int ix = ix0 + q, u = u0 + threadIdx.x;
    if (ix < nx && u < P) {
      const int64_t site = (int64_t)iy * nx + ix;
      const int64_t o = ((int64_t)r * N + site) * P + u;
      const C<R> a = cscale(tile[threadIdx.x][q], scale);
      C<R> out;
      if (MODE == 2) {
        out = a;
      } else if (MODE == 0) {
        out = csub(x[o], cmul(T[r * tstride + site * P + u], a));
      } else {
        out = csub(x[o], a);
      }
      y[o] = out;
    }
  }
}

// Bgrid[(c*L + u)*L + u'][iy][ix] = B_o[c][u][u'] (BT[o][c][u'][u] holds the blocks
// transposed, row stride LP) on compact grids: offset o goes to (CX - dx, CY - dy) of a
// (2 CY + 1) x (2 CX + 1) grid, i.e. b(-o) shifted by (CX, CY); the transforms zero-pad it
// to Mx x My and the shift becomes the phase e^{-2 pi i (kx CX / Mx + ky CY / My)}, which
// the block product removes per frequency.
template <typename R>
__global__ void fft_scatter_blocks_kernel(const C<R>* __restrict__ BT, const int2* __restrict__ off, int K, int L, int LP,
                                          int CX, int CY, C<R>* __restrict__ Bgrid) {
  const int o = blockIdx.x;
  if (o >= K) return;
  const int2 d = off[o];
  const int gw = 2 * CX + 1, gh = 2 * CY + 1;
  const int ix = CX - d.x, iy = CY - d.y;
  const int64_t G = (int64_t)gw * gh;
  for (int e = threadIdx.x; e < 2 * L * L; e += blockDim.x) {
    const int c = e / (L * L), u = (e / L) % L, up = e % L;
    Bgrid[(int64_t)e * G + (int64_t)iy * gw + ix] = BT[(((int64_t)o * 2 + c) * L + up) * LP + u];
  }
}

// Per frequency f and class c: Y^[r][c L + u][f] = sum_u' G[u][u'] X^[r][c L + u'][f] with
// G = B^[c][u][u'][f] (MODE 0, 2) or B^[c][u'][u][-f] (MODE 1). RC RHS per pass share
// the B^ loads.
// Mirror pairs: the blocks obey B_(dx,-dy) = D J B_(dx,dy) J D (J: the m -> -m partner in
// the class, D = diag((-1)^p); the offset set and the window are symmetric in dy), hence
// B^(kx, -ky) = D J B^(kx, ky) J D for the true spectra (times msign = -1 for blocks that
// are odd in dy, such as their dy-derivatives), and for the adjoint's B^(-f)^T the
// same with -f. One read of G at f1 = (kx, ky) therefore serves f2 = (kx, -ky):
//   Y^(f1) = ph G X^(f1),   Y^(f2)[J u] = ph D[u] (G w)[u],  w[v] = D[v] X^(f2)[J v],
// ph the phase of f1 (or -f1) that undoes the compact-grid shift. A thread takes one item
// (kx, ky <= My / 2) of one class; ky = 0 and My / 2 are their own mirror. The thread's X^
// values sit in its own column of shared memory, not in registers.
constexpr int FFT_MUL_THREADS = 128;
template <typename R, int L, int MODE, int RC>
__global__ void __launch_bounds__(FFT_MUL_THREADS, 2)
fft_mul_kernel(const C<R>* __restrict__ Bh, const C<R>* __restrict__ Xh, C<R>* __restrict__ Yh, int Mx, int My,
               int R_, int CX, int CY, const int* __restrict__ mirror, int msign, int64_t bstride) {
  constexpr int P = 2 * L, TS = FFT_MUL_THREADS;
  extern __shared__ __align__(16) unsigned char xsm[];
  C<R>* x1 = reinterpret_cast<C<R>*>(xsm) + threadIdx.x;  // [RC][L][TS]: X^(f1), this thread's column
  C<R>* x2 = x1 + RC * L * TS;                             // [RC][L][TS]: w of f2
  const int64_t F = (int64_t)Mx * My;
  const int hy = My >= 2 ? My / 2 + 1 : 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (t >= (int64_t)Mx * hy) return;  // no block barrier below
  const int kx0 = (int)(t / hy), ky0 = (int)(t % hy);
  const int64_t f1 = (int64_t)kx0 * My + ky0, f2 = (int64_t)kx0 * My + (My - ky0) % My;
  const bool pair = f2 != f1;
  int64_t fb = f1;
  int kx = kx0, ky = ky0;
  if (MODE == 1) {
    kx = (Mx - kx) % Mx;
    ky = (My - ky) % My;
    fb = (int64_t)kx * My + ky;
  }
  // the stored spectra carry e^{-2 pi i (kx CX / Mx + ky CY / My)} of the compact grids:
  // undo it (the fraction of a turn is reduced exactly in integers)
  C<R> ph;
  {
    const int64_t num = ((int64_t)kx * CX * My + (int64_t)ky * CY * Mx) % F;
    double sn, cs;
    sincospi(2.0 * (double)num / (double)F, &sn, &cs);
    ph = cfrom64<R>(cs, sn);
  }
  const int* mir = mirror + c * L;
  for (int r0 = 0; r0 < R_; r0 += RC) {
#pragma unroll
    for (int q = 0; q < RC; ++q)
#pragma unroll
      for (int v = 0; v < L; ++v) {
        const bool live = r0 + q < R_;
        const int64_t row = (int64_t)(r0 + q) * P + c * L;
        x1[(q * L + v) * TS] = live ? Xh[(row + v) * F + f1] : czero<R>();
        C<R> w = czero<R>();
        if (live && pair) {
          const int m = mir[v];
          w = Xh[(row + (m & 0xffff)) * F + f2];
          if (m >> 16) w = cneg(w);
        }
        x2[(q * L + v) * TS] = w;
      }
    // rows of G double-buffered in registers (complex64, L <= 24): row u + 1 is in flight
    // while row u is used
    C<R> gA[L], gB[L];
#define FFT_MUL_LOAD(U, DST)                                                                 \
  _Pragma("unroll") for (int v = 0; v < L; ++v) {                                            \
    const int comp = MODE == 1 ? (c * L + v) * L + (U) : (c * L + (U)) * L + v;              \
    DST[v] = Bh[(int64_t)r0 * bstride + (int64_t)comp * F + fb];                             \
  }
#define FFT_MUL_USE(U, G)                                                                    \
  {                                                                                          \
    __syncwarp(); /* the X^ columns are re-read per row, not hoisted into registers */       \
    C<R> acc1[RC], acc2[RC];                                                                 \
    _Pragma("unroll") for (int q = 0; q < RC; ++q) acc1[q] = acc2[q] = czero<R>();          \
    _Pragma("unroll") for (int v = 0; v < L; ++v) {                                          \
      _Pragma("unroll") for (int q = 0; q < RC; ++q) {                                       \
        cfma(acc1[q], G[v], x1[(q * L + v) * TS]);                                           \
        cfma(acc2[q], G[v], x2[(q * L + v) * TS]);                                           \
      }                                                                                      \
    }                                                                                        \
    const int m = mir[(U)];                                                                  \
    const C<R> ph2 = ((m >> 16) != 0) != (msign < 0) ? cneg(ph) : ph;                      \
    _Pragma("unroll") for (int q = 0; q < RC; ++q) if (r0 + q < R_) {                        \
      const int64_t row = (int64_t)(r0 + q) * P + c * L;                                     \
      Yh[(row + (U)) * F + f1] = cmul(acc1[q], ph);                                          \
      if (pair) Yh[(row + (m & 0xffff)) * F + f2] = cmul(acc2[q], ph2);                      \
    }                                                                                        \
  }
    if constexpr (std::is_same_v<R, float> && L <= 24) {
      FFT_MUL_LOAD(0, gA)
#pragma unroll 1
      for (int u = 0; u < L; u += 2) {
        if (u + 1 < L) FFT_MUL_LOAD(u + 1, gB)
        FFT_MUL_USE(u, gA)
        if (u + 1 < L) {
          if (u + 2 < L) FFT_MUL_LOAD(u + 2, gA)
          FFT_MUL_USE(u + 1, gB)
        }
      }
    } else {  // wider rows or fp64: one row in flight (the register file holds no second)
      (void)gB;
#pragma unroll 1
      for (int u = 0; u < L; ++u) {
        FFT_MUL_LOAD(u, gA)
        FFT_MUL_USE(u, gA)
      }
    }
#undef FFT_MUL_LOAD
#undef FFT_MUL_USE
  }
}

// ---- quad-mirror block product (complex64) ---------------------------------------------
// Besides the two mirror identities the blocks obey reciprocity, B_(-o) = J B_o^T J, and the
// full inversion B_(-o) = Dm B_o Dm with Dm = diag((-1)^m); together B_o^T = S B_o S with
// S = J Dm (an involution), so C_o = B_o S is symmetric. All of this is linear in the
// blocks, so with the true spectra B^(f) (shift phase removed) and an item (kx, ky),
// 0 <= kx <= Mx/2, 0 <= ky <= My/2, the one symmetric matrix C = B^(kx, ky) S gives the
// products at all four frequencies f1 = (kx, ky), f2 = (kx, -ky), f3 = (-kx, ky),
// f4 = (-kx, -ky), for the forward operator and its transpose:
//   forward  Y(f1) = C (S X)         Y(f2) = Dy J C (Dx X)   Y(f3) = Dx J C (Dy X)   Y(f4) = Dm C (J X)
//   adjoint  Y(f1) = J C (Dm X)      Y(f2) = Dy C (J Dx X)   Y(f3) = Dx C (J Dy X)   Y(f4) = J Dm C X
// (adjoint: Y(f) = B^(-f)^T X(f)), with Dx = diag((-1)^(m+p)), Dy = diag((-1)^p). Every
// input and output map is a signed permutation (J or identity, times one of the diagonal
// signs, all J-invariant), so one read of C (one quarter of the full spectra) serves four
// frequencies and both directions. C is staged per tile of NI consecutive ky by one bulk
// copy into shared memory; thread (item, class, u) forms row u of Z = C W for the 4 x RC
// columns W (the transformed inputs), reading C[v][u] = C[u][v] (consecutive u: no bank
// conflicts) and the column values by broadcast.
constexpr uint32_t FFT4_WAIT_LIMIT = 1u << 22;  // polls of a bounded mbarrier wait

template <int L, int RC_ = 2, typename CR = float>
struct Fft4Cfg {
  static constexpr int NI = L <= 24 ? 4 : 2;  // items (consecutive ky) per tile
  static constexpr int THREADS = NI * 2 * L;
  static constexpr int RC = RC_;              // RHS per pass (1 when every RHS has its own spectra)
  static constexpr int NCOL = 4 * RC;         // columns: 4 frequencies x RC RHS
  // stride of one class block of C in complex values: >= L^2 and = 8 (mod 16), so that the
  // two class blocks of an item start 16 banks apart (a warp spanning both reads C without
  // bank conflicts); kept in the global layout too, so one bulk copy moves a whole tile
  static constexpr int SC = ((L * L + 7) / 16) * 16 + 8;
  // stride of one (item, class) block of the transformed inputs in complex values: two
  // values past a multiple of 64 bytes, so the class-0 and class-1 lanes of a warp (two
  // broadcast addresses per 16-byte load) fall on different banks
  static constexpr int SW = L * NCOL + 2;
  static constexpr size_t C_BYTES = (size_t)NI * 2 * SC * sizeof(C<CR>);
  static constexpr size_t W_BYTES = (size_t)NI * 2 * SW * sizeof(C<CR>);
  static constexpr size_t SMEM = C_BYTES + W_BYTES + 16;
  // resident CTAs per SM the registers allow (double-float: shared memory allows two)
  static constexpr int MIN_BLOCKS = std::is_same_v<CR, float> ? (L <= 24 ? 4 : 2) : (L <= 24 ? 2 : 1);
};

// sign selector: 0 none, 1 Dx = (-1)^(m+p), 2 Dy = (-1)^p, 3 Dm = (-1)^m
__device__ __forceinline__ bool fft4_neg(int sel, int mpar, int p) {
  return sel == 1 ? ((mpar ^ p) != 0) : sel == 2 ? (p != 0) : sel == 3 ? (mpar != 0) : false;
}

__device__ __forceinline__ bool fft4_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < FFT4_WAIT_LIMIT; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// per column k (frequency f1..f4) and direction D (0 forward / coupling, 1 transposed), see
// the block comment above: the input is permuted by J for k in {0, 3} (forward) or {1, 2}
// (transposed) and the output for the other two; the input sign is (Dm, Dx, Dy, 1) and the
// output sign (1, Dy, Dx, Dm) over k = 0..3 (selectors of fft4_neg)
__device__ __forceinline__ bool fft4_in_j(int D, int k) { return ((k == 0 || k == 3) ? 0 : 1) == D; }
__device__ __forceinline__ bool fft4_out_j(int D, int k) { return !fft4_in_j(D, k); }
__device__ __forceinline__ int fft4_in_s(int k) { return k == 0 ? 3 : (k == 1 ? 1 : (k == 2 ? 2 : 0)); }
__device__ __forceinline__ int fft4_out_s(int k) { return k == 0 ? 0 : (k == 1 ? 2 : (k == 2 ? 1 : 3)); }

// cstride: complex values between the spectra of consecutive RHS (0: one operator for all
// RHS; otherwise RC = 1 and every RHS pass stages its own C)
// CR = float: complex64 spectra and arithmetic; CR = DF: double-float pairs (the complex128
// operators' fp64-accurate residuals), the same maps and staging.
template <typename CR, int L, int MODE, int RC_>
__global__ void __launch_bounds__(Fft4Cfg<L, RC_, CR>::THREADS, Fft4Cfg<L, RC_, CR>::MIN_BLOCKS)
fft_mul4_kernel(const C<CR>* __restrict__ Cq, const C<CR>* __restrict__ Xh, C<CR>* __restrict__ Yh, int Mx, int My,
                int R_, const int* __restrict__ sym, int* __restrict__ err, int64_t cstride) {
  pdl_wait();
  using Cfg = Fft4Cfg<L, RC_, CR>;
  using CT = C<CR>;
  constexpr int NI = Cfg::NI, RC = Cfg::RC, NCOL = Cfg::NCOL, P = 2 * L, SC = Cfg::SC, SW = Cfg::SW,
                NT = Cfg::THREADS;
  constexpr int D = MODE == 1 ? 1 : 0;
  extern __shared__ __align__(128) unsigned char fsm4[];
  CT* Cs = reinterpret_cast<CT*>(fsm4);                  // [NI][2][SC]
  CT* Ws = reinterpret_cast<CT*>(fsm4 + Cfg::C_BYTES);   // [NI][2][SW >= L * NCOL]
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(fsm4 + Cfg::C_BYTES + Cfg::W_BYTES);
  const uint32_t cs_addr = (uint32_t)__cvta_generic_to_shared(Cs);
  const int t = threadIdx.x;
  const int it = t / (2 * L), c = (t / L) & 1, u = t % L;  // compute role: row u of item it, class c
  const int64_t F = (int64_t)Mx * My;
  const int hx = Mx >= 2 ? Mx / 2 + 1 : 1, hy = My >= 2 ? My / 2 + 1 : 1;
  const int tpr = (hy + NI - 1) / NI;
  const int64_t ntiles = (int64_t)hx * tpr;
  const int su = sym[c * L + u];
  const int mpar = (su >> 16) & 1, pp = (su >> 17) & 1;
  if ((int64_t)blockIdx.x >= ntiles) return;  // uniform over the CTA
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();

  // the tile's four frequencies of item i (kx fixed per tile) and which are distinct
  auto tile_of = [&](int64_t tl, int& kx, int& ky0, int& ni) {
    kx = (int)(tl / tpr);
    ky0 = (int)(tl % tpr) * NI;
    ni = min(NI, hy - ky0);
  };
  auto issue_c = [&](int64_t tl, int r0) {
    int kx, ky0, ni;
    tile_of(tl, kx, ky0, ni);
    const uint32_t bytes = (uint32_t)(ni * 2 * SC * sizeof(CT));
    const CT* src = Cq + (int64_t)r0 * cstride + ((int64_t)kx * hy + ky0) * 2 * SC;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(cs_addr), "l"(src), "r"(bytes), "r"(bar) : "memory");
  };
  // load role: value e = t + j NT of the tile's transformed inputs, item fastest (the NI
  // items of a tile are consecutive frequencies: one 32-byte sector per plane for NI = 4)
  CT wv[NCOL];
  auto load_w = [&](int64_t tl, int r0) {
    int kx, ky0, ni;
    tile_of(tl, kx, ky0, ni);
    const int kxm = (Mx - kx) % Mx;
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      const int e = t + j * NT;
      const int item = e % NI, rest = e / NI;
      const int col = rest % NCOL, row = rest / NCOL;
      const int cc = row / L, v = row % L, k = col / RC, q = col % RC;
      const int ky = ky0 + item, kym = (My - ky) % My;
      const bool ok = item < ni && r0 + q < R_ && ((k & 1) == 0 || kym != ky) && ((k & 2) == 0 || kxm != kx);
      CT w = czero<CR>();
      if (ok) {
        const int sv = sym[cc * L + v];
        const int comp = fft4_in_j(D, k) ? (sv & 0xffff) : v;
        const int64_t f = (int64_t)((k & 2) ? kxm : kx) * My + ((k & 1) ? kym : ky);
        w = Xh[((int64_t)(r0 + q) * P + cc * L + comp) * F + f];
        if (fft4_neg(fft4_in_s(k), (sv >> 16) & 1, (sv >> 17) & 1)) w = cneg(w);
      }
      wv[j] = w;
    }
  };
  auto store_w = [&]() {
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      const int e = t + j * NT;
      const int item = e % NI, rest = e / NI;
      const int col = rest % NCOL, row = rest / NCOL;
      Ws[(item * 2 + row / L) * SW + (row % L) * NCOL + col] = wv[j];
    }
  };

  int64_t tile = blockIdx.x;
  uint32_t phase = 0;
  if (t == 0) issue_c(tile, 0);
  load_w(tile, 0);
  store_w();
  for (;;) {
    int kx, ky0, ni;
    tile_of(tile, kx, ky0, ni);
    const int kxm = (Mx - kx) % Mx;
    for (int r0 = 0; r0 < R_; r0 += RC) {
      int bad = 0;
      const uint32_t wphase = phase;
      if (r0 == 0 || cstride) {
        bad = !fft4_wait(bar, wphase);
        if (cstride) phase ^= 1u;  // one copy per RHS pass
      }
      bad = __syncthreads_or(bad);  // also makes this stage's Ws visible
      if (bad) {
        if (t == 0) {
          atomicAdd(err, 1);
          fft4_wait(bar, wphase);  // let the copy in flight land before the CTA leaves
        }
        return;
      }
      CT acc[NCOL];
#pragma unroll
      for (int j = 0; j < NCOL; ++j) acc[j] = czero<CR>();
      const CT* Ci = Cs + (it * 2 + c) * SC + u;
      if constexpr (std::is_same_v<CR, float>) {
        const float4* Wi = reinterpret_cast<const float4*>(Ws + (it * 2 + c) * SW);
#pragma unroll 4
        for (int v = 0; v < L; ++v) {
          const float2 g = Ci[v * L];
#pragma unroll
          for (int j = 0; j < NCOL / 2; ++j) {
            const float4 w2 = Wi[v * (NCOL / 2) + j];
            cfma(acc[2 * j], g, make_float2(w2.x, w2.y));
            cfma(acc[2 * j + 1], g, make_float2(w2.z, w2.w));
          }
        }
      } else {
        const CT* Wc = Ws + (it * 2 + c) * SW;
#pragma unroll 2
        for (int v = 0; v < L; ++v) {
          const CT g = Ci[v * L];
#pragma unroll
          for (int j = 0; j < NCOL; ++j) cfma(acc[j], g, Wc[v * NCOL + j]);
        }
      }
      __syncthreads();  // every read of Cs and Ws of this stage is done
      // this thread's outputs, with their output signs, into the staging area (Ws); the
      // stores below take them item-fastest, so the NI items of a tile fill whole sectors
      {
        CT* zrow = Ws + (it * 2 + c) * SW + u * NCOL;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int q = 0; q < RC; ++q) {
            CT z = acc[k * RC + q];
            if (fft4_neg(fft4_out_s(k), mpar, pp)) z = cneg(z);
            zrow[k * RC + q] = z;
          }
      }
      __syncthreads();
      // next stage: its C copy (new tile) and its input loads go out before this stage's
      // outputs are written
      const bool more_rhs = r0 + RC < R_;
      const int64_t ntile = more_rhs ? tile : tile + gridDim.x;
      const bool have_next = ntile < ntiles;
      if (have_next) {
        if ((!more_rhs || cstride) && t == 0) issue_c(ntile, more_rhs ? r0 + RC : 0);
        load_w(ntile, more_rhs ? r0 + RC : 0);
      }
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const int e = t + j * NT;
        const int item = e % NI, rest = e / NI;
        const int col = rest % NCOL, row = rest / NCOL;
        const int cc = row / L, v = row % L, k = col / RC, q = col % RC;
        const int iky = ky0 + item, ikym = (My - iky) % My;
        const bool ok = item < ni && r0 + q < R_ && ((k & 1) == 0 || ikym != iky) && ((k & 2) == 0 || kxm != kx);
        if (ok) {
          const int comp = fft4_out_j(D, k) ? (sym[cc * L + v] & 0xffff) : v;
          const int64_t f = (int64_t)((k & 2) ? kxm : kx) * My + ((k & 1) ? ikym : iky);
          Yh[((int64_t)(r0 + q) * P + cc * L + comp) * F + f] = Ws[(item * 2 + cc) * SW + v * NCOL + col];
        }
      }
      __syncthreads();  // the staged outputs are read
      if (have_next) store_w();
    }
    tile += gridDim.x;
    if (tile >= ntiles) break;
    if (!cstride) phase ^= 1u;
  }
}

// C[item][c][u][v] = ph(f1) Bs[(c L + u) L + J(v)][f1] (-1)^(m_v) from the stored spectra
// (component-major, with the compact-grid shift phase, undone here); item = kx * hy + ky,
// class blocks SC complex values apart (the padding is left zero).
// the shift phase of every item, once (the pack kernel reads it for all 2 L^2 entries)
template <typename CR>
__global__ void fft_quad_phase_kernel(int Mx, int My, int CX, int CY, C<CR>* __restrict__ ph) {
  const int hy = My >= 2 ? My / 2 + 1 : 1, hx = Mx >= 2 ? Mx / 2 + 1 : 1;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)hx * hy) return;
  const int kx = (int)(item / hy), ky = (int)(item % hy);
  const int64_t F = (int64_t)Mx * My;
  const int64_t num = ((int64_t)kx * CX * My + (int64_t)ky * CY * Mx) % F;
  double sn, cs;
  sincospi(2.0 * (double)num / (double)F, &sn, &cs);
  ph[item] = cfrom64<CR>(cs, sn);
}

template <typename CR>
__global__ void fft_pack_quad_kernel(const C<CR>* __restrict__ Bs, int Mx, int My, int L, int SC,
                                     const C<CR>* __restrict__ ph, const int* __restrict__ sym,
                                     C<CR>* __restrict__ Cq) {
  const int hy = My >= 2 ? My / 2 + 1 : 1, hx = Mx >= 2 ? Mx / 2 + 1 : 1;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.y;  // (c, u, v)
  if (item >= (int64_t)hx * hy) return;
  const int c = e / (L * L), u = (e / L) % L, v = e % L;
  const int kx = (int)(item / hy), ky = (int)(item % hy);
  const int64_t F = (int64_t)Mx * My, f1 = (int64_t)kx * My + ky;
  const int sv = sym[c * L + v];
  const C<CR> b = Bs[((int64_t)(c * L + u) * L + (sv & 0xffff)) * F + f1];
  C<CR> z = cmul(ph[item], b);
  if ((sv >> 16) & 1) z = cneg(z);
  Cq[(item * 2 + c) * SC + u * L + v] = z;
}

// Forward 2-D transform of nb component grids [nb][ny][nx] into [nb][Mx][My] (via tmp).
template <typename R>
static int fft2_forward(tmat_ctx* ctx, const C<R>* grid, int nx, int ny, int Mx, int My, int64_t nb, C<R>* tmp,
                        C<R>* out, const double2* tw) {
  // F1: rows iy (ny of them), FFT along ix, write transposed tmp[b][kx][iy] (pitch ny)
  TM_TRY((fft_rows<R, true, false, false, true>(ctx, grid, (int64_t)ny * nx, nx, nx, ny, tmp, (int64_t)Mx * ny, ny, Mx,
                                                Mx, nb, -1, tw)));
  // F2: rows kx (Mx), FFT along iy zero-padded to My -> out[b][kx][ky] (storage format)
  TM_TRY((fft_rows<R, false, false, true, true>(ctx, tmp, (int64_t)Mx * ny, ny, ny, Mx, out, (int64_t)Mx * My, My, My,
                                                My, nb, -1, tw)));
  return TMAT_OK;
}

// Inverse: [nb][Mx][My] -> [nb][ny][nx] (unnormalised), keeping iy < ny, ix < nx.
template <typename R>
static int fft2_inverse(tmat_ctx* ctx, const C<R>* spec, int nx, int ny, int Mx, int My, int64_t nb, C<R>* tmp,
                        C<R>* out, const double2* tw) {
  // I2: rows kx, inverse along ky, keep iy < ny, transposed -> tmp[b][iy][kx] (pitch Mx)
  TM_TRY((fft_rows<R, true, false, true, true>(ctx, spec, (int64_t)Mx * My, My, My, Mx, tmp, (int64_t)ny * Mx, Mx, ny,
                                               My, nb, +1, tw)));
  // I1: rows iy, inverse along kx, keep ix < nx -> out[b][iy][ix]
  TM_TRY((fft_rows<R, false, false, true, false>(ctx, tmp, (int64_t)ny * Mx, Mx, Mx, ny, out, (int64_t)ny * nx, nx, nx,
                                                 Mx, nb, +1, tw)));
  return TMAT_OK;
}

bool lattice_fft_fits(int nx, int ny, int CX, int CY) {
  return nx + CX <= FFT_MAXLEN && ny + CY <= FFT_MAXLEN;
}

// B^ of the operator (forward blocks; the adjoint reads it transposed at -f).
template <typename R>
static int fft_prepare_t(tmat_ctx* ctx, LatOp* a, const char* name) {
  const int Mx = pow2_at_least(a->nx + a->CX), My = pow2_at_least(a->ny + a->CY);
  const int L = a->L;
  const int64_t ncomp = 2 * (int64_t)L * L;
  const int64_t F = (int64_t)Mx * My;
  const double2* tw;
  TM_TRY(fft_twiddles(ctx, &tw));
  C<R>*Bh, *grid, *tmp;
  TM_TRY(scratch(ctx, name, sizeof(C<R>) * ncomp * F, (void**)&Bh));
  // staging: the compact (2 CY + 1) x (2 CX + 1) grids of the offsets and the transposed
  // intermediate Mx x (2 CY + 1); only these rows carry data, so only they are transformed
  const int gw = 2 * a->CX + 1, gh = 2 * a->CY + 1;
  TM_TRY(scratch(ctx, "fft_bgrid", sizeof(C<R>) * ncomp * gw * gh, (void**)&grid));
  TM_TRY(scratch(ctx, "fft_btmp", sizeof(C<R>) * ncomp * Mx * gh, (void**)&tmp));
  TM_CUDA(ctx, cudaMemsetAsync(grid, 0, sizeof(C<R>) * ncomp * gw * gh, ctx->stream));
  fft_scatter_blocks_kernel<R><<<a->K, 256, 0, ctx->stream>>>((const C<R>*)a->BT, a->off, a->K, L, a->LP, a->CX, a->CY,
                                                              grid);
  TM_LAUNCHED(ctx);
  // stored without the shift phase; the block product applies it per frequency
  TM_TRY(fft2_forward<R>(ctx, grid, gw, gh, Mx, My, ncomp, tmp, Bh, tw));
  a->fft_Mx = Mx;
  a->fft_My = My;
  a->fft_Bhat = Bh;
  a->use_fft = true;
  a->fft_C = nullptr;
  // the quad-mirror form (complex64 operators, and the double-float pairs of complex128 ones)
  if (a->fft_quad_ok && a->fft_mirror_sign == 1 && a->fft_sym && ctx->fft_quad) {
    using CR = typename fft_compute<R>::t;
    using CS = C<CR>;
    const int hx = Mx >= 2 ? Mx / 2 + 1 : 1, hy = My >= 2 ? My / 2 + 1 : 1;
    const int64_t items = (int64_t)hx * hy;
    const int SC = ((L * L + 7) / 16) * 16 + 8;  // Fft4Cfg<L>::SC
    std::string cn = std::string(name) + "_quad";
    CS* Cq;
    int* err;
    TM_TRY(scratch(ctx, cn.c_str(), sizeof(CS) * items * 2 * SC, (void**)&Cq));
    TM_TRY(scratch(ctx, "fft_quad_err", sizeof(int), (void**)&err));
    TM_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    TM_CUDA(ctx, cudaMemsetAsync(Cq, 0, sizeof(CS) * items * 2 * SC, ctx->stream));
    CS* qph;
    TM_TRY(scratch(ctx, "fft_quad_ph", sizeof(CS) * items, (void**)&qph));
    fft_quad_phase_kernel<CR><<<(unsigned)cdiv(items, 128), 128, 0, ctx->stream>>>(Mx, My, a->CX, a->CY, qph);
    TM_LAUNCHED(ctx);
    dim3 g((unsigned)cdiv(items, 128), (unsigned)(2 * L * L));
    fft_pack_quad_kernel<CR><<<g, 128, 0, ctx->stream>>>(reinterpret_cast<const CS*>(Bh), Mx, My, L, SC, qph,
                                                         a->fft_sym, Cq);
    TM_LAUNCHED(ctx);
    a->fft_C = Cq;
    a->fft_err = err;
  }
  return TMAT_OK;
}

int lattice_fft_prepare(tmat_ctx* ctx, LatOp* a, const char* name) {
  if (a->K == 0 || !lattice_fft_fits(a->nx, a->ny, a->CX, a->CY)) return TMAT_OK;
  if (a->fp32) return fft_prepare_t<float>(ctx, a, name ? name : "fft_Bh32");
  return fft_prepare_t<double>(ctx, a, name ? name : "fft_Bh64");
}

template <typename R, int L, int MODE>
static int fft_apply_t(tmat_ctx* ctx, const LatOp& a, const void* xv, void* yv, int R_) {
  constexpr int P = 2 * L;
  const int Mx = a.fft_Mx, My = a.fft_My, nx = a.nx, ny = a.ny;
  const int64_t F = (int64_t)Mx * My;
  const int64_t nb = (int64_t)R_ * P;
  const double2* tw;
  TM_TRY(fft_twiddles(ctx, &tw));
  const char* s1 = sizeof(R) == 4 ? "fft_w1_32" : "fft_w1_64";
  const char* s2 = sizeof(R) == 4 ? "fft_w2_32" : "fft_w2_64";
  C<R>*w1, *w2;  // w1: component grids / transposed intermediates; w2: spectra
  TM_TRY(scratch(ctx, s1, sizeof(C<R>) * nb * std::max<int64_t>((int64_t)Mx * ny, (int64_t)nx * ny), (void**)&w1));
  TM_TRY(scratch(ctx, s2, sizeof(C<R>) * 2 * nb * F, (void**)&w2));
  C<R>* Xh = w2;
  C<R>* Yh = w2 + nb * F;
  C<R>* grid = Yh;  // the input grids live in the (not yet used) output spectrum buffer
  const C<R>* x = (const C<R>*)xv;
  const C<R>* T = (const C<R>*)a.T;
  cudaEvent_t ev_all = timing_begin(ctx);
  dim3 tb(32, 8);
  dim3 tg((unsigned)cdiv(nx, 32), (unsigned)ny, (unsigned)(R_ * cdiv(P, 32)));
  // 256 x 256 grids: the passes read x and write y in place through the component-innermost
  // intermediates T1 [r][kx][iy][P] and T2 [r][iy][kx][P] (w1)
  const bool ci = Mx == 256 && My == 256;
  const int64_t Nsite = (int64_t)nx * ny;
  const F256Lay lx{Nsite * P, 1, (int64_t)nx * P, P};                         // x, y: line iy, col ix
  const F256Lay lspec{(int64_t)P * F, F, My, 1};                              // spectra: line kx, col ky
  const F256Lay lt1_out{(int64_t)Mx * ny * P, 1, P, (int64_t)ny * P};         // T1 written: line iy, k kx
  const F256Lay lt1_in{(int64_t)Mx * ny * P, 1, (int64_t)ny * P, P};          // T1 read: line kx, col iy
  const F256Lay lt2_out{(int64_t)ny * Mx * P, 1, P, (int64_t)Mx * P};         // T2 written: line kx, k iy
  const F256Lay lt2_in{(int64_t)ny * Mx * P, 1, (int64_t)Mx * P, P};          // T2 read: line iy, col kx
  const dim3 gy((unsigned)ny, (unsigned)cdiv(P, 16), (unsigned)R_), gk((unsigned)Mx, (unsigned)cdiv(P, 16), (unsigned)R_);
  using CR = typename fft_compute<R>::t;
  using CS = C<CR>;  // storage of the intermediates and spectra (double-float pairs for complex128)
  if (ci) {
    const G<CR>* xg = reinterpret_cast<const G<CR>*>(x);
    const G<CR>* Tg = reinterpret_cast<const G<CR>*>(T);
    CS* w1s = reinterpret_cast<CS*>(w1);
    auto k1 = MODE == 1 ? fft256_ci_kernel<CR, true, true, 2, -1, false, true>
                        : fft256_ci_kernel<CR, true, true, 0, -1, false, true>;
    auto k2 = fft256_ci_kernel<CR, true, false, 0, -1, true, true>;
    const size_t sm = F256Smem<CR, -1>::BYTES;
    if (sm > 48 * 1024) {
      TM_TRY(set_smem_limit(ctx, (const void*)k1, sm));
      TM_TRY(set_smem_limit(ctx, (const void*)k2, sm));
    }
    TM_CUDA(ctx, launch_pdl(ctx->stream, k1, gy, dim3(256), sm, xg, lx, nx, w1s, lt1_out, Mx, P, -1, tw, Tg,
                            a.t_stride, (const G<CR>*)nullptr, 1.f));
    TM_LAUNCHED(ctx);
    TM_CUDA(ctx, launch_pdl(ctx->stream, k2, gk, dim3(256), sm, (const CS*)w1s, lt1_in, ny, reinterpret_cast<CS*>(Xh),
                            lspec, My, P, -1, tw, Tg, a.t_stride, (const G<CR>*)nullptr, 1.f));
    TM_LAUNCHED(ctx);
  } else {
    fft_embed_kernel<R, MODE == 1 ? 1 : 0><<<tg, tb, 0, ctx->stream>>>(x, T, nx, ny, P, R_, grid, a.t_stride);
    TM_LAUNCHED(ctx);
    TM_TRY(fft2_forward<R>(ctx, grid, nx, ny, Mx, My, nb, w1, Xh, tw));
  }
  bool quad_done = false;
  if (a.fft_C) {
    // one RHS per pass when every RHS has its own operator
    using Cfg = Fft4Cfg<L, 2, CR>;
    auto kern = a.fft_cstride ? fft_mul4_kernel<CR, L, MODE == 1 ? 1 : 0, 1> : fft_mul4_kernel<CR, L, MODE == 1 ? 1 : 0, 2>;
    const size_t smem = a.fft_cstride ? Fft4Cfg<L, 1, CR>::SMEM : Cfg::SMEM;
    if (smem > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, smem));
    const int hx = Mx >= 2 ? Mx / 2 + 1 : 1, hy = My >= 2 ? My / 2 + 1 : 1;
    const int64_t ntiles = (int64_t)hx * cdiv(hy, Cfg::NI);
    int per_sm = 0;  // queried once per kernel (its block size and shared memory are fixed)
    auto occ = ctx->occupancy.find((const void*)kern);
    if (occ != ctx->occupancy.end()) {
      per_sm = occ->second;
    } else {
      TM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, smem));
      ctx->occupancy[(const void*)kern] = per_sm;
    }
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * std::max(1, per_sm));
    cudaEvent_t ev = timing_begin(ctx);
    TM_CUDA(ctx, launch_pdl(ctx->stream, kern, dim3((unsigned)grid), dim3(Cfg::THREADS), smem,
                            reinterpret_cast<const CS*>(a.fft_C), reinterpret_cast<const CS*>(Xh),
                            reinterpret_cast<CS*>(Yh), Mx, My, R_, a.fft_sym, a.fft_err, a.fft_cstride));
    TM_LAUNCHED(ctx);
    // the quad-form spectra once, the RHS spectra in and out
    const double mul_bytes =
        (double)sizeof(CS) * ((double)hx * hy * 2.0 * Cfg::SC * (a.fft_cstride ? R_ : 1) + 2.0 * nb * F);
    timing_end(ctx, sizeof(R) == 4 ? "lattice_fft_mul32" : "lattice_fft_mul64", ev, mul_bytes);
    quad_done = true;
  }
  if (!quad_done) {
    // the mirror-pair product (complex128 operators: in double-float on spectra stored as
    // pairs), where the quad form is not built
    using CM = typename fft_compute<R>::t;
    constexpr int RC2 = (sizeof(R) == 4 && L <= 24) ? 2 : 1;
    const int RC = a.fft_bstride ? 1 : RC2;  // one RHS per pass when every RHS has its own spectra
    const size_t msm = sizeof(C<CM>) * 2 * (size_t)RC * L * FFT_MUL_THREADS;
    auto kern = RC == 1 ? fft_mul_kernel<CM, L, MODE, 1> : fft_mul_kernel<CM, L, MODE, RC2>;
    if (msm > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)kern, msm));
    const int64_t items = (int64_t)Mx * (My >= 2 ? My / 2 + 1 : 1);
    dim3 g((unsigned)cdiv(items, FFT_MUL_THREADS), 2);
    cudaEvent_t ev = timing_begin(ctx);
    kern<<<g, FFT_MUL_THREADS, msm, ctx->stream>>>((const C<CM>*)a.fft_Bhat, (const C<CM>*)Xh, (C<CM>*)Yh, Mx, My, R_,
                                                   a.CX, a.CY, a.fft_mirror, a.fft_mirror_sign, a.fft_bstride);
    TM_LAUNCHED(ctx);
    // the block spectra of one frequency per mirror pair, the RHS spectra in and out
    const double mul_bytes = (double)sizeof(C<R>) * (items * 2.0 * L * L * (a.fft_bstride ? R_ : 1) + 2.0 * nb * F);
    timing_end(ctx, sizeof(R) == 4 ? "lattice_fft_mul32" : "lattice_fft_mul64", ev, mul_bytes);
  }
  if (ci) {
    const G<CR>* xg = reinterpret_cast<const G<CR>*>(x);
    const G<CR>* Tg = reinterpret_cast<const G<CR>*>(T);
    CS* w1s = reinterpret_cast<CS*>(w1);
    auto k3 = fft256_ci_kernel<CR, false, true, 0, -1, true, true>;
    auto k4 = fft256_ci_kernel<CR, true, true, 0, MODE, true, false>;
    const size_t sm3 = F256Smem<CR, -1>::BYTES, sm4 = F256Smem<CR, MODE>::BYTES;
    if (sm3 > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)k3, sm3));
    if (sm4 > 48 * 1024) TM_TRY(set_smem_limit(ctx, (const void*)k4, sm4));
    TM_CUDA(ctx, launch_pdl(ctx->stream, k3, gk, dim3(256), sm3, reinterpret_cast<const CS*>(Yh), lspec, My, w1s,
                            lt2_out, ny, P, +1, tw, Tg, a.t_stride, (const G<CR>*)nullptr, 1.f));
    TM_LAUNCHED(ctx);
    TM_CUDA(ctx, launch_pdl(ctx->stream, k4, gy, dim3(256), sm4, (const CS*)w1s, lt2_in, Mx, reinterpret_cast<G<CR>*>(yv),
                            lx, nx, P, +1, tw, Tg, a.t_stride, xg, (float)(1.0 / (double)F)));
    TM_LAUNCHED(ctx);
  } else {
    C<R>* Yc = Xh;  // X^ is no longer needed
    TM_TRY(fft2_inverse<R>(ctx, Yh, nx, ny, Mx, My, nb, w1, Yc, tw));
    fft_extract_kernel<R, MODE><<<tg, tb, 0, ctx->stream>>>(Yc, x, T, nx, ny, P, (R)(1.0 / (double)F), (C<R>*)yv,
                                                            a.t_stride);
    TM_LAUNCHED(ctx);
  }
  timing_end(ctx, sizeof(R) == 4 ? "lattice_apply_fft32" : "lattice_apply_fft64", ev_all);
  return TMAT_OK;
}

template <typename R, int L>
static int fft_apply_l(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  if (mode == TMAT_OP_FORWARD) return fft_apply_t<R, L, 0>(ctx, a, x, y, R_);
  if (mode == TMAT_OP_ADJOINT) return fft_apply_t<R, L, 1>(ctx, a, x, y, R_);
  return fft_apply_t<R, L, 2>(ctx, a, x, y, R_);
}

template <typename R>
static int fft_apply_r(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  switch (a.nmax) {
    case 1: return fft_apply_l<R, 3>(ctx, a, mode, x, y, R_);
    case 2: return fft_apply_l<R, 8>(ctx, a, mode, x, y, R_);
    case 3: return fft_apply_l<R, 15>(ctx, a, mode, x, y, R_);
    case 4: return fft_apply_l<R, 24>(ctx, a, mode, x, y, R_);
    case 5: return fft_apply_l<R, 35>(ctx, a, mode, x, y, R_);
    case 6: return fft_apply_l<R, 48>(ctx, a, mode, x, y, R_);
  }
  return set_error(ctx, TMAT_ENOTSUP, "FFT lattice apply: nmax %d", a.nmax);
}

int lattice_fft_apply(tmat_ctx* ctx, const LatOp& a, int mode, const void* x, void* y, int R_) {
  if (a.fp32) return fft_apply_r<float>(ctx, a, mode, x, y, R_);
  return fft_apply_r<double>(ctx, a, mode, x, y, R_);
}

}  // namespace tmat
