// Integer geometry: interaction neighbour lists and sub-region index sets.
#include "internal.h"

namespace tmat {

// d2 exactly as the definition states: dx*dx + dy*dy + dz*dz, left to right, every
// product and sum rounded separately (the _rn intrinsics are never contracted).
__device__ __forceinline__ double dist2_rn(const double* a, const double* b) {
  double dx = __dsub_rn(a[0], b[0]);
  double dy = __dsub_rn(a[1], b[1]);
  double dz = __dsub_rn(a[2], b[2]);
  double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return __dadd_rn(s, __dmul_rn(dz, dz));
}

// One warp per target row i: count (col == nullptr) or fill the row.
__global__ void nbr_kernel(const double* __restrict__ pos, int64_t N, double c2, int all,
                           const int64_t* __restrict__ row_ptr, int64_t* __restrict__ counts,
                           int32_t* __restrict__ col) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= N) return;
  double pi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  int64_t base = col ? row_ptr[i] : 0;
  int64_t cnt = 0;
  for (int64_t j0 = 0; j0 < N; j0 += 32) {
    int64_t j = j0 + lane;
    bool ok = false;
    if (j < N && j != i) ok = all ? true : (dist2_rn(pi, pos + 3 * j) <= c2);
    unsigned m = __ballot_sync(0xffffffffu, ok);
    if (col && ok) col[base + cnt + __popc(m & ((1u << lane) - 1u))] = (int32_t)j;
    cnt += __popc(m);
  }
  if (!col && lane == 0) counts[i] = cnt;
}

// single-block exclusive scan of N counts into row_ptr[0..N]
__global__ void scan_rows_kernel(const int64_t* counts, int64_t N, int64_t* row_ptr) {
  __shared__ int64_t part[1024];
  int t = threadIdx.x, T = blockDim.x;
  int64_t per = (N + T - 1) / T;
  int64_t b = t * per, e = min(N, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < T; ++k) {
      int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    row_ptr[N] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t i = b; i < e; ++i) {
    row_ptr[i] = run;
    run += counts[i];
  }
}

int build_neighbors(tmat_ctx* ctx, const double* d_pos, int64_t N, double cutoff, int64_t* d_row_ptr,
                    int32_t* d_col, int64_t* nnz_out) {
  int all = !(cutoff > 0);
  double c2 = cutoff * cutoff;
  const int warps = 8;
  unsigned grid = (unsigned)cdiv(N, warps);
  if (!d_col) {
    int64_t* counts;
    TM_TRY(scratch(ctx, "nbr_counts", sizeof(int64_t) * (N + 1), (void**)&counts));
    if (N > 0) {
      nbr_kernel<<<grid, warps * 32, 0, ctx->stream>>>(d_pos, N, c2, all, nullptr, counts, nullptr);
      TM_LAUNCHED(ctx);
    }
    scan_rows_kernel<<<1, 1024, 0, ctx->stream>>>(counts, N, d_row_ptr);
    TM_LAUNCHED(ctx);
    int64_t* pin = (int64_t*)ctx->pinned;
    TM_CUDA(ctx, cudaMemcpyAsync(pin, d_row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *nnz_out = pin[0];
    return TMAT_OK;
  }
  if (N > 0) {
    nbr_kernel<<<grid, warps * 32, 0, ctx->stream>>>(d_pos, N, c2, all, d_row_ptr, nullptr, d_col);
    TM_LAUNCHED(ctx);
  }
  return TMAT_OK;
}

// sub-region sets: one thread per sub-region writes its core and simulated sets
__global__ void subregion_kernel(int64_t nx, int64_t ny, int64_t cx, int64_t cy, int64_t buf, int64_t nax,
                                 int64_t nsub, int64_t* core_ptr, int64_t* core_idx, int64_t* sim_ptr,
                                 int64_t* sim_idx, int count_only) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nsub) return;
  int64_t ax = a % nax, ay = a / nax;
  int64_t x0 = ax * cx, x1 = min((ax + 1) * cx, nx), y0 = ay * cy, y1 = min((ay + 1) * cy, ny);
  int64_t px0 = max((int64_t)0, x0 - buf), px1 = min(nx, x1 + buf);
  int64_t py0 = max((int64_t)0, y0 - buf), py1 = min(ny, y1 + buf);
  if (count_only) {
    core_ptr[a] = (x1 - x0) * (y1 - y0);
    sim_ptr[a] = (px1 - px0) * (py1 - py0);
    return;
  }
  int64_t o = core_ptr[a];
  for (int64_t iy = y0; iy < y1; ++iy)
    for (int64_t ix = x0; ix < x1; ++ix) core_idx[o++] = iy * nx + ix;
  o = sim_ptr[a];
  for (int64_t iy = py0; iy < py1; ++iy)
    for (int64_t ix = px0; ix < px1; ++ix) sim_idx[o++] = iy * nx + ix;
}

}  // namespace tmat

using namespace tmat;

extern "C" int tmat_neighbors(tmat_ctx* ctx, const double* pos, int64_t N, double cutoff, int64_t* row_ptr,
                              int32_t* col, int64_t* nnz_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || (!pos && N > 0) || !row_ptr || (!col && !nnz_out))
    return set_error(ctx, TMAT_EINVAL, "tmat_neighbors: bad arguments");
  if (N > 2147483647LL) return set_error(ctx, TMAT_EINVAL, "tmat_neighbors: N too large for int32 columns");
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  Staged sp, sr, sc;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  int64_t nnz = 0;
  if (!col) {
    TM_TRY(stage_out(ctx, "st_rowptr", row_ptr, sizeof(int64_t) * (N + 1), &sr));
    TM_TRY(build_neighbors(ctx, (const double*)sp.dev, N, cutoff, (int64_t*)sr.dev, nullptr, &nnz));
    TM_TRY(finish_out(ctx, &sr));
    if (nnz_out) *nnz_out = nnz;
    return TMAT_OK;
  }
  TM_TRY(stage_in(ctx, "st_rowptr", row_ptr, sizeof(int64_t) * (N + 1), &sr));
  int64_t* pin = (int64_t*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, (const int64_t*)sr.dev + N, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int64_t total = pin[0];
  TM_TRY(stage_out(ctx, "st_col", col, sizeof(int32_t) * total, &sc));
  TM_TRY(build_neighbors(ctx, (const double*)sp.dev, N, cutoff, (int64_t*)sr.dev, (int32_t*)sc.dev, &nnz));
  TM_TRY(finish_out(ctx, &sc));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (nnz_out) *nnz_out = total;
  return TMAT_OK;
}

extern "C" int tmat_subregions(tmat_ctx* ctx, int64_t nx, int64_t ny, int64_t cx, int64_t cy, int64_t buf,
                               int64_t* core_ptr, int64_t* core_idx, int64_t* sim_ptr, int64_t* sim_idx,
                               int64_t* n_sub_out, int64_t* sim_total_out) {
  if (!ctx) return TMAT_EINVAL;
  if (nx <= 0 || ny <= 0 || cx <= 0 || cy <= 0 || buf < 0 || !core_ptr || !sim_ptr)
    return set_error(ctx, TMAT_EINVAL, "tmat_subregions: bad arguments");
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t nax = cdiv(nx, cx), nay = cdiv(ny, cy), nsub = nax * nay;
  Staged scp, ssp, sci, ssi;
  int64_t *cnt_core, *cnt_sim;
  TM_TRY(scratch(ctx, "sub_cnt_core", sizeof(int64_t) * (nsub + 1), (void**)&cnt_core));
  TM_TRY(scratch(ctx, "sub_cnt_sim", sizeof(int64_t) * (nsub + 1), (void**)&cnt_sim));
  TM_TRY(stage_out(ctx, "st_coreptr", core_ptr, sizeof(int64_t) * (nsub + 1), &scp));
  TM_TRY(stage_out(ctx, "st_simptr", sim_ptr, sizeof(int64_t) * (nsub + 1), &ssp));
  subregion_kernel<<<(unsigned)cdiv(nsub, 128), 128, 0, ctx->stream>>>(nx, ny, cx, cy, buf, nax, nsub, cnt_core,
                                                                         nullptr, cnt_sim, nullptr, 1);
  TM_LAUNCHED(ctx);
  scan_rows_kernel<<<1, 1024, 0, ctx->stream>>>(cnt_core, nsub, (int64_t*)scp.dev);
  TM_LAUNCHED(ctx);
  scan_rows_kernel<<<1, 1024, 0, ctx->stream>>>(cnt_sim, nsub, (int64_t*)ssp.dev);
  TM_LAUNCHED(ctx);
  int64_t* pin = (int64_t*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, (int64_t*)ssp.dev + nsub, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int64_t sim_total = pin[0];
  if (n_sub_out) *n_sub_out = nsub;
  if (sim_total_out) *sim_total_out = sim_total;
  if (core_idx && sim_idx) {
    TM_TRY(stage_out(ctx, "st_coreidx", core_idx, sizeof(int64_t) * nx * ny, &sci));
    TM_TRY(stage_out(ctx, "st_simidx", sim_idx, sizeof(int64_t) * sim_total, &ssi));
    subregion_kernel<<<(unsigned)cdiv(nsub, 128), 128, 0, ctx->stream>>>(nx, ny, cx, cy, buf, nax, nsub,
                                                                           (int64_t*)scp.dev, (int64_t*)sci.dev,
                                                                           (int64_t*)ssp.dev, (int64_t*)ssi.dev, 0);
    TM_LAUNCHED(ctx);
    TM_TRY(finish_out(ctx, &sci));
    TM_TRY(finish_out(ctx, &ssi));
  }
  TM_TRY(finish_out(ctx, &scp));
  TM_TRY(finish_out(ctx, &ssp));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TMAT_OK;
}
