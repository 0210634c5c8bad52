// Integer geometry: interaction neighbour lists and sub-region index sets.
#include <algorithm>
#include <cmath>

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

// ---- enclosing-sphere overlap (App. I-C: the enclosing spheres must not intersect) ----
// Two scatterers overlap when |x_i - x_j| < r_i + r_j (touching is allowed), tested in fp64
// as d2 < (r_i + r_j)^2 with every product and sum rounded separately. The points are binned
// on a uniform grid of cells no smaller than 2 max r, so a pair can overlap only if its
// cells are neighbours (27 cells in 3-D): O(N) work instead of all pairs.

// bounding box and largest radius: out[0..2] min, out[3..5] max, out[6] max r, out[7] min r,
// out[8] = 1 if a value is not finite
__global__ void bbox_kernel(const double* __restrict__ pos, const double* __restrict__ rad, int64_t N,
                            double* __restrict__ out) {
  __shared__ double red[8][256];
  double v[8] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0, 1e300};
  int bad = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double x = pos[3 * i + c];
      if (!isfinite(x)) bad = 1;
      v[c] = fmin(v[c], x);
      v[3 + c] = fmax(v[3 + c], x);
    }
    if (!isfinite(rad[i])) bad = 1;
    v[6] = fmax(v[6], rad[i]);
    v[7] = fmin(v[7], rad[i]);
  }
  for (int c = 0; c < 8; ++c) red[c][threadIdx.x] = v[c];
  bad = __syncthreads_or(bad);
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 8; ++c) {
        const double a = red[c][threadIdx.x], b = red[c][threadIdx.x + s];
        red[c][threadIdx.x] = (c < 3 || c == 7) ? fmin(a, b) : fmax(a, b);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < 8; ++c) out[c] = red[c][0];
    out[8] = bad;
  }
}

struct CellGrid {
  double x0, y0, z0, h;
  int64_t gx, gy, gz;
};

__device__ __forceinline__ int64_t cell_coord(double x, double x0, double h, int64_t g) {
  int64_t c = (int64_t)floor((x - x0) / h);
  return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__device__ __forceinline__ int64_t cell_of(const double* p, const CellGrid& g) {
  return (cell_coord(p[2], g.z0, g.h, g.gz) * g.gy + cell_coord(p[1], g.y0, g.h, g.gy)) * g.gx +
         cell_coord(p[0], g.x0, g.h, g.gx);
}

__global__ void cell_count_kernel(const double* __restrict__ pos, int64_t N, CellGrid g, int64_t* __restrict__ cnt,
                                  int64_t* __restrict__ cell) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cell_of(pos + 3 * i, g);
    cell[i] = c;
    atomicAdd((unsigned long long*)&cnt[c], 1ull);
  }
}

__global__ void cell_fill_kernel(const int64_t* __restrict__ cell, int64_t N, const int64_t* __restrict__ start,
                                 int64_t* __restrict__ cursor, int64_t* __restrict__ members) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cell[i];
    const int64_t k = (int64_t)atomicAdd((unsigned long long*)&cursor[c], 1ull);
    members[start[c] + k] = i;
  }
}

// first overlapping pair (smallest i * N + j, i < j) into *pair (initialised to N * N)
__global__ void overlap_kernel(const double* __restrict__ pos, const double* __restrict__ rad, int64_t N, CellGrid g,
                               const int64_t* __restrict__ start, const int64_t* __restrict__ members,
                               unsigned long long* __restrict__ pair) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double* p = pos + 3 * i;
    const int64_t cx = cell_coord(p[0], g.x0, g.h, g.gx), cy = cell_coord(p[1], g.y0, g.h, g.gy),
                  cz = cell_coord(p[2], g.z0, g.h, g.gz);
    for (int64_t dz = -1; dz <= 1; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          const int64_t x = cx + dx, y = cy + dy, z = cz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= g.gx || y >= g.gy || z >= g.gz) continue;
          const int64_t c = (z * g.gy + y) * g.gx + x;
          for (int64_t k = start[c]; k < start[c + 1]; ++k) {
            const int64_t j = members[k];
            if (j <= i) continue;
            const double s = __dadd_rn(rad[i], rad[j]);
            if (dist2_rn(p, pos + 3 * j) < __dmul_rn(s, s))
              atomicMin(pair, (unsigned long long)(i * N + j));
          }
        }
  }
}

// TMAT_OK, or TMAT_EOVERLAP with the first pair in pair_out (nullable); synchronises
int check_overlap(tmat_ctx* ctx, const double* d_pos, const double* d_rad, int64_t N, int64_t* pair_out) {
  if (N < 2) return TMAT_OK;
  double* box;
  TM_TRY(scratch(ctx, "ov_box", sizeof(double) * 9, (void**)&box));
  bbox_kernel<<<1, 256, 0, ctx->stream>>>(d_pos, d_rad, N, box);
  TM_LAUNCHED(ctx);
  double hb[9];
  double* pin = (double*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pin, box, sizeof(double) * 9, cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < 9; ++c) hb[c] = pin[c];
  if (hb[8] != 0 || hb[7] < 0)
    return set_error(ctx, TMAT_EINVAL, "overlap check: positions and radii must be finite, radii >= 0");
  if (!(hb[6] > 0)) return TMAT_OK;  // every radius zero: nothing can overlap
  CellGrid g;
  g.x0 = hb[0];
  g.y0 = hb[1];
  g.z0 = hb[2];
  g.h = 2.0 * hb[6] * (1.0 + 1e-12);
  auto dims = [&](double h, int64_t* d) {
    for (int c = 0; c < 3; ++c) d[c] = (int64_t)std::min(4.0e9, floor((hb[3 + c] - hb[c]) / h)) + 1;
  };
  int64_t d[3];
  dims(g.h, d);
  // at most ~4 N cells: coarser cells stay correct (neighbours still cover every overlap)
  while ((double)d[0] * d[1] * d[2] > 4.0 * N + 64) {
    g.h *= 1.5;
    dims(g.h, d);
  }
  g.gx = d[0];
  g.gy = d[1];
  g.gz = d[2];
  const int64_t ncell = g.gx * g.gy * g.gz;
  int64_t *cnt, *start, *cell, *members;
  unsigned long long* pair;
  TM_TRY(scratch(ctx, "ov_cnt", sizeof(int64_t) * (ncell + 1), (void**)&cnt));
  TM_TRY(scratch(ctx, "ov_start", sizeof(int64_t) * (ncell + 1), (void**)&start));
  TM_TRY(scratch(ctx, "ov_cell", sizeof(int64_t) * N, (void**)&cell));
  TM_TRY(scratch(ctx, "ov_members", sizeof(int64_t) * N, (void**)&members));
  TM_TRY(scratch(ctx, "ov_pair", sizeof(unsigned long long), (void**)&pair));
  TM_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (ncell + 1), ctx->stream));
  const unsigned long long none = (unsigned long long)N * (unsigned long long)N;
  TM_CUDA(ctx, cudaMemcpyAsync(pair, &none, sizeof(none), cudaMemcpyHostToDevice, ctx->stream));
  const unsigned gb = (unsigned)std::min<int64_t>(cdiv(N, 256), 8192);
  cell_count_kernel<<<gb, 256, 0, ctx->stream>>>(d_pos, N, g, cnt, cell);
  TM_LAUNCHED(ctx);
  scan_rows_kernel<<<1, 1024, 0, ctx->stream>>>(cnt, ncell, start);
  TM_LAUNCHED(ctx);
  TM_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (ncell + 1), ctx->stream));  // reused as cursors
  cell_fill_kernel<<<gb, 256, 0, ctx->stream>>>(cell, N, start, cnt, members);
  TM_LAUNCHED(ctx);
  overlap_kernel<<<gb, 256, 0, ctx->stream>>>(d_pos, d_rad, N, g, start, members, pair);
  TM_LAUNCHED(ctx);
  unsigned long long* pp = (unsigned long long*)ctx->pinned;
  TM_CUDA(ctx, cudaMemcpyAsync(pp, pair, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const unsigned long long found = pp[0];
  if (found >= none) return TMAT_OK;
  const int64_t i = (int64_t)(found / (unsigned long long)N), j = (int64_t)(found % (unsigned long long)N);
  if (pair_out) {
    pair_out[0] = i;
    pair_out[1] = j;
  }
  return set_error(ctx, TMAT_EOVERLAP, "enclosing spheres of scatterers %lld and %lld intersect", (long long)i,
                   (long long)j);
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

extern "C" int tmat_check_overlap(tmat_ctx* ctx, const double* pos, int64_t N, const double* radii,
                                  int64_t* pair_out) {
  if (!ctx) return TMAT_EINVAL;
  if (N < 0 || (N > 0 && (!pos || !radii))) return set_error(ctx, TMAT_EINVAL, "tmat_check_overlap: bad arguments");
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  Staged sp, sr;
  TM_TRY(stage_in(ctx, "st_pos", pos, sizeof(double) * 3 * N, &sp));
  TM_TRY(stage_in(ctx, "st_rad", radii, sizeof(double) * N, &sr));
  return check_overlap(ctx, (const double*)sp.dev, (const double*)sr.dev, N, pair_out);
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
