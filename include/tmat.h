/*
 * tmat.h - C ABI of the B300 (sm_103a) T-matrix multiple-scattering library.
 *
 * The library solves the collective-scattering problem of arXiv 2107.09879,
 * App. I: N scatterers, each with a T-matrix in a vector-spherical-wave basis
 * truncated at multipole order nmax, coupled by translation coefficients, solved
 * matrix-free by GMRES, plus the adjoint gradient of App. IV and the sub-region
 * decomposition of the main text. Spheres on a plane are supported (all z equal).
 *
 * Conventions (used by every call)
 * --------------------------------
 *  - Wave number k = 2 pi n_bg / wavelength. Lengths in the caller's unit.
 *  - Coefficient index of one scatterer (App. I-B, Eq. def_tmatrix):
 *        n(l, m) = l(l+1) + m - 1 in [0, L),  L = nmax(nmax+2),
 *        flat    = p * L + n(l, m),   p = 0 (grad phi x r waves), p = 1 (curl of those),
 *    so one scatterer holds P = 2 L complex coefficients (P = 2 lmax(lmax+2), App. I-B).
 *  - Complex numbers are interleaved (re, im): tmat_c128 = two doubles.
 *  - Multi-RHS arrays are [R][N][P] (RHS-major, scatterer, coefficient).
 *  - Positions are [N][3] doubles.
 *
 * Memory and streams
 * ------------------
 *  - Array arguments may be device pointers or host pointers; the library asks
 *    the CUDA driver which one it got (cudaPointerGetAttributes). Host arrays are
 *    copied to library-owned device buffers on the context stream and results are
 *    copied back before the call returns. Device arrays are used in place.
 *  - The caller owns every array it passes. The library allocates only scratch
 *    (Krylov bases, tables, neighbour lists) from the context and frees it in
 *    tmat_ctx_destroy or tmat_solution_free.
 *  - All work is issued on the context stream. Calls that return status or
 *    iteration info synchronise that stream before returning.
 *  - A context is not thread-safe: one host thread at a time per context.
 *
 * Errors
 * ------
 *  Every call returns 0 (TMAT_OK) or a negative TMAT_E* code; tmat_last_error()
 *  gives a one-line message for the last failing call on that context. On error
 *  no output array is guaranteed to be written, except TMAT_ENOCONV, where the
 *  outputs hold the best iterate and the info struct says how far it got.
 */
#ifndef TMAT_H
#define TMAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TMAT_OK 0
#define TMAT_EINVAL (-1)     /* bad size, nmax outside 1..6, NaN input, non-coplanar lattice */
#define TMAT_EOVERLAP (-2)   /* the enclosing spheres of two scatterers intersect (App. I-C) */
#define TMAT_ENOMEM (-3)     /* device allocation failed */
#define TMAT_ENOCONV (-4)    /* iteration cap reached; outputs hold the best iterate */
#define TMAT_EBREAKDOWN (-5) /* GMRES breakdown with a non-zero residual */
#define TMAT_ECUDA (-6)      /* a CUDA runtime call failed */
#define TMAT_ENOTSUP (-7)    /* valid request this build does not implement */

#define TMAT_NMAX_MAX 6
#define TMAT_MAX_RHS 16

typedef struct { double re, im; } tmat_c128;
typedef struct { float re, im; } tmat_c64;

typedef struct tmat_ctx tmat_ctx;
typedef struct tmat_solution tmat_solution;

/* One spherical meta-atom: radius and complex refractive index of the sphere. */
typedef struct {
  double radius;
  double n_re;
  double n_im;
} tmat_atom;

/* Arithmetic of the iterated operator. */
enum {
  TMAT_PREC_FP64 = 0,  /* complex128 apply, vectors and Arnoldi */
  TMAT_PREC_MIXED = 1, /* complex64 apply and vectors inside GMRES; fp64 Arnoldi/Givens;
                          fp64-accurate refinement residual (iterative refinement). On the
                          lattice path with tensor cores enabled and nmax <= 4 the residual
                          uses the TMAT_PREC_FP64_TC apply. */
  TMAT_PREC_FP64_TC = 2, /* complex128 vectors and Arnoldi; the operator applied with fp64-class
                            accuracy (relative error ~1e-12) as exact products of 8-bit bf16
                            slices on the tensor cores. Lattice path, nmax <= 4 only
                            (TMAT_ENOTSUP otherwise). */
};

/* Which kernel applies the operator. */
enum {
  TMAT_PATH_AUTO = 0,      /* lattice path when opts.lattice_nx > 0, else neighbour path */
  TMAT_PATH_NEIGHBOUR = 1, /* neighbour-list (CSR) apply, blocks generated per pair */
  TMAT_PATH_LATTICE = 2,   /* rectangular lattice: one block per lattice offset, reused */
};

/* Options of tmat_solve. Zero-initialise, then set what you need. */
typedef struct {
  double tol;          /* stop when ||b - K x|| / ||b|| <= tol (true residual, fp64). 0 -> 1e-6 */
  int restart;         /* GMRES restart length m. 0 -> 40 */
  int max_iter;        /* cap on GMRES iterations in total (all restarts, all refinements). 0 -> 2000 */
  double cutoff;       /* interaction cutoff (inclusive, |x_i - x_j| <= cutoff); <= 0: every pair */
  int precision;       /* TMAT_PREC_* */
  double inner_tol;    /* mixed: relative tolerance of each inner fp32 solve. 0 -> 1e-4 */
  int path;            /* TMAT_PATH_* */
  int lattice_nx;      /* lattice path: sites per row; positions must be the row-major lattice */
  int lattice_ny;      /*   x = x0 + ix*pitch, y = y0 + iy*pitch, z = z0 */
  double lattice_pitch;
  double taper;        /* width of a raised-cosine fall-off of the coupling that ends at the cutoff:
                          pair weight 1 for d <= cutoff - taper, 0.5(1 + cos(pi (d - cutoff + taper)/taper))
                          up to the cutoff. 0: hard cutoff. Must be <= cutoff. */
  const double* enclosing_radii; /* nullable [N] (host or device): radius of each scatterer's enclosing
                          sphere; when given, the solve first checks that no two enclosing spheres
                          intersect (|x_i - x_j| < r_i + r_j; touching is allowed) and returns
                          TMAT_EOVERLAP naming the first such pair (App. I-C assumes none). */
} tmat_solve_opts;

/* Per-call result summary (host struct). */
typedef struct {
  int iterations;            /* GMRES iterations (applications of K), all RHS together */
  int refinements;           /* mixed: outer refinement steps */
  int converged;             /* 1 if every RHS met tol */
  int n_rhs;
  double rel_residual[TMAT_MAX_RHS]; /* final true ||b - K x|| / ||b|| per RHS (fp64) */
  double seconds;            /* wall time of the call */
} tmat_solve_info;

/* ---- context ------------------------------------------------------------ */

/* Create a context on `device`, issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). */
int tmat_ctx_create(int device, void* cuda_stream, tmat_ctx** out);
int tmat_ctx_set_stream(tmat_ctx* ctx, void* cuda_stream);
int tmat_ctx_destroy(tmat_ctx* ctx);
const char* tmat_last_error(const tmat_ctx* ctx);
/* Device memory this context holds as scratch (bytes, host int64): what it has allocated
 * for Krylov bases, block spectra, work grids and tables; freed by tmat_ctx_destroy. */
int tmat_ctx_memory(const tmat_ctx* ctx, int64_t* bytes_out);
/* Number of kernels this context has launched so far (for launch accounting). */
int64_t tmat_ctx_launch_count(const tmat_ctx* ctx);

/* Kernel timing for measurement: when enabled, CUDA events are recorded on the
 * context stream around every operator-apply launch. tmat_ctx_kernel_time
 * synchronises and returns the launch count and summed duration of one kernel
 * kind since timing was (re)enabled: "lattice_apply_fp32", "lattice_apply_fp64",
 * "nbr_apply_fp32", "nbr_apply_fp64". Enabling again resets the record.
 * enable = 0 off, 1 every launch, n > 1: in the Arnoldi iterations of the complex64 inner
 * solves only one iteration in n is timed (the events cost host and device time at every
 * launch); launches outside those iterations are all timed. TMAT_EINVAL for enable < 0. */
int tmat_ctx_set_timing(tmat_ctx* ctx, int enable);
/* Calls of one kernel kind since timing was (re)enabled, timed or not (with enable = n > 1
 * the timed launches of tmat_ctx_kernel_time are a sample of these). */
int tmat_ctx_kernel_calls(tmat_ctx* ctx, const char* kind, int64_t* calls);
/* Lattice operators (tmat_apply_lattice, the lattice path of tmat_solve, tmat_sweep)
 * are applied by FFT convolution when the grid fits (nx + max|dx| <= 1024 and
 * ny + max|dy| <= 1024): y_i = sum_o B_o x_{i+o} as a circular convolution on a
 * zero-padded power-of-two grid, one L x L block product per frequency, in the
 * operator's precision (complex64 or complex128 arithmetic throughout). enable = 0
 * selects the direct block-Toeplitz kernels (tensor cores / CUDA cores). Default: 1,
 * where the complex64 block products use the quad-mirror form (one symmetric matrix per
 * frequency quadruple (+-kx, +-ky), a quarter of the spectra read per apply); enable = 2
 * keeps the FFT with the mirror-pair products (one spectrum per pair (kx, +-ky)).
 * Timing kinds: "lattice_apply_fft32", "lattice_apply_fft64" (whole applies),
 * "lattice_fft_mul32", "lattice_fft_mul64" (the per-frequency block products). */
int tmat_ctx_set_lattice_fft(tmat_ctx* ctx, int enable);

/* Precision of near-field evaluations (tmat_field, tmat_point_fom, tmat_sweep's fields):
 * TMAT_PREC_FP64 (default) or TMAT_PREC_MIXED, where the distance, k|d| and its reduction
 * modulo 2 pi stay fp64 and the rest of each wave (sin/cos of the reduced phase, Hankel and
 * Legendre recurrences, products with complex64 copies of the coefficients) is fp32, summed in
 * fp64 across scatterers: relative error ~1e-7, for results of a mixed solve (1e-6 target).
 * Far-field amplitudes stay fp64. Timing kinds: "field64", "field32", "farfield". */
int tmat_ctx_set_field_precision(tmat_ctx* ctx, int precision);

/* Mixed-precision solves: inner complex64 GMRES solves whose tolerance is >= 1e-2 keep
 * their final Krylov vectors as fp16 pairs scaled by sqrt(n) (half the basis traffic; the
 * arithmetic stays fp32 and every refinement step is closed by the fp64-accurate residual),
 * enable = 1 (default); 0 keeps every basis in complex64. */
int tmat_ctx_set_compressed_basis(tmat_ctx* ctx, int enable);

/* Complex64 lattice applies run on the tcgen05 tensor cores (3xTF32, nmax <= 4)
 * unless disabled here (enable = 0: the CUDA-core fp32 kernel runs, and the mixed
 * refinement residual uses the fp64 CUDA-core kernel). enable = 1
 * (default) picks the window-view kernel where its windows fit in shared memory;
 * enable = 2 forces the gather kernel. Timing kinds: "lattice_apply_tcv" (window view),
 * "lattice_apply_tc" (gather), "lattice_apply_oz" (TMAT_PREC_FP64_TC apply). */
int tmat_ctx_set_tensor_cores(tmat_ctx* ctx, int enable);
int tmat_ctx_kernel_time(tmat_ctx* ctx, const char* kind, int64_t* launches, double* total_ms);
/* Algorithmic bytes (what the launches of `kind` must read and write: operands, basis
 * vectors, spectra; not cache re-reads) summed over the timed launches. Kinds with a
 * byte count: "arnoldi_dots32", "arnoldi_update32" (the complex64 Arnoldi passes),
 * "lattice_fft_mul32", "lattice_fft_mul64". */
int tmat_ctx_kernel_bytes(tmat_ctx* ctx, const char* kind, double* bytes);

/* Measured FMA issue rate of `device` in TFLOP/s (2 flop per fused multiply-add), the
 * denominator of the ALU-bound rooflines: precision TMAT_PREC_MIXED probes fp32 FMA,
 * TMAT_PREC_FP64 probes fp64 FMA. Every thread runs 16 independent FMA chains; the grid
 * fills every SM; the best of five ~5 ms launches on the legacy default stream of
 * `device` (synchronous). Not part of the method: a measurement utility. */
int tmat_measure_fma_peak(int device, int precision, double* tflops_out);

/* ---- geometry (integer, bit-exact) -------------------------------------- */

/* Interaction neighbour lists (a cutoff is this library's parameter; the paper
 * couples every pair, App. I-D). Source j is a neighbour of target i when j != i
 * and d2 <= cutoff*cutoff, with d2 = dx*dx + dy*dy + dz*dz evaluated in fp64 left
 * to right with every product and sum rounded (no fused multiply-add).
 * cutoff <= 0 couples every pair. Output CSR: row_ptr[N+1] (int64), col[nnz]
 * (int32, ascending within a row). Two passes: call with col == NULL to get
 * row_ptr and *nnz_out, allocate col, call again with the same row_ptr. */
int tmat_neighbors(tmat_ctx* ctx, const double* pos, int64_t N, double cutoff,
                   int64_t* row_ptr, int32_t* col, int64_t* nnz_out);

/* Enclosing-sphere overlap check (App. I-C: the method assumes that the enclosing spheres of
 * the scatterers do not intersect): returns TMAT_EOVERLAP when |x_i - x_j| < r_i + r_j for
 * some pair (fp64, every product and sum rounded; touching spheres pass), with the first
 * such pair (smallest i, then j) in pair_out[2] (nullable, host), else TMAT_OK. radii[N]
 * >= 0. Cell-binned: O(N) work. Host or device arrays; synchronises. */
int tmat_check_overlap(tmat_ctx* ctx, const double* pos, int64_t N, const double* radii, int64_t* pair_out);

/* Sub-region index sets (main text: jinc-source groups with a padding region;
 * Fig. 3 caption). On an nx x ny lattice (site index iy*nx + ix), sub-region
 * a = ay*nax + ax (nax = ceil(nx/cx)) has core sites ix in [ax*cx, (ax+1)*cx),
 * iy in [ay*cy, (ay+1)*cy) (clipped), and simulated sites = core grown by `buf`
 * on every side (clipped). Outputs: core_ptr[n_sub+1], core_idx[nx*ny],
 * sim_ptr[n_sub+1], sim_idx[sim_ptr[n_sub]] (int64, ascending per set). Pass
 * core_idx == sim_idx == NULL first to get the pointers and *sim_total_out. */
int tmat_subregions(tmat_ctx* ctx, int64_t nx, int64_t ny, int64_t cx, int64_t cy, int64_t buf,
                    int64_t* core_ptr, int64_t* core_idx, int64_t* sim_ptr, int64_t* sim_idx,
                    int64_t* n_sub_out, int64_t* sim_total_out);

/* ---- per-scatterer T-matrices (App. I-B; spheres: Lorenz-Mie) ---------- */

/* T_diag_out[N][P]: the diagonal of each sphere's T-matrix,
 * t_{l,p=0} = -b_l, t_{l,p=1} = -a_l (Bohren & Huffman Mie coefficients, relative
 * index n_sphere / n_bg, size parameter k r). dTdr_out (nullable): d t / d radius. */
int tmat_build(tmat_ctx* ctx, const tmat_atom* atoms, int64_t N, double wavelength, double n_bg,
               int nmax, tmat_c128* T_diag_out, tmat_c128* dTdr_out);

/* ---- null-field T-matrices of cylinders (App. I-B) ------------------------ */

/* An upright circular cylinder (axis along z, centred on its position) of complex
 * refractive index n_re + i n_im; its enclosing sphere has radius
 * sqrt(radius^2 + (height/2)^2). */
typedef struct {
  double radius;
  double height;
  double n_re;
  double n_im;
} tmat_cylinder;

/* Full T-matrices of n cylinders by the null-field method (App. I-B, the P and Q surface
 * integrals over the scatterer surface and T = -Q P^-1; the two terms of the integrand are
 * added): T_out[n][P][P] complex128, rows the outgoing (scattered) index, columns the
 * incident index, flat coefficient order. The body of revolution makes the azimuthal
 * integral exact (T couples m = m' only), and the profile integral uses n_quad Gauss-Legendre
 * nodes on each face (bottom disc, side, top disc; 0 -> 48; at most 512). A cylinder
 * centred on its position is z-mirror symmetric, so T preserves the class (l + m + p) mod 2.
 * dTdr_out (nullable): d T / d radius by a central difference of the same build (step
 * 1e-5 wavelengths in the background medium; relative error ~1e-9). n <= 65535 per call;
 * radius, height > 0, n_re > 0, n_im >= 0 (TMAT_EINVAL otherwise). Host or device arrays;
 * synchronises the context stream. */
int tmat_build_cylinder(tmat_ctx* ctx, const tmat_cylinder* cyl, int64_t n, double wavelength, double n_bg,
                        int nmax, int n_quad, tmat_c128* T_out, tmat_c128* dTdr_out);

/* ---- incident field (App. II-A) ----------------------------------------- */

/* Plane waves A_r exp(i k khat_r . x), khat = (sin b cos a, sin b sin a, cos b),
 * dirs[R][2] = (b, a) in radians, pol[R][3] complex polarisation (transverse).
 * a0_out[R][N][P] = exp(i k khat_r . x_i) a_lmp(b, a) (App. II-A, explicit forms). */
int tmat_incident_planewave(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength,
                            double n_bg, int nmax, const double* dirs, const tmat_c128* pol,
                            int R, tmat_c128* a0_out);

/* Incident coefficients of one group of jinc sources (App. II). Sources sit on
 * the plane z = z0 at src_xy[S][2] with transverse amplitudes src_A[R][S][2]
 * (one set per right-hand side, R <= 4) on a grid of pitch src_pitch (<= 0: the
 * paper's lambda/2 grid). Each source is the cell-weighted sample
 * (a^2/(4 pi^2)) int_{|k^T|<k0} A_s e^{i k^T.(x^T - x_s)} d^2k^T propagated along +z
 * (on z = z0 it is A_s (a^2 k0^2/(2 pi)) J1(k0 rho)/(k0 rho), = (pi/2) J1/(k0 rho) on the
 * lambda/2 grid); every plane-wave component is
 * completed to a transverse vector and expanded about each sphere (App. II-A).
 * The integral over the disc uses Gauss-Legendre in the polar angle (n_beta nodes
 * on [0, pi/2]) times the trapezoid rule in the azimuth (n_alpha nodes); with
 * n_beta or n_alpha <= 0 the rule is sized from the largest sphere-source
 * separation D (bounding boxes): n_beta = ceil(k0 D pi/4) + 24,
 * n_alpha = ceil(k0 D) + 32 rounded up to a multiple of 4.
 * precision: TMAT_PREC_FP64, or TMAT_PREC_MIXED (complex64 accumulation per node
 * tile with fp64-reduced phases, fp64 sums across tiles). a0_out[R][N][P]. */
int tmat_incident_jinc(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
                       int nmax, const double* src_xy, const tmat_c128* src_A, int64_t S, int R,
                       double z0, double src_pitch, int n_beta, int n_alpha, int precision,
                       tmat_c128* a0_out);

/* ---- translation coefficients (App. I-C, Eqs. tran_coeff) --------------- */

/* xi_out[M][P][P]: the outgoing-to-regular translation matrix xi(k d_m) for each
 * displacement d_m = disp[m] (any direction), rows (l,m,p), columns (l',m',p'):
 * Phi_{lmp}(k(x - x_a)) = sum xi_{lmp;l'm'p'}(k (x_b - x_a)) RPhi_{l'm'p'}(k(x - x_b)). */
int tmat_translation(tmat_ctx* ctx, int nmax, double k, const double* disp, int64_t M,
                     tmat_c128* xi_out);

/* ---- the operator (App. I-C/D) ------------------------------------------ */

enum {
  TMAT_OP_FORWARD = 0, /* y = x - T (A x)      : K = M Omega of App. I-C with M = diag(T) */
  TMAT_OP_ADJOINT = 1, /* y = x - A^T (T x)    : the transposed operator of App. IV */
  TMAT_OP_COUPLE = 2,  /* y = A x              : field incident from the other scatterers */
};

/* One application of the operator to R vectors x[R][N][P] -> y[R][N][P], with
 * A_ij = w(|x_i - x_j|) xi(k(x_i - x_j))^T for j in the CSR row of i (row_ptr/col
 * from tmat_neighbors), w the coupling window of tmat_solve_opts (cutoff, taper;
 * taper 0 gives w = 1). precision: TMAT_PREC_FP64 (complex128 arithmetic) or
 * TMAT_PREC_MIXED (complex64 arithmetic; x and y are still complex128 here);
 * TMAT_PREC_FP64_TC only on the lattice (tmat_apply_lattice).
 * Coplanar positions (equal z) use the parity-class split of the blocks; otherwise every
 * block is formed in full from the 3-D coupling constants (nmax <= 5, TMAT_ENOTSUP above;
 * blocks in fp64, vectors in the requested precision). The same holds for tmat_solve on
 * the neighbour path (the lattice path needs a common plane: TMAT_EINVAL) and for
 * tmat_adjoint of such a solution. Non-finite coordinates: TMAT_EINVAL. */
int tmat_apply(tmat_ctx* ctx, int op, int precision, const double* pos, int64_t N, double k,
               int nmax, const tmat_c128* T_diag, const int64_t* row_ptr, const int32_t* col,
               double cutoff, double taper, const tmat_c128* x, int R, tmat_c128* y);

/* The same operator on a row-major nx x ny lattice with spacing `pitch`
 * (site index iy*nx + ix, all z equal): one translation block per lattice
 * offset inside the cutoff (offset test (dx*pitch)^2 + (dy*pitch)^2 <= cutoff^2,
 * cutoff <= 0: every pair; `taper` as in tmat_solve_opts), reused by all pairs
 * with that offset. Same modes,
 * precisions and layouts as tmat_apply. */
int tmat_apply_lattice(tmat_ctx* ctx, int op, int precision, int nx, int ny, double pitch, double cutoff,
                       double taper, double k, int nmax, const tmat_c128* T_diag, const tmat_c128* x, int R,
                       tmat_c128* y);

/* ---- solve (App. I-C/D) -------------------------------------------------- */

/* Solve (I - T A) s = T a0 for R <= TMAT_MAX_RHS right-hand sides by restarted
 * GMRES, x0 = 0. T_diag[N][P] from tmat_build; a0[R][N][P]; s_out[R][N][P]. With
 * TMAT_PREC_MIXED the solve is iterative refinement: fp64-accurate residual,
 * inner GMRES with a complex64 operator to opts.inner_tol. `keep` (nullable)
 * receives an opaque solution object that holds what tmat_adjoint needs
 * (positions, T, a0, s, neighbour lists); free it with tmat_solution_free.
 * info (nullable, host). */
int tmat_solve(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
               int nmax, const tmat_c128* T_diag, const tmat_c128* a0, int R,
               const tmat_solve_opts* opts, tmat_c128* s_out, tmat_solution** keep,
               tmat_solve_info* info);
int tmat_solution_free(tmat_solution* sol);

/* The same solve with full per-scatterer T-blocks (App. I-B, Eq. def_tmatrix: s_i = T_i a_i
 * with T_i a P x P matrix, e.g. from tmat_build_cylinder): (I - T A) s = T a0 with
 * T = diag(T_1 .. T_N).
 *   T_blocks[n_types][P][P]  complex128, rows outgoing index, columns incident index;
 *   type[N]                  int32 index into T_blocks per scatterer (nullable: scatterer i
 *                            uses block i, n_types must equal N); an index outside
 *                            [0, n_types) returns TMAT_EINVAL.
 * A block may couple every index (no class or m structure is assumed). The operator applies
 * A (forward: coupling only) and then the blocks per scatterer; the transposed operator
 * applies T^T first. Paths, precisions (TMAT_PREC_FP64 or TMAT_PREC_MIXED; TMAT_PREC_FP64_TC
 * returns TMAT_ENOTSUP), options, layouts and errors as tmat_solve. `keep` receives a solution
 * for tmat_adjoint_tblocks. */
int tmat_solve_tblocks(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg, int nmax,
                       const tmat_c128* T_blocks, const int32_t* type, int64_t n_types, const tmat_c128* a0,
                       int R, const tmat_solve_opts* opts, tmat_c128* s_out, tmat_solution** keep,
                       tmat_solve_info* info);

/* ---- batched independent problems (served sub-region jobs) --------------- */

/* One lattice problem of a batch: an nx x ny row-major lattice (site iy*nx + ix at
 * (ix*pitch, iy*pitch, 0)), its own wavelength, T_diag[nx*ny][P] (tmat_build at that
 * wavelength), one incident set a0[nx*ny][P] and the output s_out[nx*ny][P]. */
typedef struct {
  int nx, ny;
  double wavelength;
  const tmat_c128* T_diag;
  const tmat_c128* a0;
  tmat_c128* s_out;
} tmat_batch_problem;

/* Solve n <= TMAT_MAX_RHS independent lattice problems of one nmax (the sub-region jobs of
 * the main text) together: each is placed at the origin of a canvas_nx x canvas_ny canvas
 * lattice (0: the largest problem's size) with T = 0 and a0 = 0 on the sites it does not
 * own, which leaves its solution unchanged, and the problems become the right-hand sides of
 * one batched operator on the FFT lattice path: every kernel launch of the apply (with each
 * problem's own block spectra and T) and of GMRES covers the whole batch, and a problem
 * that has converged leaves the Arnoldi work. A problem's result depends only on its own
 * data and the canvas size (fix the canvas per size class to make results independent of
 * the rest of the batch). opts: tol, restart, max_iter, cutoff, taper, inner_tol and
 * precision (TMAT_PREC_FP64 or TMAT_PREC_MIXED) as tmat_solve; the path is the lattice.
 * infos[n] (nullable, host): per problem (iterations and refinements are the batch's).
 * TMAT_ENOTSUP when the canvas does not fit the FFT operator; TMAT_ENOCONV when some
 * problem did not converge (every output holds its best iterate). Host or device arrays;
 * synchronises. */
int tmat_solve_batch(tmat_ctx* ctx, const tmat_batch_problem* probs, int n, double n_bg, int nmax, double pitch,
                     int canvas_nx, int canvas_ny, const tmat_solve_opts* opts, tmat_solve_info* infos);

/* ---- sub-region sweep (main text; Fig. 3) -------------------------------- */

/* Geometry and decomposition of a large-area sweep. Sites (ix, iy) of an
 * nx x ny lattice sit at (x0 + ix*pitch, y0 + iy*pitch, z); every site also
 * carries one jinc source on the plane z = z0 at the site's (x, y) (the
 * lambda/2 sampling of App. II, so pitch should not exceed wavelength/(2 n_bg)).
 * Sub-region a = ay*nax + ax has the core [ax*core_x, (ax+1)*core_x) x
 * [ay*core_y, ...) and simulates the core grown by `buffer` sites on every side
 * (clipped), as tmat_subregions. Sub-regions [first, first + count) are processed
 * (count <= 0: all), so a sweep can be split into resumable pieces. */
typedef struct {
  int nx, ny;
  double pitch, x0, y0, z;
  int core_x, core_y, buffer;
  double z0;
  int n_beta, n_alpha;  /* jinc rule per sub-region (<= 0: sized per sub-region) */
  int first, count;
} tmat_sweep_opts;

typedef struct {
  int subregions;          /* processed by this call */
  int total_subregions;
  int unconverged;
  int iterations;          /* GMRES iterations summed over sub-regions */
  int64_t scatterer_solves;/* sum of padded sub-region sizes */
  double worst_rel_residual;
  double seconds;
} tmat_sweep_info;

/* For every sub-region: T-matrices of the padded set (atoms[nx*ny]), jinc-group
 * incident coefficients of the core's sources (src_A[R][nx*ny][2] transverse
 * amplitudes, R <= 4), the solve (opts; the lattice path is forced), and the
 * scattered field of the padded set at the detectors pts[M][3], ADDED to
 * E_out[R][M][3] in sub-region order. The sum over all sub-regions is the
 * decomposed scattered field of the whole array (the paper adds the sub-region
 * fields). */
int tmat_sweep(tmat_ctx* ctx, const tmat_sweep_opts* sw, const tmat_atom* atoms, double wavelength,
               double n_bg, int nmax, const tmat_c128* src_A, int R, const tmat_solve_opts* opts,
               const double* pts, int64_t M, tmat_c128* E_out, tmat_sweep_info* info);

/* ---- one forward simulation in a single call (App. I) -------------------- */

/* The whole forward step of App. I for spheres: Lorenz-Mie T-matrices of atoms[N]
 * (tmat_build), plane-wave incident coefficients of the R <= TMAT_MAX_RHS incidences
 * dirs[R][2] = (beta, alpha) with polarisations pol[R][3] (tmat_incident_planewave),
 * the solve (I - T A) s = T a0 with opts (tmat_solve; the mixed and fp64 paths, the
 * lattice path when opts asks for it), and the scattered field of every incidence at
 * pts[M][3] (tmat_field). Each pointer may be host or device memory; T, a0 and s stay
 * on the device (context scratch) between the steps, host inputs are copied in and host
 * outputs copied back. s_out[R][N][P] (nullable: not returned), E_out[R][M][3] (nullable
 * when M = 0), info (nullable, host). Returns what tmat_solve returns (TMAT_ENOCONV: the
 * outputs hold the best iterate and its field); argument errors as the four calls. */
int tmat_forward(tmat_ctx* ctx, const double* pos, int64_t N, const tmat_atom* atoms, double wavelength,
                 double n_bg, int nmax, const double* dirs, const tmat_c128* pol, int R,
                 const tmat_solve_opts* opts, const double* pts, int64_t M, tmat_c128* s_out,
                 tmat_c128* E_out, tmat_solve_info* info);

/* ---- fields (App. I-C, Eq. sca_fld_concise) ------------------------------ */

/* E_out[M][3] = sum_i s_i^T Phi(k(x - x_i)) at the points pts[M][3] (scattered
 * field of coefficients s[N][P]). Points must not coincide with a centre. */
int tmat_field(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
               int nmax, const tmat_c128* s, const double* pts, int64_t M, tmat_c128* E_out);

/* Far-field amplitude F(rhat) with E_sca(r rhat) -> e^{ikr}/(kr) F(rhat),
 * dirs[M][2] = (theta, phi). */
int tmat_farfield(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
                  int nmax, const tmat_c128* s, const double* dirs, int64_t M, tmat_c128* F_out);

/* ---- adjoint (App. IV) ---------------------------------------------------- */

/* Point figure of merit FoM = sum_c |E_inc,c(x_f) + E_sca,c(x_f)|^2 (App. IV,
 * Eq. performance_metric with a point detector and f = |.|^2) and its adjoint
 * source v[N][P] = dFoM/ds in the sense dFoM = 2 Re(v^T ds),
 * v_i = sum_c conj(E_c) Phi_c(k(x_f - x_i)). E_inc_f: the incident field at x_f
 * (3 complex). fom_out: host double. v_out nullable. */
int tmat_point_fom(tmat_ctx* ctx, const double* pos, int64_t N, double wavelength, double n_bg,
                   int nmax, const tmat_c128* s, const double* x_f, const tmat_c128* E_inc_f,
                   double* fom_out, tmat_c128* v_out);

/* Radius gradient of a figure of merit whose adjoint source is v[N][P] (App. IV,
 * Eq. grad_geometry_overlap): solves (I - A^T T) mu = v with the operator,
 * precision and tolerance of the forward solve kept in `sol`, then
 * grad_out[i] = 2 Re sum_n mu_{i,n} dTdr_{i,n} e_{i,n}, e = a0 + A s (RHS 0 of sol).
 * dTdr[N][P] from tmat_build. mu_out (nullable) receives mu. */
int tmat_adjoint(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* v,
                 const tmat_c128* dTdr, double* grad_out, tmat_c128* mu_out,
                 tmat_solve_info* info);

/* Parameter gradient of a figure of merit for a T-block solution of tmat_solve_tblocks
 * (App. IV): solves (I - A^T T^T) mu = v and returns
 * grad_out[i] = 2 Re mu_i^T (dT_{type_i} e_i),  e = a0 + A s (RHS 0 of sol),
 * with dT_blocks[n_types][P][P] the derivative of each T-block with respect to its
 * scatterer's parameter (e.g. dTdr_out of tmat_build_cylinder), indexed by the solve's types.
 * mu_out (nullable) receives mu. TMAT_EINVAL for a solution of tmat_solve. */
int tmat_adjoint_tblocks(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* v, const tmat_c128* dT_blocks,
                         double* grad_out, tmat_c128* mu_out, tmat_solve_info* info);

/* Position gradient of the point figure of merit: dFoM/d(x_i, y_i) for every scatterer
 * (App. IV, with the in-plane positions as the geometry parameters). Lattice solutions
 * (TMAT_PATH_LATTICE) only: the derivative is taken at the lattice configuration, where
 * the derivative blocks dF/dd of the coupling (window included) depend only on the offset.
 *   mu[N][P]        the adjoint solution for this figure of merit (tmat_adjoint's mu_out);
 *   da0_dx, da0_dy  [N][P] d a0_i / d x_i and d a0_i / d y_i of the incident coefficients
 *                   (for a plane wave of wave vector k_inc: i k_inc,x a0_i and i k_inc,y a0_i);
 *                   both NULL when the incident field does not move with the scatterers;
 *   x_f[3], E_f[3]  the focal point and the total field there (incident + scattered);
 *   grad_out[N][2]  dFoM/dx_i, dFoM/dy_i.
 * grad = 2 Re[(T mu)_i . (A'_q s + da0_q)_i - (A'_q^T T mu)_i . s_i] + the explicit term
 * 2 Re sum_c conj(E_c) s_i . d Phi_c(k(x_f - x_i)) / d q_i, the latter by a central
 * difference of the fp64 wave functions (step 1e-4 / k, relative error ~2e-9). The two
 * derivative operators are applied in fp64 (four applies), by FFT convolution with their
 * own block spectra where the lattice grid fits, else on the CUDA cores.
 * Errors: TMAT_EINVAL (NULL required argument, only one of da0_dx/da0_dy, wrong device),
 * TMAT_ENOTSUP (neighbour-path solution). All arrays host or device. */
int tmat_position_gradient(tmat_ctx* ctx, const tmat_solution* sol, const tmat_c128* mu,
                           const tmat_c128* da0_dx, const tmat_c128* da0_dy, const double* x_f,
                           const tmat_c128* E_f, double* grad_out);

/* ---- allocation-free variant (no counterpart in the paper) ------------------ */

/* Capacity of the fixed device scratch of tmat_field_noalloc, in complex
 * partial sums; a call needs 3 * M of them, so M <= TMAT_NOALLOC_FIELD_SLOTS / 3. */
#define TMAT_NOALLOC_FIELD_SLOTS 65536

/* Scattered field like tmat_field, for callers that must not allocate device
 * memory during a call: code that runs inside another framework's fixed device
 * memory budget, or in a loop where a cudaMalloc/cudaFree (which may
 * synchronise the whole device and stall work on other streams) is not
 * acceptable. It takes no context, allocates nothing (no cudaMalloc, cudaFree
 * or pinned host memory) and uses a fixed 1 MiB scratch array that lives in the
 * library's device image (every GPU that loads the library keeps it until the
 * process exits).
 *  - All array arguments must be device (or managed) memory of the current
 *    device; host pointers and pointers into another GPU's memory are rejected
 *    with TMAT_EINVAL. Work is issued on `cuda_stream` (a cudaStream_t of the
 *    current device, NULL = legacy default stream); after the first call on a
 *    device (below) a call does not synchronise.
 *  - M above TMAT_NOALLOC_FIELD_SLOTS / 3 points, N < 0, nmax outside
 *    1..TMAT_NMAX_MAX or a bad pointer returns TMAT_EINVAL before any work is
 *    issued (there is no context, so there is no error message). A CUDA error
 *    left pending by the caller's earlier work is reported as TMAT_ECUDA and
 *    left pending (not cleared); errors of this call's own launches are
 *    consumed and reported as TMAT_ECUDA.
 *  - The first call on each device does a one-time set-up: it looks up the
 *    scratch array's device address and copies the Legendre recurrence
 *    constants from host memory into the library's constant memory on
 *    `cuda_stream`, then synchronises `cuda_stream`. Make that first call
 *    before any stream capture begins.
 *  - All calls on one device share its scratch array: two calls whose work
 *    overlaps on that GPU (for example on two streams) race and give wrong
 *    results; order them (one stream, or events). Every scratch slot a call
 *    reads is written earlier in the same call, so nothing needs clearing. */
int tmat_field_noalloc(void* cuda_stream, const double* pos, int64_t N, double wavelength, double n_bg,
                       int nmax, const tmat_c128* s, const double* pts, int64_t M, tmat_c128* E_out);

#ifdef __cplusplus
}
#endif

#endif /* TMAT_H */
