/*
 * tpt.h -- C ABI of the GB300 tensor-product--Thomas Poisson/Helmholtz solver.
 *
 * The library solves, on one GPU, the constant-coefficient problem
 *
 *     (alpha I + beta L) phi = f
 *
 * on a staggered, cell-centred Cartesian grid with non-uniform spacing in every
 * direction (paper Sec. 2.2).  L is the Kronecker sum of the three 1D
 * second-difference operators of Eq. (poisson-fd2)/(tridiagonal-coefficients)
 * (Sec. 2.2.2).  Poisson is (alpha, beta) = (0, 1); the Crank--Nicolson
 * Helmholtz problem of Sec. 2.1 is (1, -gamma nu dt / 2).  The x and y
 * operators are diagonalised in their numerical eigenbases (Sec. 2.2.1,
 * Eq. reverse-similarity-transform, Eq. q-from-tildeq), or by FFT/DCT in a
 * uniform direction; one tridiagonal system per (i, j) mode pair remains along
 * z and is solved by the Thomas algorithm (Sec. 2.2.2, solution steps 2.1-2.5;
 * Algorithm 1 steps 1, 3, 5, 7, 9).
 *
 * Conventions shared by every entry point:
 *  - Fields are float64, Fortran order (Nx, Ny, Nz): x fastest, element
 *    (i, j, k) at i + Nx*(j + Ny*k).
 *  - Every call returns an int status (TPT_OK = 0); no exception or abort
 *    crosses the ABI.  tpt_status_string() names a status.
 *  - Pointers named *_dev are device pointers on the plan's device; pointers
 *    named *_host are host pointers.  The caller owns every buffer it passes;
 *    the plan owns only its own device tables (eigenbases, eigenvalues,
 *    operator rows) and frees them in tpt_plan_destroy().
 *  - Calls taking a `stream` (a cudaStream_t passed as void*, NULL = legacy
 *    default stream) are asynchronous on that stream unless stated otherwise.
 */
#ifndef TPT_H
#define TPT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TPT_OK                 0
#define TPT_ERR_INVALID_ARG    1  /* null pointer, size <= 0, bad enum, bad spacing */
#define TPT_ERR_UNSUPPORTED    2  /* valid request this build does not implement    */
#define TPT_ERR_OOM            3  /* device allocation failed                        */
#define TPT_ERR_CUDA           4  /* a CUDA runtime/driver call failed               */
#define TPT_ERR_NOT_CONVERGED  5  /* refinement did not reach rtol in max_refine     */
#define TPT_ERR_TIMEOUT        6  /* a bounded device-side wait gave up              */
#define TPT_ERR_NONFINITE      7  /* NaN/Inf in the right-hand side or residual      */
#define TPT_ERR_NUMERICAL      8  /* eigensolver failed or null pivot did not vanish */
#define TPT_PENDING            9  /* a served request has not finished yet          */

/* ---- enumerations ---------------------------------------------------- */
/* Boundary rows of Sec. 2.2.1 ("modified as required by the boundary
 * conditions"): Neumann drops the outside coupling; periodic keeps it as the
 * cyclic corner (set on both ends); homogeneous Dirichlet (zero wall value at
 * the face) drops it and adds 2/dx^2 to -b of that row.  DIRICHLET_NODE is
 * homogeneous Dirichlet with the zero value at the neighbouring node, a
 * centre spacing away (dxc[0] below the first unknown, dxc[n] above the
 * last): the coupling is dropped and its coefficient kept on the diagonal;
 * this is the wall row of face-centred unknowns (the wall-normal velocity,
 * see tpt_grid_faces).  NONE (on both ends of x and/or y) removes the
 * direction from the operator: the implicit-diffusion options of Sec. 2.1 /
 * Sec. 3 in which only y, z ("yz") or only z ("z") are implicit, so the
 * problem decouples along the removed direction and no transform runs along
 * it (its eigenbasis is the identity with zero eigenvalues); it needs
 * alpha != 0 and never applies to z.                                       */
enum { TPT_BC_PERIODIC = 0, TPT_BC_NEUMANN = 1, TPT_BC_DIRICHLET = 2, TPT_BC_DIRICHLET_NODE = 3,
       TPT_BC_NONE = 4 };

/* Transform of a diagonalised direction (x or y), Sec. 3: numerical eigenbasis
 * applied as a GEMM, or the Fourier-based transform of a uniform direction
 * (real DFT for periodic, DCT-II/III for Neumann-Neumann; Makhoul's
 * reordering, footnote to Sec. 4.2).  FFT needs uniform spacing and a
 * power-of-two size (16 to 4096 points on a mixed-precision plan, whose
 * corrections then transform that direction in float32 instead of on the
 * tensor cores).  AUTO picks it where it applies on float64 and Ozaki plans
 * and keeps the GEMM on mixed-precision plans.                             */
enum { TPT_XFORM_AUTO = 0, TPT_XFORM_GEMM = 1, TPT_XFORM_FFT = 2 };

/* Arithmetic of the transforms and the Thomas sweep.  FP64: float64
 * throughout.  MIXED_*: correction solves with the transforms on the tensor
 * cores (BF16, split BF16 with three products, or TF32; FP32 accumulation),
 * FP32 Thomas except the singular null line (float64), and a float64
 * residual driving iterative refinement to `rtol`.  FP64_OZAKI: the float64
 * solve with its eigenbasis-transform GEMMs on the bf16 tensor cores by the
 * Ozaki scheme (each operand row split into seven bf16 slices of six bits,
 * slice products summed exactly in float32 level by level and the levels in
 * float64; ~1e-13 of sum |a||b| per product) -- float64-accurate after the
 * plan's float64 refinement steps, everything else as FP64; GEMM directions
 * of at most 576 points (else UNSUPPORTED).  Reported as TPT_PREC_FP64 by the
 * plan's inspection calls.                                                   */
enum { TPT_PREC_FP64 = 0, TPT_PREC_MIXED_BF16 = 1, TPT_PREC_MIXED_BF16X3 = 2,
       TPT_PREC_MIXED_TF32 = 3, TPT_PREC_FP64_OZAKI = 4 };

/* ---- plan ------------------------------------------------------------ */
typedef struct tpt_plan_s* tpt_plan;

typedef struct {
  int n[3];              /* Nx, Ny, Nz >= 1                                        */
  const double* dxf[3];  /* host, n[d] cell widths dx_i > 0 (copied at create)     */
  const double* dxc[3];  /* host, n[d]+1 centre spacings: dxc[i] = distance between
                            the centres of cells i-1 and i (1 <= i < n); dxc[0] and
                            dxc[n] are the wrap spacing, read only when periodic   */
  int bc[3][2];          /* lower/upper boundary per direction (TPT_BC_*)          */
  int xform[2];          /* transform for x and y (TPT_XFORM_*); z is Thomas       */
  double alpha, beta;    /* operator alpha I + beta L                              */
  int precision;         /* TPT_PREC_*                                             */
  double rtol;           /* refinement target ||f - A phi||_2 / ||f||_2; <= 0 runs
                            exactly max_refine refinement steps with no host sync  */
  int max_refine;        /* refinement steps after the first solve (>= 0)          */
} tpt_desc;

typedef struct {
  int iters;             /* correction solves performed (first solve included)     */
  double rel_residual;   /* last ||f - A phi||_2 / ||f||_2 (f after projection);
                            -1 when no residual was evaluated                      */
  double compat_defect;  /* singular problems: cell-volume-weighted mean removed
                            from f to make it compatible; 0 otherwise              */
  float ms_stage[8];     /* with tpt_set_stage_timing(plan, 1), mixed plans: GPU
                            milliseconds: [0] input conversion, summed over the
                            corrections [1] x forward, [2] y forward, [3] Thomas,
                            [4] y inverse, [5] x inverse, [6] residual, and [7]
                            gauge and float64 output; 0 otherwise                 */
} tpt_info;

/* Build a plan on CUDA device `cuda_device` (or, with cuda_device < 0, a
 * host-only plan holding the setup tables for inspection through
 * tpt_plan_eigenvalues / tpt_plan_rows; every device entry point rejects it
 * with INVALID_ARG).  Setup: 1D rows with boundary rows,
 * symmetrisation D^{1/2} T D^{-1/2}, symmetric eigendecomposition on the host
 * in float64 with eigenvalues refined as long-double Rayleigh quotients, the
 * forward/inverse transform matrices Q^{-1} = Q~^T D^{1/2}, Q = D^{-1/2} Q~
 * (Sec. 2.2.1 steps 1.1-1.3; Algorithm 1 initialisation), and their upload.
 * For a TPT_PREC_MIXED_* plan the transform matrices are also rounded to
 * the operand format on the device.
 * Synchronous.  Errors: INVALID_ARG (bad descriptor), UNSUPPORTED (FFT on a
 * non-uniform direction, periodic z, a product of two sizes of 2^31 or
 * more), NUMERICAL (eigensolver did not
 * converge), OOM, CUDA.  On error *out is set to NULL.                    */
int tpt_plan_create(const tpt_desc* desc, int cuda_device, tpt_plan* out);

/* Bytes of device workspace tpt_solve() needs (256-byte aligned).          */
int tpt_workspace_bytes(tpt_plan plan, size_t* bytes);

/* Solve (alpha I + beta L) phi = f.  f_dev and phi_dev hold Nx*Ny*Nz float64
 * (phi_dev may equal f_dev); work_dev holds tpt_workspace_bytes() bytes, is
 * 256-byte aligned and is not used concurrently by another call.  With
 * rtol > 0 the call reads the residual norm on the host after every
 * correction (so it synchronises `stream`) and stops at rtol; otherwise it
 * runs 1 + max_refine corrections asynchronously.  A singular problem
 * (alpha = 0, every direction periodic or Neumann-Neumann) is solved for the
 * solution with zero cell-volume-weighted mean after removing that mean from
 * f.  `info` may be NULL; it is filled when the call returns if rtol > 0,
 * else after `stream` is synchronised.  Errors: INVALID_ARG, CUDA,
 * NOT_CONVERGED (phi holds the last iterate), NONFINITE (a NaN or Inf in f
 * or in a residual; the float64 path reports it as a status when rtol > 0,
 * otherwise as a non-finite info->rel_residual once `stream` is
 * synchronised), TIMEOUT.                                                  */
int tpt_solve(tpt_plan plan, const double* f_dev, double* phi_dev, void* work_dev,
              void* stream, tpt_info* info);

/* End-to-end solve from host memory: copies f_host to the device, solves, and
 * copies phi back to phi_host, all on `stream`; returns after the stream is
 * synchronised.  Device buffers: f_dev/phi_dev staging of Nx*Ny*Nz doubles
 * (may be equal) and work_dev as for tpt_solve().  Pinned host memory gives
 * full copy bandwidth.                                                     */
int tpt_solve_host(tpt_plan plan, const double* f_host, double* phi_host, double* f_dev,
                   double* phi_dev, void* work_dev, void* stream, tpt_info* info);

/* Change alpha and beta of an existing plan: the eigenbases do not depend on
 * them (Sec. 2.2.2: Poisson and Helmholtz share eigenvectors; Helmholtz is a
 * modal shift).  Not to be called while a solve on this plan is in flight.  */
int tpt_set_coefficients(tpt_plan plan, double alpha, double beta);

int tpt_plan_destroy(tpt_plan plan);
const char* tpt_status_string(int status);

/* ---- single steps of the solve (the same kernels tpt_solve launches) ---- */
/* Forward or inverse transform along x (dir = 0) or y (dir = 1) in float64:
 * forward applies Q^{-1} (Eq. forward-xy), inverse applies Q (Eq. inverse-xy),
 * with whichever transform the plan chose for that direction.  in_dev and
 * out_dev hold Nx*Ny*Nz doubles and must not overlap.                      */
int tpt_transform(tpt_plan plan, int dir, int inverse, const double* in_dev, double* out_dev,
                  void* stream);

/* Modal tridiagonal solve along z for every (i, j) (solution step 2.3):
 * (alpha + beta(lx_i + ly_j)) phi + beta T_z phi = fhat, float64, in place
 * allowed.  For a singular problem the null line is projected to compatible
 * form, its last modal unknown set to zero and the line shifted to zero
 * dz-weighted mean.  scratch_dev holds Nx*Ny*Nz doubles.                   */
int tpt_thomas(tpt_plan plan, const double* fhat_dev, double* phihat_dev, double* scratch_dev,
               void* stream);

/* Same computation and arguments as tpt_thomas(), for callers that cannot
 * allocate device memory when they call the solver (code inside a host
 * callback or a framework hook where CUDA allocation calls are not allowed,
 * callers whose device memory is owned by another allocator's pool, and
 * latency-sensitive callers that cannot pay for cudaFree's implicit
 * device-wide synchronisation).  The paper has no counterpart: this is a
 * packaging variant of the Thomas step.  It allocates nothing: the
 * elimination scratch is a fixed 32 MiB device array inside the library
 * (every GPU that loads the library holds it until the process exits), so
 * the field may have at most 4,194,304 points (Nx*Ny*Nz); larger plans get
 * TPT_ERR_UNSUPPORTED.  The first call on a device looks up the array's
 * device address on that device (make that first call before any stream
 * capture) and keeps it for the life of the process, like the device tables
 * of a plan: after cudaDeviceReset (or anything else that destroys the
 * device's primary context) neither this entry point nor any plan created
 * before it may be used again.  All calls share the one array, so calls whose kernels overlap on
 * the GPU race and give wrong results: serialise them (one stream, or events).
 * The scratch is fully rewritten before it is read, so nothing needs clearing
 * between calls.  The compatibility constant of a singular problem is not
 * reported.  Errors: INVALID_ARG, UNSUPPORTED (too large), CUDA.          */
int tpt_thomas_noalloc(tpt_plan plan, const double* fhat_dev, double* phihat_dev, void* stream);

/* r = f - (alpha I + beta L) phi with the 7-point stencil of the plan's 1D rows
 * (Sec. 4.1 residual), float64.  sums_dev (may be NULL) receives 3 doubles:
 * sum r^2, sum r, sum vol*r.                                               */
int tpt_residual(tpt_plan plan, const double* f_dev, const double* phi_dev, double* r_dev,
                 double* sums_dev, void* stream);

/* Tensor-core GEMM of the mixed-precision transforms on its own, for kernel
 * tests: D = A B^T with A (M x K) and B (N x K) row-major float64 on the
 * device, rounded to the operand format of `precision` (TPT_PREC_MIXED_*:
 * bf16, bf16 hi/lo pair with three products, tf32), multiplied with
 * tcgen05.mma in float32, and written to D column-major (element (m, n) at
 * m + M*n) as float64.  tile: column-tile width (0 = default, else 32, 64,
 * 128, 256); pair: two-CTA clusters sharing an operand tile (0 none, 1 pairs
 * of m-tiles share B, 2 pairs of n-tiles share A; used for split bf16 with
 * 128/256-column tiles and an even tile count, else ignored).  Runs on the
 * current device; work_dev is 256-byte aligned scratch of at least
 * 8*(M+N)*(K+8) + 1024 bytes.                                               */
int tpt_tc_gemm(int precision, int M, int N, int K, const double* A_dev, const double* B_dev,
                double* D_dev, void* work_dev, void* stream, int tile, int pair);

/* The same GEMM writing one of the transforms' intermediate formats, for
 * kernel tests of the output paths: element (m, n) of D goes to index
 *   (m % rm) + (m / rm) * sm + n * sn
 * of out0 (and of out1, the low part, for TPT_GEMM_OUT_SPLIT_BF16), as
 * float32 (TPT_GEMM_OUT_F32), bf16 rounded to nearest (TPT_GEMM_OUT_BF16) or
 * a bf16 hi/lo pair (TPT_GEMM_OUT_SPLIT_BF16: hi = bf16(d), lo = bf16(d - hi)).
 * tma_out = 1 lets the kernel stage each 32 x 32 output chunk in shared
 * memory and store it with a bulk tensor copy, where the layout allows it
 * (128/256-column tiles; rm >= M, or rm a multiple of 32 dividing M; 16-byte
 * aligned bases and strides); 0 forces per-thread stores.  pair: two-CTA
 * clusters as in tpt_tc_gemm.  Elements outside the index set are left
 * untouched.  Output buffers are the caller's, on the
 * current device; other arguments as tpt_tc_gemm.  TPT_ERR_INVALID_ARG for
 * an unknown kind, a non-positive size or rm, or a null pointer.           */
#define TPT_GEMM_OUT_F32 0
#define TPT_GEMM_OUT_BF16 1
#define TPT_GEMM_OUT_SPLIT_BF16 2
int tpt_tc_gemm_out(int precision, int M, int N, int K, const double* A_dev, const double* B_dev,
                    int out_kind, int rm, long long sm, long long sn, void* out0_dev, void* out1_dev,
                    void* work_dev, void* stream, int tile, int tma_out, int pair);

/* Host copies of the plan's tables, for inspection and tests.  lam: n[dir]
 * eigenvalues of direction dir (0 = x, 1 = y) in the plan's mode order;
 * a, b, c: the 1D rows of direction dir (0..2), n[dir] each.              */
int tpt_plan_eigenvalues(tpt_plan plan, int dir, double* lam_host);
/* Transform the plan chose for x and y (TPT_XFORM_GEMM or TPT_XFORM_FFT; AUTO
 * resolves to FFT on a uniform power-of-two periodic or Neumann-Neumann
 * direction of a float64 plan).  For FFT directions the mode order is the
 * real-DFT half-complex order (periodic: constant, cos 1, sin 1, ..., Nyquist)
 * or the DCT-II order (Neumann), and lam holds matching eigenvalues.        */
int tpt_plan_transforms(tpt_plan plan, int* xform_host /* 2 ints */);
int tpt_plan_rows(tpt_plan plan, int dir, double* a_host, double* b_host, double* c_host);

/* ---- diagnostics -------------------------------------------------------- */
/* Number of CUDA kernels this library has launched since it was loaded
 * (every device, every thread); benchmarks read it before and after a timed
 * region to count the kernels inside it.                                   */
int tpt_kernel_launches(unsigned long long* count);

/* Whether ptr points into device memory of cuda_device (1) or not (0: host,
 * pinned, managed or another GPU's memory, a null pointer, or a device that
 * does not exist).  The transform GEMMs pair two CTAs that share an operand
 * tile by TMA multicast only when every operand plane passes this test on
 * the current device; otherwise they run one CTA per tile.  The paper has no
 * counterpart.  INVALID_ARG for a null on_device or a negative device.      */
int tpt_pointer_on_device(const void* ptr, int cuda_device, int* on_device);

/* Record CUDA events around each stage of tpt_solve on a TPT_PREC_MIXED_*
 * plan and report the summed stage times in tpt_info.ms_stage (filled only
 * when `info` is given; the call then synchronises the stream once per
 * correction).  enable = 0 turns it off.                                    */
int tpt_set_stage_timing(tpt_plan plan, int enable);

/* Change rtol and max_refine of an existing plan (same meaning and limits as
 * in tpt_desc).  Not to be called while a solve on this plan is in flight.  */
int tpt_set_refinement(tpt_plan plan, double rtol, int max_refine);

/* ---- pressure projection ------------------------------------------------- */
/* The projection step of the fractional-step scheme (Sec. 2.1, the
 * pressure-correction equation Eq. poi_ns and the velocity correction after
 * it): with g = gamma_k dt,
 *     L Phi = D u* / g ,    u = u* - g G Phi ,
 * on the staggered grid of the plan.  u (Nx+1, Ny, Nz), v (Nx, Ny+1, Nz) and
 * w (Nx, Ny, Nz+1) are the face-normal velocities on the x-, y- and z-faces
 * (Fortran order; face i of a line lies between cells i-1 and i), updated in
 * place.  (D u)_cell = sum over directions of (u_{i+1} - u_i) / dx_i;
 * (G Phi) on interior face i is (Phi_i - Phi_{i-1}) / dx_{i-1/2}, on a
 * periodic direction also across the shared boundary face (0 and N, which
 * must hold equal values), and zero on wall faces, whose values are left as
 * given (no penetration).  The plan must be the Poisson operator (alpha 0,
 * beta 1) with periodic or Neumann directions; Phi (Nx*Ny*Nz doubles,
 * phi_dev) gets zero volume-weighted mean, and a net wall flux is removed as
 * the compatibility defect (info->compat_defect).  work_dev holds
 * tpt_project_workspace_bytes() bytes.  Errors as tpt_solve, UNSUPPORTED for a
 * Dirichlet direction, INVALID_ARG for other coefficients.                 */
int tpt_project_workspace_bytes(tpt_plan plan, size_t* bytes);
int tpt_project(tpt_plan plan, double* u, double* v, double* w, double gamma_dt, double* phi_dev,
                void* work_dev, void* stream, tpt_info* info);

/* ---- transform tiles ---------------------------------------------------- */
/* Tile autotuner for the transform GEMMs of a TPT_PREC_MIXED_* plan (the
 * forward/inverse eigenbasis projections of Algorithm 1 steps 1, 3, 7, 9):
 * times the four GEMMs of one correction (x forward, y forward, y inverse,
 * x inverse) over the column-tile widths 32, 64, 128, 256 that do not exceed
 * the GEMM's column count rounded up to a power of two, and keeps the fastest
 * per stage for later solves.  work_dev as for tpt_solve (its contents are
 * overwritten); synchronises `stream`.  tiles_out (4 ints, may be NULL)
 * receives the chosen widths.  A float64 plan is left unchanged and reports
 * zeros.  Errors: INVALID_ARG, CUDA, TIMEOUT.                              */
int tpt_plan_autotune(tpt_plan plan, void* work_dev, void* stream, int* tiles_out);

/* Set the four column-tile widths directly (0 = default: the smallest of
 * 32..256 covering the column count), e.g. to reuse a tuned choice on a plan
 * of the same shape.  Each width 0, 32, 64, 128 or 256, else INVALID_ARG.
 * Not to be called while a solve on this plan is in flight.                */
int tpt_plan_set_tiles(tpt_plan plan, const int* tiles);
int tpt_plan_get_tiles(tpt_plan plan, int* tiles_out);

/* Two-CTA operand sharing of the four transform GEMMs (0 none; 1 pairs of
 * m-tiles share the B tile, 2 pairs of n-tiles share the A tile, through
 * TMA multicast in a cluster of two): chosen by tpt_plan_autotune, or set
 * here (each 0, 1 or 2, else INVALID_ARG; a mode that does not apply to a
 * GEMM falls back to one CTA per tile).                                     */
int tpt_plan_set_pairing(tpt_plan plan, const int* pairs);
int tpt_plan_get_pairing(tpt_plan plan, int* pairs_out);

/* Residual kernel of a TPT_PREC_MIXED_* plan (Sec. 4.1 residual in float
 * pairs): 0 automatic (plane tiles staged in shared memory by TMA when Nx is
 * a multiple of 4, else direct loads), 1 direct loads, 2 TMA-staged tiles
 * where Nx allows.  Both compute every point with the same operations in the
 * same order, so R is the same to the bit; only the summation order of the
 * residual norm differs.  For kernel tests and measurements.  INVALID_ARG
 * for another value; a no-op on float64 plans.                              */
int tpt_plan_set_residual_kernel(tpt_plan plan, int variant);

/* Modal Thomas kernel of a TPT_PREC_MIXED_* plan (Sec. 2.2.2 solution step
 * 2.3 / Algorithm 1 step 5 in float32, by the partition method): 0
 * automatic, 1 one modal line per thread (segments of up to 32 rows, 16 per
 * line), 2 two neighbouring lines per thread (segments of up to 16 rows, 32
 * per line; Nz <= 512).  Automatic takes 2 for 192 < Nz <= 512.  The two
 * partition the lines differently, so results agree to float32 rounding,
 * not to the bit.  For kernel tests and measurements.  INVALID_ARG for
 * another value; a no-op on float64 plans.                                 */
int tpt_plan_set_thomas_kernel(tpt_plan plan, int variant);

/* That Thomas step alone, for kernel tests: t2_dev holds the modal right
 * sides f-hat in float32, element (x mode p, y mode q, row k) at
 * q + ldy (p + Nx k) with ldy = Ny rounded up to a multiple of 8 (entries
 * with q >= Ny are padding and are solved as dummy lines); the solution
 * phi-hat is written in the same layout in the plan's operand format:
 * float32 (TPT_PREC_MIXED_TF32), bf16 (TPT_PREC_MIXED_BF16), or bf16 hi in
 * t3_dev and lo in t3_lo_dev (TPT_PREC_MIXED_BF16X3).  A singular plan
 * solves the null line (0, 0) in float64 on its second stream (the
 * compatibility part of that line removed, zero dz-weighted mean).  work_dev
 * is a workspace of tpt_workspace_bytes (its scalars are overwritten).
 * Synchronises `stream`.  Errors: INVALID_ARG (float64 plan, null pointer),
 * CUDA, TIMEOUT.                                                           */
int tpt_mixed_thomas(tpt_plan plan, const float* t2_dev, void* t3_dev, void* t3_lo_dev, void* work_dev,
                     void* stream);

/* ---- batched solves ------------------------------------------------------ */
/* A batch owns `count` plans of possibly different sizes and coefficients on
 * one device (Sec. 2.2: each instance is an independent tensor-product-Thomas
 * solve).  tpt_batch_solve runs every instance with a fixed 1 + max_refine
 * corrections and a final residual (rtol only classifies the result) as one
 * CUDA graph: the instances are spread over `nstreams` capture streams
 * (longest first onto the least-loaded stream; 0 picks min(count, 8)) so
 * that independent instances overlap on the device, and the whole batch is
 * replayed with one graph launch.  The graph is captured on the first call
 * and again whenever a buffer pointer or a plan's coefficients or tiles
 * change; a capturing call runs the batch eagerly first.                   */
typedef struct tpt_batch_s* tpt_batch;

int tpt_batch_create(const tpt_desc* descs, int count, int cuda_device, int nstreams, tpt_batch* out);

/* Device workspace of one tpt_batch_solve (256-byte aligned): per capture
 * stream the largest tpt_workspace_bytes of its instances.                 */
int tpt_batch_workspace_bytes(tpt_batch batch, size_t* bytes);

/* Borrowed handle of instance i (owned by the batch; valid until
 * tpt_batch_destroy).  Changing its coefficients or tiles makes the next
 * tpt_batch_solve recapture.                                                */
int tpt_batch_plan(tpt_batch batch, int i, tpt_plan* out);

/* Autotune the transform tiles of every distinct (size, precision) in the
 * batch once and share the choice among instances of that shape.            */
int tpt_batch_autotune(tpt_batch batch, void* work_dev, void* stream);

/* Solve every instance: f_dev[i] and phi_dev[i] hold instance i's field
 * (phi_dev[i] may equal f_dev[i]; distinct instances must not overlap).
 * work_dev holds tpt_batch_workspace_bytes() bytes.  Asynchronous on
 * `stream` when infos and statuses are both NULL; otherwise the call
 * synchronises `stream` and fills infos[i] (iters, rel_residual,
 * compat_defect; ms_stage zero) and statuses[i] (OK, NOT_CONVERGED against
 * the instance's rtol when rtol > 0, NONFINITE, TIMEOUT).  Returns the
 * first failing status of an instance, else OK; INVALID_ARG, CUDA.        */
int tpt_batch_solve(tpt_batch batch, const double* const* f_dev, double* const* phi_dev, void* work_dev,
                    void* stream, tpt_info* infos, int* statuses);

/* Per-instance reports of the last tpt_batch_solve, after its stream has
 * been synchronised by the caller.  Returns as tpt_batch_solve does.        */
int tpt_batch_infos(tpt_batch batch, tpt_info* infos, int* statuses);

/* Kernels one graph replay launches (0 before the first capture).           */
int tpt_batch_launches(tpt_batch batch, unsigned long long* count);

/* Grouped mode of a batch (the default where it applies): every stage of
 * every correction is one kernel over all instances (one per Thomas segment
 * length and per residual variant), whose CTAs take their units -- GEMM
 * tiles, tiles of modal lines, plane tiles -- from all instances at once
 * through device job tables; an instance that has met its rtol stops and its
 * units are passed over by the later kernels.  A batch of ~100 instances
 * then replays O(10) kernels per correction instead of ~10 per instance.  It
 * applies when every instance is TPT_PREC_MIXED_BF16X3 with rtol > 0, Nx a
 * multiple of 4 and Nz <= 512, and the fields are 16-byte aligned; each
 * instance then runs until it meets rtol or the largest 1 + max_refine of the
 * batch, and has its own region of the workspace (tpt_batch_workspace_bytes
 * reports the mode's size: query it after switching).  grouped = 0 selects
 * the capture streams; UNSUPPORTED when grouped mode does not apply (a solve
 * whose buffers it cannot take also returns UNSUPPORTED and switches the
 * batch back to streams).  The paper's closest analogue is the autotuned
 * decomposition of its GPU runs (Sec. 3, Sec. 4.2.2).                      */
int tpt_batch_set_grouped(tpt_batch batch, int grouped);
int tpt_batch_get_grouped(tpt_batch batch, int* grouped);

int tpt_batch_destroy(tpt_batch batch);

/* ---- shared eigenbases ---------------------------------------------------- */
/* A cache of direction eigenbases on one device.  The eigendecomposition of a
 * direction (Sec. 2.2.1) depends only on its cell widths, centre spacings,
 * boundary pair and transform kind -- not on alpha, beta (Sec. 2.2.2) nor on
 * the other directions -- so plans created through one cache share the
 * eigenbasis and device tables of every direction they have in common, and
 * the O(n^3) host eigendecomposition runs once per distinct direction.
 * cuda_device < 0 makes a host-only cache (for host-only plans).
 * budget_bytes: device memory the cache keeps for tables that no live plan
 * uses (least recently used entries beyond it are freed).                  */
typedef struct tpt_cache_s* tpt_cache;

int tpt_cache_create(int cuda_device, size_t budget_bytes, tpt_cache* out);

/* As tpt_plan_create on the cache's device, sharing eigenbases through the
 * cache.  The plan's own tables are stream-ordered allocations from the
 * cache's memory pool, so creating or destroying it does not synchronise the
 * device; destroy it only after the solves that use it have completed, and
 * before the cache.  Safe to call from several host threads at once.      */
int tpt_plan_create_cached(const tpt_desc* desc, tpt_cache cache, tpt_plan* out);

/* hits / misses of direction lookups, device bytes held, entries (each may
 * be NULL).                                                                 */
int tpt_cache_stats(tpt_cache cache, unsigned long long* hits, unsigned long long* misses,
                    size_t* device_bytes, size_t* entries);
int tpt_cache_destroy(tpt_cache cache);

/* ---- serving ---------------------------------------------------------------- */
/* A request server on one device with continuous batching: requests (a
 * descriptor and a right-hand side in host memory) are queued as they arrive;
 * `setup_threads` host threads build their plans ahead of admission through a
 * shared eigenbasis cache; `slots` host threads each own a CUDA stream and
 * admit the oldest planned request as soon as it fits in the device-memory
 * budget (right-hand side, solution, workspace), copy its right-hand side in,
 * solve it (adaptive refinement when the descriptor's rtol > 0) and copy the
 * solution out.  Requests that arrive while others are on the device are
 * admitted as slots and memory free up, and their work overlaps on the device
 * through the slot streams.  Same-shape batching (config.merge > 1): a slot
 * that admits a request of fewer than 2^24 points also takes the other ready
 * requests of the same grid size and precision (up to `merge` in all, within
 * the budget; only when at least three are ready, smaller groups being
 * served faster one by one) and solves them together as one grouped batch (see
 * tpt_batch_set_grouped; split-bf16 requests with rtol > 0, Nx a multiple of
 * 4, Nz <= 512): one set of grouped kernels for all of them, their buffers and
 * job tables from the server's memory pool.  Each result is that of its own
 * solve to within the refinement target.  cuda_device < 0 is a dry run on the host: plans
 * are host-only and a solve is simulated as a sleep of dry_run_ns_per_point
 * per grid point, which exercises queueing and admission without a GPU.    */
typedef struct tpt_server_s* tpt_server;

typedef struct {
  int cuda_device;
  int slots;                    /* concurrent requests on the device, >= 1          */
  int setup_threads;            /* plan-building threads, >= 1                       */
  size_t memory_budget;         /* device bytes for admitted requests' buffers       */
  size_t cache_budget;          /* device bytes for unused cached eigenbases         */
  double dry_run_ns_per_point;  /* simulated solve time (cuda_device < 0 only)       */
  int merge;                    /* same-shape batching: up to `merge` ready requests
                                   of one shape solved together (0 or 1: each alone) */
} tpt_server_config;

typedef struct {
  int status;                   /* TPT_OK or the solve's / setup's error             */
  tpt_info info;
  double t_submit, t_planned, t_admit, t_done;   /* seconds on the server's clock    */
  size_t device_bytes;          /* bytes charged to the memory budget                */
  int failed_step;              /* 0 none; where a failing request failed:
                                   TPT_STEP_* below                                  */
  int cuda_error;               /* the cudaError_t behind TPT_ERR_CUDA / _OOM, else 0;
                                   tpt_cuda_error_name() names it                    */
  double t_copied, t_solved;    /* when the input copy and the solve had finished
                                   (server clock; 0 if not reached)                  */
  int merged;                   /* requests solved together with this one (1: alone) */
} tpt_result;
#define TPT_STEP_PLAN 1         /* plan creation (host setup, cached tables)        */
#define TPT_STEP_ALLOC 2        /* request buffers from the server's pool            */
#define TPT_STEP_H2D 3          /* right-hand side copy to the device                */
#define TPT_STEP_SOLVE 4        /* tpt_solve                                         */
#define TPT_STEP_D2H 5          /* solution copy to the host                         */
#define TPT_STEP_SYNC 6         /* the slot stream's final synchronisation           */

/* ---- failure-detection tests (no GPU fault involved) --------------------- */
/* Allocation-failure injection: after `after` (>= 0) more device
 * allocations of the library (plan and cache tables, server request
 * buffers) succeed, every later one fails as if the device were out of
 * memory, and the calls that made them return TPT_ERR_OOM (a server result
 * records cudaErrorMemoryAllocation and the step); after < 0 turns the
 * injection off.  Process-wide.  The paper has no counterpart.            */
int tpt_test_fail_allocations(long long after);

/* A 256 x 256 x 64 bf16 transform GEMM on the current device whose TMA
 * producer issues no loads, with `polls` polls for every bounded
 * mbarrier wait (about 0.1 ms for 1024): the waits run out, the kernel frees
 * its tensor memory and returns, and the call reports TPT_ERR_TIMEOUT.  The
 * context stays usable.  work_dev: at least 1 MiB of device scratch.  The
 * paper has no counterpart.                                                */
int tpt_test_gemm_timeout(unsigned polls, void* work_dev, size_t work_bytes, void* stream);

/* Name of a cudaError_t value as reported in tpt_result.cuda_error.        */
const char* tpt_cuda_error_name(int cuda_error);

typedef struct {
  unsigned long long submitted, completed, rejected;
  unsigned long long cache_hits, cache_misses;
  size_t cache_bytes, peak_bytes;
  int peak_inflight;
} tpt_serving_stats;

int tpt_server_create(const tpt_server_config* cfg, tpt_server* out);

/* Queue one solve.  desc (its spacing arrays included) is copied; f_host
 * (Nx*Ny*Nz doubles) must stay valid and phi_host (as many) writable until
 * the request has finished.  Pinned host memory gives full copy bandwidth.
 * ticket receives the request's id.                                        */
int tpt_server_submit(tpt_server s, const tpt_desc* desc, const double* f_host, double* phi_host,
                      unsigned long long* ticket);

/* Build the eigenbases (and their device tables) of desc's x and y
 * directions in the server's cache now, so that later requests with those
 * directions find them: a deployment warms the cache with its mesh library
 * before traffic arrives.  Also grows the server's pool of request buffers
 * (fields and workspaces; plan tables come from a separate pool) to hold
 * `slots` requests of desc's shape (as far as the memory budget allows), so
 * the first ones do not wait for the driver to map memory.
 * Synchronous; safe beside running requests.                               */
int tpt_server_warm(tpt_server s, const tpt_desc* desc);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; on completion
 * fills *result, forgets the ticket and returns TPT_OK (the request's own
 * outcome is result->status); TPT_PENDING on timeout; INVALID_ARG for an
 * unknown ticket.                                                           */
int tpt_server_wait(tpt_server s, unsigned long long ticket, double timeout_s, tpt_result* result);

/* Seconds on the server's steady clock (the clock of tpt_result).           */
int tpt_server_now(tpt_server s, double* t);
int tpt_server_stats(tpt_server s, tpt_serving_stats* out);

/* Finishes every submitted request, then stops the threads.                 */
int tpt_server_destroy(tpt_server s);

/* ---- grid helper -------------------------------------------------------- */
/* Cell widths and centre spacings of an n-cell grid on [0, L] whose faces are
 * x(k/n), k = 0..n, of Eq. (tanh_stretching) (Sec. 4.1); stretch = 0 is the
 * uniform grid.  dxf_out: n doubles; dxc_out: n+1 doubles with the wrap
 * spacing (dx_0 + dx_{n-1})/2 at both ends.                               */
int tpt_grid_tanh(int n, double L, double stretch, double* dxf_out, double* dxc_out);

/* Spacings of the face-centred unknowns of one direction (a velocity
 * component normal to the faces, Sec. 2.1), from the cell-centred spacings:
 * each unknown sits on a face and its control volume spans the two adjacent
 * centres.  Walls (periodic = 0): the n - 1 interior faces are the unknowns,
 * widths dxc[1..n-1], centre spacings dxf[0..n-1] (use TPT_BC_DIRICHLET_NODE,
 * the wall faces being boundary nodes); periodic: the n faces 0..n-1, widths
 * dxc[0..n-1], spacings dxf[n-1], dxf[0..n-2], dxf[n-1] (wrap at both ends).
 * Outputs: *n_out, dxf_out (*n_out values), dxc_out (*n_out + 1 values).    */
int tpt_grid_faces(int n, const double* dxf, const double* dxc, int periodic, int* n_out, double* dxf_out,
                   double* dxc_out);

#ifdef __cplusplus
}
#endif
#endif /* TPT_H */
