// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/tpt.h"

namespace tpt {

// ----------------------------------------------------------------- host setup
// One direction's 1D operator rows (Eq. tridiagonal-coefficients with boundary
// rows) and, for diagonalised directions, its eigenbasis.
struct Dir1D {
  int n = 0;
  int bc[2] = {TPT_BC_NEUMANN, TPT_BC_NEUMANN};
  bool periodic = false;
  bool uniform = false;           // all cell widths and centre spacings equal
  std::vector<double> dxf, dxc;   // n, n+1
  std::vector<double> a, b, c;    // rows: a_i phi_{i-1} + b_i phi_i + c_i phi_{i+1}
  bool has_null() const {
    return periodic || (bc[0] == TPT_BC_NEUMANN && bc[1] == TPT_BC_NEUMANN);
  }
  bool excluded() const { return bc[0] == TPT_BC_NONE; }   // not in the operator
};

// Eigenbasis of one diagonalised direction: T = Q Lambda Q^{-1} with
// Q = D^{-1/2} Q~ and Q^{-1} = Q~^T D^{1/2}.  Modes are sorted by decreasing
// eigenvalue, so a null mode (lambda = 0) is mode 0.
struct Eigen1D {
  std::vector<double> lam;        // n
  std::vector<double> qt;         // Q~, column-major n x n (column p = mode p)
  int null_mode = -1;
};

int build_dir(int n, const double* dxf, const double* dxc, const int bc[2], Dir1D* out);
// Fourier-based transform of a uniform direction: true when N is a power of
// two, the spacing uniform and the boundary pair periodic or Neumann-Neumann.
bool fft_supported(const Dir1D& d);
// Eigenvalues in the mode order of the Fourier-based transform (real DFT for
// periodic, DCT-II for Neumann), as Rayleigh quotients of the exact
// trigonometric vectors with the float64 rows; kind: 0 real DFT, 1 DCT.
int fft_dir(const Dir1D& d, Eigen1D* out, int* kind);
int eigen_dir(const Dir1D& d, Eigen1D* out);
int grid_tanh(int n, double L, double stretch, double* dxf, double* dxc);
int grid_faces(int n, const double* dxf, const double* dxc, int periodic, int* n_out, double* dxf_out,
               double* dxc_out);

// ----------------------------------------------------------------- device memory
// Device tables of a plan or of a shared eigenbasis.  With a pool the tables
// are stream-ordered allocations on `stream` (no device-wide synchronisation
// when they are created or freed, so plans can come and go while other solves
// run); otherwise plain cudaMalloc.  Uploads are asynchronous copies on
// `stream`; the owner synchronises `stream` before the tables are used.
struct DevArena {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  int alloc(size_t n, void** out);
  int upload(const void* h, size_t n, void** out);
  void release();
};

struct DirEntry;      // shared eigenbasis of one direction (cache.cu)
class BasisCache;

// ----------------------------------------------------------------- device plan
// operand formats of the low-precision path: bf16 hi/lo pair, bf16, float32
enum { kFmtSplit = 0, kFmtBF16 = 1, kFmtF32 = 2 };

// Device tables of the mixed-precision path.
struct MixedTables {
  int fmt = kFmtSplit;
  int ldx = 0, ldy = 0;            // Nx, Ny rounded up to 8 (operand row strides)
  void* q[2][2][2] = {};           // [x|y][forward Q^{-1} | inverse Q][plane], row-major
  float* lam_f[2] = {nullptr, nullptr};
  float* zrows_f = nullptr;        // a|b|c of z in float32
  float* dfrows[3] = {nullptr, nullptr, nullptr};   // beta*(a|c|w) as float pairs: ah|al|ch|cl|wh|wl
  int has_w[3] = {0, 0, 0};        // direction has a nonzero diagonal remainder (Dirichlet wall)
  double rows_beta = 0.0;          // beta the tables were scaled with
  float* dfgeom[3] = {nullptr, nullptr, nullptr};   // cell widths as float pairs: h|l
  double* null_cp = nullptr;       // factorisation of T_z (beta = 1) for the null line:
  double* null_invm = nullptr;     //   c'_k and 1/m_k, k < Nz - 1
  cudaStream_t side = nullptr;     // second stream for the null line, with fork/join events
  cudaEvent_t fork = nullptr, join = nullptr;
  // transform GEMM tiles per stage (x forward, y forward, y inverse, x
  // inverse): column tile width (0 = default) and persistent-CTA cap (0 = all)
  int gemm_bn[4] = {0, 0, 0, 0};
  int gemm_ctas[4] = {0, 0, 0, 0};
  int gemm_pair[4] = {0, 0, 0, 0};
  int res_kernel = 0;               // residual: 0 automatic, 1 direct loads, 2 TMA-staged tiles
  int thomas_kernel = 0;            // modal Thomas: 0 automatic, 1 one line per thread, 2 two lines
  // Fourier-transformed directions (x, y): float32 tables cos, sin of
  // 2 pi m / N and cos, sin of pi k / 2N, and the transform kind
  const float* fft_tw[2][4] = {};
  int fft_kind[2] = {0, 0};
};

struct FftTables {    // device tables of a Fourier-transformed direction
  int kind = 0;          // 0 real DFT (periodic), 1 DCT-II/III (Neumann)
  double* twc = nullptr; // cos, sin of 2 pi m / N, m < N/2
  double* tws = nullptr;
  double* hc = nullptr;  // cos, sin of pi k / 2N, k < N (DCT pre/post rotation)
  double* hs = nullptr;
};

struct DevDir {       // device tables of a diagonalised direction (float64)
  double* fwd = nullptr;  // forward transform operand (layout set by the GEMM role)
  double* inv = nullptr;  // inverse transform operand
  double* lam = nullptr;  // eigenvalues in mode order
};

}  // namespace tpt

struct tpt_plan_s {
  int dev = 0;
  int n[3] = {0, 0, 0};
  int xform[2] = {TPT_XFORM_GEMM, TPT_XFORM_GEMM};
  double alpha = 0.0, beta = 1.0;
  int precision = TPT_PREC_FP64;
  double rtol = 0.0;
  int max_refine = 1;
  std::atomic<int> last_iters{0};   // corrections the last adaptive mixed solve used (0: none yet)
  // The adaptive mixed solve as one CUDA graph, captured on the second call with
  // the same (f, phi, work, planned corrections, generation) and replayed after;
  // taken by one caller at a time (graph_busy).
  cudaGraphExec_t solve_exec = nullptr;
  const void* gkey[3] = {nullptr, nullptr, nullptr};
  const void* gprev[3] = {nullptr, nullptr, nullptr};
  int gkey_planned = 0, gprev_planned = 0;
  unsigned gkey_gen = 0, gprev_gen = 0;
  unsigned long long graph_launches = 0;   // kernels in the captured solve
  cudaStream_t cap_stream = nullptr;
  double* h_scal = nullptr;                // pinned, mapped slot for the workspace scalars
  double* d_hscal = nullptr;               // its device address
  std::atomic<bool> graph_busy{false};
  // The null line runs on the plan's second stream between a fork and a join
  // event shared by all solves of the plan: solves enqueued from several host
  // threads take turns for that sequence, so no solve waits on another's
  // event; a graph capture holds it throughout, since the second stream is
  // part of the capture until it ends.
  std::recursive_mutex side_mu;
  bool singular = false;
  int null_i = 0, null_j = 0;     // mode indices of the null line when singular
  tpt::Dir1D dir[3];
  tpt::Eigen1D eig[2];
  tpt::DevDir ddir[2];
  tpt::FftTables fft[2];
  double null_g[2] = {1.0, 1.0};  // f-hat of a constant 1 on the null mode, per direction
  double* d_rows[3] = {nullptr, nullptr, nullptr};  // a|b|c per direction, 3n doubles
  double* d_dxf[3] = {nullptr, nullptr, nullptr};
  double* d_inv_dxf[3] = {nullptr, nullptr, nullptr};   // 1 / cell widths (projection)
  double* d_inv_dxc[3] = {nullptr, nullptr, nullptr};   // 1 / centre spacings, n + 1 each
  double* d_scal = nullptr;       // device scalars of the single-step entry points
  double* h_ring = nullptr;       // pinned host slots for asynchronous info reports
  int ring_next = 0;
  double vol = 1.0;               // domain volume Lx Ly Lz
  tpt::MixedTables mixed;
  // float64 transforms by the Ozaki scheme (TPT_PREC_FP64_OZAKI; ozaki.cu):
  // bf16 slices of the four transform matrices (x forward, x inverse, y
  // forward, y inverse) and the padded contraction lengths of x and y
  bool ozaki = false;
  void* oz_tab[4] = {nullptr, nullptr, nullptr, nullptr};
  int oz_kp[2] = {0, 0};
  void* oz_scratch = nullptr;      // scratch of the single-step transform entry point
  int stage_timing = 0;           // record per-stage CUDA events in tpt_solve
  cudaEvent_t ev[12] = {};        // stage boundaries (created on first use)
  unsigned generation = 0;        // bumped when coefficients or tiles change
  tpt::DevArena arena;            // every device table owned by the plan
  bool own_stream = false;        // arena.stream was created for this plan
  std::shared_ptr<tpt::DirEntry> basis[2];   // shared eigenbases of x and y (cached plans)
};

namespace tpt {

size_t npts(const tpt_plan_s* p);

// Process-wide pool of 16-double host slots in pinned, device-mapped memory,
// for scalars a kernel writes straight into host memory (no copy engine, so
// they do not queue behind large host transfers of other streams).  Blocks
// are never returned to the driver (freeing pinned memory synchronises the
// device).  `dev` receives the slot's device address; nullptr on failure.
double* pinned_slot_acquire(double** dev);
void pinned_slot_release(double* host);

// The last CUDA error this thread turned into a TPT_ERR_* status (cudaSuccess:
// none since the last clear), so that a caller that gets TPT_ERR_CUDA or
// TPT_ERR_OOM can say which CUDA error it was.
void note_cuda_error(cudaError_t e);
cudaError_t last_cuda_error();
void clear_cuda_error();

// Failure-detection tests: true when an armed allocation-failure injection
// makes this device allocation fail (tpt_test_fail_allocations); the caller
// then returns TPT_ERR_OOM exactly as for a real failed allocation.
bool injected_alloc_failure();

// Count of kernels this library has launched (all devices, all threads).
void note_launch(unsigned long long k = 1);
unsigned long long launch_count();
void forget_launches(unsigned long long k);   // undo counts of captured (not run) launches

// ----------------------------------------------------------------- kernels
// Batched column-major float64 GEMM: C_b = A_b B_b (+ C_b when accumulate),
// A_b = A + b*sA (M x K, lda), B_b = B + b*sB (K x N, ldb), C_b (M x N, ldc).
cudaError_t dgemm_cm(int M, int N, int K, const double* A, int lda, long long sA,
                     const double* B, int ldb, long long sB, double* C, int ldc, long long sC,
                     int batch, bool accumulate, cudaStream_t s);

// `defect` (device, may be NULL) receives the physical constant removed from
// the right-hand side of a singular problem.
// Fourier-based transform along x (d = 0) or y (d = 1) of a float64 field in
// the natural layout (fft.cu); out (+)= result.
cudaError_t fft_fp64(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                     bool accumulate, cudaStream_t s);

// Float32 Fourier-based transform of a uniform direction inside a mixed-
// precision correction (fft.cu): nlines contiguous input rows (line l at
// in + l * ldi, operand format in_fmt: split bf16 planes in0/in1, bf16 in0,
// or float32 in0), written in tc output mode out_mode as contiguous rows
// (L1 == 0: line l at l * ldo) or transposed (L1 > 0: element t of line
// a + L1 * b at b * ldo * N + t * ldo + a); kOutDF updates the float pair
// (out0, out1) when accumulate is set and overwrites it otherwise.  tw: the
// float32 tables cos, sin of 2 pi m / N (m < N/2) and cos, sin of pi k / 2N
// (k < N).  Kernels return at entry when *stop (device, may be NULL) is set.
struct FftMixedArgs {
  int kind = 0;                 // 0 real DFT, 1 DCT-II / DCT-III
  bool inverse = false;
  int N = 0;
  long long nlines = 0;
  const void* in0 = nullptr;
  const void* in1 = nullptr;
  int in_fmt = kFmtSplit;
  long long ldi = 0;
  void* out0 = nullptr;
  void* out1 = nullptr;
  int out_mode = 0;
  long long ldo = 0, L1 = 0;
  int accumulate = 0;
  const float* tw[4] = {nullptr, nullptr, nullptr, nullptr};
  const int* stop = nullptr;
};
cudaError_t fft_mixed(const FftMixedArgs& a, cudaStream_t s);

cudaError_t thomas_fp64(const tpt_plan_s* p, const double* fhat, double* phihat, double* scratch,
                        double* defect, cudaStream_t s);

// out += in over n values
cudaError_t add_fp64(long long n, const double* in, double* out, cudaStream_t s);

// sums[0..2] += (sum f^2, sum f, sum vol*f) over the field
cudaError_t field_sums(const tpt_plan_s* p, const double* f, double* sums, cudaStream_t s);

// phi -= its volume-weighted mean (the canonical gauge of a singular
// problem, reading R4), summed exactly to a few ulps; scratch (16-byte
// aligned) holds the block partial sums, *mean (device) receives the mean.
cudaError_t remove_weighted_mean(const tpt_plan_s* p, double* phi, void* scratch, size_t scratch_bytes,
                                 double* mean, cudaStream_t s);

// r = (f - fshift) - (alpha I + beta L) phi; fshift (device scalar) may be NULL.
// sums (may be NULL): [0] += sum r^2, and with all_sums [1] += sum r, [2] +=
// sum vol*r.
cudaError_t residual_fp64(const tpt_plan_s* p, const double* f, const double* phi, double* r,
                          double* sums, const double* fshift, cudaStream_t s, bool all_sums = false);

// mixed-precision path (mixed.cu)
int mixed_setup(tpt_plan_s* p);
int mixed_set_beta(tpt_plan_s* p);   // rescale the residual tables after a coefficient change
size_t mixed_workspace_bytes(const tpt_plan_s* p);
int mixed_solve(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s,
                tpt_info* info);
// The modal Thomas step of a mixed plan on its own (kernel tests): T2 float32
// in the (q, p, k) layout with rows of ldy, T3 planes in the operand format.
int mixed_thomas_test(tpt_plan_s* p, const float* t2, void* t3_0, void* t3_1, void* work, cudaStream_t s);
// A transform GEMM whose producer issues no loads, with `polls` polls per
// bounded wait: TPT_ERR_TIMEOUT when the waits ran out and said so.
int gemm_timeout_test(unsigned polls, void* work, int dev, cudaStream_t s);
int tc_gemm_test(int precision, int M, int N, int K, const double* A, const double* B, double* D,
                 void* work, int dev, cudaStream_t s, int tile = 0, int pair = 0);
int tc_gemm_out_test(int precision, int M, int N, int K, const double* A, const double* B, int out_kind,
                     int rm, long long sm, long long sn, void* out0, void* out1, void* work, int dev,
                     cudaStream_t s, int tile, int tma_out, int pair);

// Capturable solves: 1 + max_refine corrections and a final residual, no host
// synchronisation; the residual sums are left in the first 16 doubles of the
// workspace.  *_info turns a host copy of those 16 doubles into a report and a
// status (TIMEOUT, NONFINITE, NOT_CONVERGED against rtol when rtol > 0).
int mixed_enqueue(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s);
int mixed_info(const tpt_plan_s* p, const double* h, tpt_info* info);
int solve_enqueue(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s);
int solve_info(const tpt_plan_s* p, const double* h, tpt_info* info);
// Grouped batch solve (mixed.cu): one kernel per stage over every instance.
// group_create returns null unless every plan qualifies (split bf16, rtol > 0,
// Nx a multiple of 4, Nz <= 512, one device).  group_prepare builds the
// device job tables for the buffers (synchronising s first; a no-op when
// they are unchanged), instance i using work + its offset; group_enqueue then issues
// the launches on s (capturable) and gathers the 16 scalars of instance i
// into d_scal[16 i ..].
struct GroupSolve;
bool group_eligible(const tpt_plan_s* p);
GroupSolve* group_create(tpt_plan_s* const* plans, int n);
// Device memory for the job tables from the caller (at least
// group_table_bytes, 256-byte aligned, kept by the caller), so that a
// grouped solve allocates nothing itself.
size_t group_table_bytes(const GroupSolve* g);
void group_set_memory(GroupSolve* g, void* mem, size_t bytes);
void group_destroy(GroupSolve* g);
size_t group_workspace_bytes(const GroupSolve* g);
unsigned long long group_kernels(const GroupSolve* g);
int group_prepare(GroupSolve* g, const double* const* f, double* const* phi, void* work, cudaStream_t s);
int group_enqueue(GroupSolve* g, double* d_scal, cudaStream_t s);
// The same solve decided on the host: the corrections the instances are
// expected to need, then one at a time while any instance is short of its
// rtol (reading the 16 scalars of every instance back into h_scal, host
// memory of 16 n doubles, after each step); synchronises s.
int group_solve_adaptive(GroupSolve* g, double* d_scal, double* h_scal, cudaStream_t s);

// Ozaki-scheme transforms (ozaki.cu): tables built at plan creation (the
// float64 transform matrices must be on the device), scratch of one transform,
// and the transform itself: out (+)= the float64-accurate transform of in.
bool ozaki_supported(const tpt_plan_s* p);
int ozaki_setup(tpt_plan_s* p);
size_t ozaki_scratch_bytes(const tpt_plan_s* p);
cudaError_t ozaki_transform(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                            bool accumulate, void* scratch, int* err, cudaStream_t s);

// Times the transform GEMMs of a mixed plan over the candidate tiles and keeps
// the fastest per stage (gemm_tune.cu).
int autotune_gemms(tpt_plan_s* p, void* work, cudaStream_t s);

}  // namespace tpt
