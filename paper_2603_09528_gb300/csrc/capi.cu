// C ABI of the solver: plan creation (host setup + upload), the solve driver
// (transforms, modal Thomas, residual, iterative refinement) and the single-step
// entry points.  Declarations and contracts: include/tpt.h.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cache.h"
#include "tc.h"
#include "tpt_internal.h"

using tpt::Dir1D;

namespace {

struct DeviceGuard {   // restores the caller's current device
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  tpt::note_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

#define TPT_TRY(expr)                 \
  do {                                \
    int st_ = (expr);                 \
    if (st_ != TPT_OK) return st_;    \
  } while (0)
#define TPT_CUDA(expr) TPT_TRY(cuda_status(expr))

template <typename T>
int upload(tpt_plan_s* p, const std::vector<T>& h, T** d) {
  void* ptr = nullptr;
  TPT_TRY(p->arena.upload(h.data(), h.size() * sizeof(T), &ptr));
  *d = static_cast<T*>(ptr);
  return TPT_OK;
}

void free_plan(tpt_plan_s* p) {
  if (!p) return;
  if (p->dev >= 0) {
    DeviceGuard g(p->dev);
    for (cudaEvent_t e : p->ev)
      if (e) cudaEventDestroy(e);
    if (p->mixed.fork) cudaEventDestroy(p->mixed.fork);
    if (p->mixed.join) cudaEventDestroy(p->mixed.join);
    if (p->mixed.side) cudaStreamDestroy(p->mixed.side);
    p->arena.release();
    if (p->own_stream && p->arena.stream) cudaStreamDestroy(p->arena.stream);
    if (p->h_ring) cudaFreeHost(p->h_ring);
    if (p->solve_exec) cudaGraphExecDestroy(p->solve_exec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->oz_scratch) cudaFree(p->oz_scratch);
    tpt::pinned_slot_release(p->h_scal);
    cudaGetLastError();
  }
  delete p;
}

bool on_device(const tpt_plan_s* p) { return p && p->dev >= 0 && p->d_scal; }

int apply_transform(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                    bool accumulate, void* oz, int* err, cudaStream_t s) {
  if (p->dir[d].excluded()) {   // identity transform: no GEMM along a direction outside the operator
    if (!accumulate) return cuda_status(cudaMemcpyAsync(out, in, tpt::npts(p) * sizeof(double),
                                                        cudaMemcpyDeviceToDevice, s));
    return cuda_status(tpt::add_fp64(static_cast<long long>(tpt::npts(p)), in, out, s));
  }
  if (p->xform[d] == TPT_XFORM_FFT) return cuda_status(tpt::fft_fp64(p, d, inverse, in, out, accumulate, s));
  if (p->ozaki) return cuda_status(tpt::ozaki_transform(p, d, inverse, in, out, accumulate, oz, err, s));
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const double* mat = inverse ? p->ddir[d].inv : p->ddir[d].fwd;
  if (d == 0) {
    return cuda_status(tpt::dgemm_cm(nx, ny * nz, nx, mat, nx, 0, in, nx, 0, out, nx, 0, 1,
                                     accumulate, s));
  }
  const long long slab = static_cast<long long>(nx) * ny;
  return cuda_status(tpt::dgemm_cm(nx, ny, ny, in, nx, slab, mat, ny, 0, out, nx, slab, nz,
                                   accumulate, s));
}

// Workspace layout (float64 path): scalars (256 B) | r | t1 | t2 | fcopy, each
// field region npts doubles, every region 256-byte aligned.  The scalars are
// [0] modal defect of the corrections, [1..3] residual sums, [4] constant
// removed from f, [5..7] sums of f.
constexpr int kRingSlots = 64, kSlot = 16;
size_t region_bytes(const tpt_plan_s* p) {
  return (tpt::npts(p) * sizeof(double) + 255) & ~static_cast<size_t>(255);
}

// One correction solve: out (=|+=) Q_x Q_y (Thomas) Q_y^{-1} Q_x^{-1} rhs.
int inner_fp64(const tpt_plan_s* p, const double* rhs, double* out, bool accumulate, double* t1,
               double* t2, double* defect, void* oz, int* err, cudaStream_t s) {
  TPT_TRY(apply_transform(p, 0, false, rhs, t1, false, oz, err, s));      // step 2.1
  TPT_TRY(apply_transform(p, 1, false, t1, t2, false, oz, err, s));       // step 2.2
  TPT_CUDA(tpt::thomas_fp64(p, t2, t2, t1, defect, s));                   // step 2.3
  TPT_TRY(apply_transform(p, 1, true, t2, t1, false, oz, err, s));        // step 2.4
  TPT_TRY(apply_transform(p, 0, true, t1, out, accumulate, oz, err, s));  // step 2.5
  return TPT_OK;
}

struct InfoCallback {
  tpt_info* info;
  const double* h_scal;   // pinned copy of the workspace scalars
  double npts, vol;
  int iters;
  bool singular;
};

double projected_norm2(double s2, double s1, double sv, double npts, double vol, bool singular) {
  if (!singular) return s2;
  const double c = sv / vol;
  return s2 - 2.0 * c * s1 + npts * c * c;
}

void CUDART_CB fill_info(void* arg) {
  InfoCallback* cb = static_cast<InfoCallback*>(arg);
  const double* h = cb->h_scal;
  const double fn2 = projected_norm2(h[5], h[6], h[7], cb->npts, cb->vol, cb->singular);
  cb->info->iters = cb->iters;
  cb->info->compat_defect = h[4];
  cb->info->rel_residual = (fn2 > 0.0) ? std::sqrt(h[1]) / std::sqrt(fn2) : std::sqrt(h[1]);
  delete cb;
}

// The float64 solve of tpt_solve(); enqueue_only runs 1 + max_refine
// corrections and a final residual with no host synchronisation (capturable
// in a CUDA graph) and leaves the sums in the workspace scalars.
int fp64_solve(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s, tpt_info* info,
               bool enqueue_only) {
  const size_t rb = region_bytes(p);
  char* w = static_cast<char*>(work);
  double* ds = reinterpret_cast<double*>(w);
  w += 256;
  double* r = reinterpret_cast<double*>(w);
  double* t1 = reinterpret_cast<double*>(w + rb);
  double* t2 = reinterpret_cast<double*>(w + 2 * rb);
  double* fcopy = reinterpret_cast<double*>(w + 3 * rb);
  const int corrections = 1 + p->max_refine;
  const bool adaptive = p->rtol > 0.0 && !enqueue_only;
  const double* fu = f;
  if (phi == f && (corrections > 1 || adaptive || info || enqueue_only)) {   // f is needed after phi is written
    TPT_CUDA(cudaMemcpyAsync(fcopy, f, tpt::npts(p) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    fu = fcopy;
  }
  TPT_CUDA(cudaMemsetAsync(ds, 0, 16 * sizeof(double), s));
  TPT_CUDA(tpt::field_sums(p, fu, ds + 5, s));
  void* oz = p->ozaki ? static_cast<void*>(w + 4 * rb) : nullptr;   // Ozaki scratch after fcopy
  int* oz_err = reinterpret_cast<int*>(ds + 10);
  TPT_TRY(inner_fp64(p, fu, phi, false, t1, t2, ds + 4, oz, oz_err, s));
  int iters = 1;
  const double np = static_cast<double>(tpt::npts(p));
  double fn2 = -1.0, rel = -1.0;
  double h[kSlot] = {0.0};
  auto read_residual = [&]() -> int {
    TPT_CUDA(cudaMemcpyAsync(h, ds, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TPT_CUDA(cudaStreamSynchronize(s));
    if (reinterpret_cast<const int*>(h + 10)[0]) return TPT_ERR_TIMEOUT;   // a bounded GEMM wait ran out
    fn2 = projected_norm2(h[5], h[6], h[7], np, p->vol, p->singular);
    if (!std::isfinite(h[1]) || !std::isfinite(fn2)) return TPT_ERR_NONFINITE;
    rel = (fn2 > 0.0) ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
    return TPT_OK;
  };
  int status = TPT_OK;
  bool converged = false;
  for (;;) {
    const bool need_residual = (iters < corrections) || adaptive || info || enqueue_only;
    if (!need_residual) break;
    TPT_CUDA(cudaMemsetAsync(ds + 1, 0, 3 * sizeof(double), s));
    TPT_CUDA(tpt::residual_fp64(p, fu, phi, r, ds + 1, p->singular ? ds + 4 : nullptr, s));
    if (adaptive) {
      TPT_TRY(read_residual());
      if (rel <= p->rtol) {
        converged = true;
        break;
      }
    }
    if (iters >= corrections) break;
    TPT_TRY(inner_fp64(p, r, phi, true, t1, t2, ds, oz, oz_err, s));
    ++iters;
  }
  // the canonical gauge: phi shifted to zero volume-weighted mean in physical
  // space (the null line's gauge fixes it only up to the eigenvectors'
  // rounding, ~1e-12 of phi on 512-point stretched grids); the final residual
  // above is unaffected, a constant being in the operator's null space
  if (p->singular) TPT_CUDA(tpt::remove_weighted_mean(p, phi, r, rb, ds + 9, s));
  if (adaptive && !converged) status = TPT_ERR_NOT_CONVERGED;
  if (info && !enqueue_only) {
    if (adaptive) {
      info->iters = iters;
      info->rel_residual = rel;
      info->compat_defect = h[4];
      for (float& t : info->ms_stage) t = 0.0f;
    } else {
      std::memset(info, 0, sizeof(*info));
      if (!p->h_ring) {   // pinned slots for asynchronous reports, made on first use
        const size_t ring_bytes = static_cast<size_t>(kRingSlots) * kSlot * sizeof(double);
        TPT_CUDA(cudaMallocHost(reinterpret_cast<void**>(&p->h_ring), ring_bytes));
        std::memset(p->h_ring, 0, ring_bytes);
      }
      double* slot = p->h_ring + static_cast<size_t>(p->ring_next) * kSlot;
      p->ring_next = (p->ring_next + 1) % kRingSlots;
      TPT_CUDA(cudaMemcpyAsync(slot, ds, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
      InfoCallback* cb = new (std::nothrow) InfoCallback{info, slot, np, p->vol, iters, p->singular};
      if (!cb) return TPT_ERR_OOM;
      TPT_CUDA(cudaLaunchHostFunc(s, fill_info, cb));
    }
  }
  return status;
}

// Plan creation: host setup (1D operators, eigenbases), then the device
// tables.  With a cache the eigenbases of x and y (and their device tables)
// are shared with every plan that has the same direction, and the plan's own
// tables are stream-ordered allocations from the cache's pool, so creating and
// destroying plans does not synchronise the device.
int create_plan_impl(const tpt_desc* desc, int cuda_device, tpt::BasisCache* cache, tpt_plan* out) {
  if (!out) return TPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return TPT_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (desc->n[d] < 1 || !desc->dxf[d] || !desc->dxc[d]) return TPT_ERR_INVALID_ARG;
  if (!std::isfinite(desc->alpha) || !std::isfinite(desc->beta)) return TPT_ERR_INVALID_ARG;
  if (desc->alpha == 0.0 && desc->beta == 0.0) return TPT_ERR_INVALID_ARG;
  if (desc->max_refine < 0 || desc->max_refine > 1000) return TPT_ERR_INVALID_ARG;
  if (desc->precision < TPT_PREC_FP64 || desc->precision > TPT_PREC_FP64_OZAKI)
    return TPT_ERR_INVALID_ARG;
  if (!std::isfinite(desc->rtol) || desc->rtol < 0.0) return TPT_ERR_INVALID_ARG;
  for (int d = 0; d < 2; ++d)
    if (desc->xform[d] < TPT_XFORM_AUTO || desc->xform[d] > TPT_XFORM_FFT) return TPT_ERR_INVALID_ARG;
  // lines of a plane and planes of a field are indexed with 32-bit integers
  if (static_cast<long long>(desc->n[0]) * desc->n[1] >= (1LL << 31) ||
      static_cast<long long>(desc->n[1]) * desc->n[2] >= (1LL << 31) ||
      static_cast<long long>(desc->n[0]) * desc->n[2] >= (1LL << 31))
    return TPT_ERR_UNSUPPORTED;

  tpt_plan_s* p = new (std::nothrow) tpt_plan_s();
  if (!p) return TPT_ERR_OOM;
  p->dev = cuda_device;
  auto fail = [&](int st) {
    free_plan(p);
    return st;
  };
  for (int d = 0; d < 3; ++d) {
    p->n[d] = desc->n[d];
    int st = tpt::build_dir(desc->n[d], desc->dxf[d], desc->dxc[d], desc->bc[d], &p->dir[d]);
    if (st != TPT_OK) return fail(st);
  }
  if (p->dir[2].periodic || p->dir[2].excluded()) return fail(TPT_ERR_UNSUPPORTED);
  if ((p->dir[0].excluded() || p->dir[1].excluded()) && desc->alpha == 0.0) return fail(TPT_ERR_INVALID_ARG);
  for (int d = 0; d < 2; ++d) {
    // Fourier-based transforms of uniform power-of-two directions: float64
    // kernels on the float64 and Ozaki paths, float32 kernels inside the
    // mixed-precision corrections (16 to 4096 points)
    const bool fp64 = desc->precision == TPT_PREC_FP64 || desc->precision == TPT_PREC_FP64_OZAKI;
    const bool ok = tpt::fft_supported(p->dir[d]) && (fp64 || (p->dir[d].n >= 16 && p->dir[d].n <= 4096));
    if (desc->xform[d] == TPT_XFORM_FFT && !ok) return fail(TPT_ERR_UNSUPPORTED);
    p->xform[d] = (desc->xform[d] == TPT_XFORM_FFT || (desc->xform[d] == TPT_XFORM_AUTO && ok && fp64))
                      ? TPT_XFORM_FFT
                      : TPT_XFORM_GEMM;
  }
  p->alpha = desc->alpha;
  p->beta = desc->beta;
  // an Ozaki plan is a float64 plan whose GEMM transforms run on the tensor cores
  p->precision = desc->precision == TPT_PREC_FP64_OZAKI ? TPT_PREC_FP64 : desc->precision;
  p->rtol = desc->rtol;
  p->max_refine = desc->max_refine;
  for (int d = 0; d < 2; ++d) {
    const bool fft = p->xform[d] == TPT_XFORM_FFT;
    if (cache) {
      int st = TPT_OK;
      p->basis[d] = cache->get(p->dir[d], p->xform[d], &st);
      if (!p->basis[d]) return fail(st);
      p->eig[d].lam = p->basis[d]->eig.lam;   // the eigenvectors stay in the shared entry
      p->eig[d].null_mode = p->basis[d]->eig.null_mode;
      p->fft[d].kind = p->basis[d]->fft_kind;
      p->null_g[d] = p->basis[d]->null_g;
    } else {
      int st = fft ? tpt::fft_dir(p->dir[d], &p->eig[d], &p->fft[d].kind) : tpt::eigen_dir(p->dir[d], &p->eig[d]);
      if (st != TPT_OK) return fail(st);
      p->null_g[d] = tpt::null_fhat(p->dir[d], p->eig[d], fft);
    }
  }
  p->singular = (p->alpha == 0.0) && p->dir[0].has_null() && p->dir[1].has_null() &&
                p->dir[2].has_null();
  p->null_i = p->eig[0].null_mode;
  p->null_j = p->eig[1].null_mode;
  p->vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    double L = 0.0;
    for (double w : p->dir[d].dxf) L += w;
    p->vol *= L;
  }
  if (cuda_device < 0) {   // host-only plan: setup tables for inspection, no device state
    *out = p;
    return TPT_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return fail(TPT_ERR_CUDA);
  }
  if (cuda_device >= ndev) return fail(TPT_ERR_INVALID_ARG);
  DeviceGuard guard(cuda_device);
  if (cache) {
    p->arena.pool = cache->pool();
    p->arena.stream = cache->stream();
  } else {
    if (cudaStreamCreateWithFlags(&p->arena.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(TPT_ERR_CUDA);
    }
    p->own_stream = true;
  }
  for (int d = 0; d < 2; ++d) {
    int st = TPT_OK;
    if (cache) {
      st = cache->device_fp64(*p->basis[d], d, &p->ddir[d], &p->fft[d]);
    } else if (p->xform[d] == TPT_XFORM_FFT) {
      st = tpt::upload_fft_tables(p->arena, p->n[d], p->eig[d], &p->fft[d], &p->ddir[d].lam);
    } else {
      st = tpt::upload_fp64_basis(p->arena, p->eig[d], p->dir[d].dxf, d, &p->ddir[d]);
    }
    if (st != TPT_OK) return fail(st);
  }
  for (int d = 0; d < 3; ++d) {
    const Dir1D& dd = p->dir[d];
    std::vector<double> rows(3 * static_cast<size_t>(dd.n));
    std::copy(dd.a.begin(), dd.a.end(), rows.begin());
    std::copy(dd.b.begin(), dd.b.end(), rows.begin() + dd.n);
    std::copy(dd.c.begin(), dd.c.end(), rows.begin() + 2 * dd.n);
    std::vector<double> ixf(dd.n), ixc(dd.n + 1);
    for (int i = 0; i < dd.n; ++i) ixf[i] = 1.0 / dd.dxf[i];
    for (int i = 0; i <= dd.n; ++i) ixc[i] = 1.0 / dd.dxc[i];
    int st = upload(p, rows, &p->d_rows[d]);
    if (st == TPT_OK) st = upload(p, dd.dxf, &p->d_dxf[d]);
    if (st == TPT_OK) st = upload(p, ixf, &p->d_inv_dxf[d]);
    if (st == TPT_OK) st = upload(p, ixc, &p->d_inv_dxc[d]);
    if (st != TPT_OK) return fail(st);
  }
  std::vector<double> scal(16, 0.0);
  int st = upload(p, scal, &p->d_scal);
  if (st != TPT_OK) return fail(st);
  if (p->precision != TPT_PREC_FP64) {
    st = tpt::mixed_setup(p);
    if (st != TPT_OK) return fail(st);
  }
  if (cudaStreamSynchronize(p->arena.stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(TPT_ERR_CUDA);
  }
  if (desc->precision == TPT_PREC_FP64_OZAKI && p->dev >= 0) {   // slices of the transform matrices
    st = tpt::ozaki_setup(p);
    if (st != TPT_OK) return fail(st);
    if (cudaStreamSynchronize(p->arena.stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(TPT_ERR_CUDA);
    }
  }
  *out = p;
  return TPT_OK;
}

}  // namespace

namespace tpt {
size_t npts(const tpt_plan_s* p) {
  return static_cast<size_t>(p->n[0]) * p->n[1] * p->n[2];
}
namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launch(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
namespace {
thread_local cudaError_t t_last_cuda_error = cudaSuccess;
}
void note_cuda_error(cudaError_t e) {
  if (e != cudaSuccess) t_last_cuda_error = e;
}
cudaError_t last_cuda_error() { return t_last_cuda_error; }
namespace {
std::atomic<long long> g_alloc_budget{-1};   // < 0: no injection
}
bool injected_alloc_failure() {
  long long b = g_alloc_budget.load(std::memory_order_relaxed);
  while (b > 0 && !g_alloc_budget.compare_exchange_weak(b, b - 1, std::memory_order_relaxed)) {
  }
  if (b == 0) {
    note_cuda_error(cudaErrorMemoryAllocation);
    return true;
  }
  return false;
}
void clear_cuda_error() { t_last_cuda_error = cudaSuccess; }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void forget_launches(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

int create_plan(const tpt_desc* desc, int cuda_device, BasisCache* cache, tpt_plan* out) {
  return create_plan_impl(desc, cuda_device, cache, out);
}

int solve_enqueue(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s) {
  if (p->precision != TPT_PREC_FP64) return mixed_enqueue(p, f, phi, work, s);
  return fp64_solve(p, f, phi, work, s, nullptr, true);
}

int solve_info(const tpt_plan_s* p, const double* h, tpt_info* info) {
  if (p->precision != TPT_PREC_FP64) return mixed_info(p, h, info);
  const double np = static_cast<double>(npts(p));
  const double fn2 = projected_norm2(h[5], h[6], h[7], np, p->vol, p->singular);
  const double rel = (fn2 > 0.0) ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = 1 + p->max_refine;
    info->rel_residual = rel;
    info->compat_defect = h[4];
  }
  if (!std::isfinite(rel)) return TPT_ERR_NONFINITE;
  if (p->rtol > 0.0 && !(rel <= p->rtol)) return TPT_ERR_NOT_CONVERGED;
  return TPT_OK;
}
}  // namespace tpt

extern "C" {

const char* tpt_status_string(int status) {
  switch (status) {
    case TPT_OK: return "ok";
    case TPT_ERR_INVALID_ARG: return "invalid argument";
    case TPT_ERR_UNSUPPORTED: return "unsupported configuration";
    case TPT_ERR_OOM: return "device out of memory";
    case TPT_ERR_CUDA: return "CUDA error";
    case TPT_ERR_NOT_CONVERGED: return "refinement did not converge";
    case TPT_ERR_TIMEOUT: return "device wait timed out";
    case TPT_ERR_NONFINITE: return "non-finite value in right-hand side or residual";
    case TPT_ERR_NUMERICAL: return "numerical failure in setup";
    case TPT_PENDING: return "request not finished";
    default: return "unknown status";
  }
}

int tpt_kernel_launches(unsigned long long* count) {
  if (!count) return TPT_ERR_INVALID_ARG;
  *count = tpt::g_launches.load(std::memory_order_relaxed);
  return TPT_OK;
}

int tpt_test_fail_allocations(long long after) {
  tpt::g_alloc_budget.store(after < 0 ? -1 : after, std::memory_order_relaxed);
  return TPT_OK;
}

int tpt_test_gemm_timeout(unsigned polls, void* work_dev, size_t work_bytes, void* stream) {
  if (!work_dev || polls == 0 || work_bytes < (1u << 20)) return TPT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status(cudaGetLastError());
  return tpt::gemm_timeout_test(polls, work_dev, dev, static_cast<cudaStream_t>(stream));
}

const char* tpt_cuda_error_name(int cuda_error) {
  return cuda_error == 0 ? "cudaSuccess" : cudaGetErrorName(static_cast<cudaError_t>(cuda_error));
}

int tpt_pointer_on_device(const void* ptr, int cuda_device, int* on_device) {
  if (!on_device || cuda_device < 0) return TPT_ERR_INVALID_ARG;
  *on_device = 0;
  if (!ptr) return TPT_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device >= ndev) {
    cudaGetLastError();
    return TPT_OK;   // no such device: nothing is its memory
  }
  DeviceGuard g(cuda_device);
  *on_device = tpt::tc::own_device_memory(ptr) ? 1 : 0;
  return TPT_OK;
}

int tpt_grid_tanh(int n, double L, double stretch, double* dxf_out, double* dxc_out) {
  return tpt::grid_tanh(n, L, stretch, dxf_out, dxc_out);
}

int tpt_grid_faces(int n, const double* dxf, const double* dxc, int periodic, int* n_out, double* dxf_out,
                   double* dxc_out) {
  return tpt::grid_faces(n, dxf, dxc, periodic, n_out, dxf_out, dxc_out);
}

int tpt_plan_create(const tpt_desc* desc, int cuda_device, tpt_plan* out) {
  return create_plan_impl(desc, cuda_device, nullptr, out);
}

int tpt_cache_create(int cuda_device, size_t budget_bytes, tpt_cache* out) {
  if (!out) return TPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (cuda_device >= 0) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
      cudaGetLastError();
      return TPT_ERR_CUDA;
    }
    if (cuda_device >= ndev) return TPT_ERR_INVALID_ARG;
  }
  tpt_cache c = new (std::nothrow) tpt_cache_s(cuda_device, budget_bytes);
  if (!c) return TPT_ERR_OOM;
  int st = TPT_OK;
  {
    DeviceGuard guard(cuda_device >= 0 ? cuda_device : 0);
    st = c->impl.init();
  }
  if (st != TPT_OK) {
    delete c;
    return st;
  }
  *out = c;
  return TPT_OK;
}

int tpt_plan_create_cached(const tpt_desc* desc, tpt_cache cache, tpt_plan* out) {
  if (!cache) return TPT_ERR_INVALID_ARG;
  const int st = create_plan_impl(desc, cache->impl.device(), &cache->impl, out);
  cache->impl.trim();
  return st;
}

int tpt_cache_stats(tpt_cache cache, unsigned long long* hits, unsigned long long* misses, size_t* device_bytes,
                    size_t* entries) {
  if (!cache) return TPT_ERR_INVALID_ARG;
  cache->impl.stats(hits, misses, device_bytes, entries);
  return TPT_OK;
}

int tpt_cache_destroy(tpt_cache cache) {
  if (!cache) return TPT_ERR_INVALID_ARG;
  delete cache;
  return TPT_OK;
}

int tpt_plan_destroy(tpt_plan p) {
  if (!p) return TPT_ERR_INVALID_ARG;
  free_plan(p);
  return TPT_OK;
}

int tpt_set_coefficients(tpt_plan p, double alpha, double beta) {
  if (!p || !std::isfinite(alpha) || !std::isfinite(beta) || (alpha == 0.0 && beta == 0.0))
    return TPT_ERR_INVALID_ARG;
  p->alpha = alpha;
  p->beta = beta;
  ++p->generation;
  p->singular = (alpha == 0.0) && p->dir[0].has_null() && p->dir[1].has_null() &&
                p->dir[2].has_null();
  if (p->precision != TPT_PREC_FP64 && p->dev >= 0 && p->mixed.dfrows[0]) {
    DeviceGuard guard(p->dev);
    return tpt::mixed_set_beta(p);
  }
  return TPT_OK;
}

int tpt_set_refinement(tpt_plan p, double rtol, int max_refine) {
  if (!p || !std::isfinite(rtol) || rtol < 0.0 || max_refine < 0 || max_refine > 1000)
    return TPT_ERR_INVALID_ARG;
  p->rtol = rtol;
  p->max_refine = max_refine;
  ++p->generation;
  return TPT_OK;
}

int tpt_plan_autotune(tpt_plan p, void* work, void* stream, int* tiles_out) {
  if (!on_device(p) || !work || reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  const int st = tpt::autotune_gemms(p, work, static_cast<cudaStream_t>(stream));
  if (tiles_out) tpt_plan_get_tiles(p, tiles_out);
  return st;
}

int tpt_plan_set_tiles(tpt_plan p, const int* tiles) {
  if (!p || !tiles) return TPT_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (tiles[i] != 0 && tiles[i] != 32 && tiles[i] != 64 && tiles[i] != 128 && tiles[i] != 256)
      return TPT_ERR_INVALID_ARG;
  if (p->precision == TPT_PREC_FP64) return TPT_OK;
  for (int i = 0; i < 4; ++i) {
    p->mixed.gemm_bn[i] = tiles[i];
    p->mixed.gemm_ctas[i] = 0;
  }
  ++p->generation;
  return TPT_OK;
}

int tpt_plan_set_pairing(tpt_plan p, const int* pairs) {
  if (!p || !pairs) return TPT_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (pairs[i] < 0 || pairs[i] > 2) return TPT_ERR_INVALID_ARG;
  if (p->precision == TPT_PREC_FP64) return TPT_OK;
  for (int i = 0; i < 4; ++i) p->mixed.gemm_pair[i] = pairs[i];
  ++p->generation;
  return TPT_OK;
}

int tpt_plan_set_residual_kernel(tpt_plan p, int variant) {
  if (!p || variant < 0 || variant > 2) return TPT_ERR_INVALID_ARG;
  if (p->precision == TPT_PREC_FP64) return TPT_OK;
  p->mixed.res_kernel = variant;
  ++p->generation;
  return TPT_OK;
}

int tpt_plan_set_thomas_kernel(tpt_plan p, int variant) {
  if (!p || variant < 0 || variant > 2) return TPT_ERR_INVALID_ARG;
  if (p->precision == TPT_PREC_FP64) return TPT_OK;
  p->mixed.thomas_kernel = variant;
  ++p->generation;
  return TPT_OK;
}

int tpt_mixed_thomas(tpt_plan p, const float* t2_dev, void* t3_dev, void* t3_lo_dev, void* work_dev,
                     void* stream) {
  if (!p) return TPT_ERR_INVALID_ARG;
  DeviceGuard g(p->dev);
  return tpt::mixed_thomas_test(p, t2_dev, t3_dev, t3_lo_dev, work_dev, static_cast<cudaStream_t>(stream));
}

int tpt_plan_get_pairing(tpt_plan p, int* pairs_out) {
  if (!p || !pairs_out) return TPT_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) pairs_out[i] = (p->precision == TPT_PREC_FP64) ? 0 : p->mixed.gemm_pair[i];
  return TPT_OK;
}

int tpt_plan_get_tiles(tpt_plan p, int* tiles_out) {
  if (!p || !tiles_out) return TPT_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) tiles_out[i] = (p->precision == TPT_PREC_FP64) ? 0 : p->mixed.gemm_bn[i];
  return TPT_OK;
}

int tpt_workspace_bytes(tpt_plan p, size_t* bytes) {
  if (!p || !bytes) return TPT_ERR_INVALID_ARG;
  *bytes = (p->precision == TPT_PREC_FP64)
               ? 256 + 4 * region_bytes(p) + (p->ozaki ? tpt::ozaki_scratch_bytes(p) : 0)
               : tpt::mixed_workspace_bytes(p);
  return TPT_OK;
}

int tpt_solve(tpt_plan p, const double* f, double* phi, void* work, void* stream, tpt_info* info) {
  if (!on_device(p) || !f || !phi || !work) return TPT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->precision != TPT_PREC_FP64) return tpt::mixed_solve(p, f, phi, work, s, info);
  return fp64_solve(p, f, phi, work, s, info, false);
}

int tpt_solve_host(tpt_plan p, const double* f_host, double* phi_host, double* f_dev,
                   double* phi_dev, void* work, void* stream, tpt_info* info) {
  if (!on_device(p) || !f_host || !phi_host || !f_dev || !phi_dev) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = tpt::npts(p) * sizeof(double);
  TPT_CUDA(cudaMemcpyAsync(f_dev, f_host, bytes, cudaMemcpyHostToDevice, s));
  int st = tpt_solve(p, f_dev, phi_dev, work, stream, info);
  if (st != TPT_OK && st != TPT_ERR_NOT_CONVERGED) return st;
  TPT_CUDA(cudaMemcpyAsync(phi_host, phi_dev, bytes, cudaMemcpyDeviceToHost, s));
  TPT_CUDA(cudaStreamSynchronize(s));
  return st;
}

int tpt_transform(tpt_plan p, int dir, int inverse, const double* in, double* out, void* stream) {
  if (!on_device(p) || !in || !out || in == out || (dir != 0 && dir != 1)) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  if (p->ozaki && !p->oz_scratch)   // this entry point's own scratch, kept by the plan
    TPT_CUDA(cudaMalloc(&p->oz_scratch, tpt::ozaki_scratch_bytes(p)));
  return apply_transform(p, dir, inverse != 0, in, out, false, p->oz_scratch, nullptr,
                         static_cast<cudaStream_t>(stream));
}

int tpt_thomas(tpt_plan p, const double* fhat, double* phihat, double* scratch, void* stream) {
  if (!on_device(p) || !fhat || !phihat || !scratch) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  return cuda_status(tpt::thomas_fp64(p, fhat, phihat, scratch, p->d_scal,
                                      static_cast<cudaStream_t>(stream)));
}

int tpt_residual(tpt_plan p, const double* f, const double* phi, double* r, double* sums,
                 void* stream) {
  if (!on_device(p) || !f || !phi || !r) return TPT_ERR_INVALID_ARG;
  DeviceGuard guard(p->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the single-step residual uses f as given (no compatibility shift)
  return cuda_status(tpt::residual_fp64(p, f, phi, r, sums, nullptr, s, true));
}

int tpt_tc_gemm(int precision, int M, int N, int K, const double* A, const double* B, double* D,
                void* work, void* stream, int tile, int pair) {
  if (tile != 0 && tile != 32 && tile != 64 && tile != 128 && tile != 256) return TPT_ERR_INVALID_ARG;
  if (pair < 0 || pair > 2) return TPT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_CUDA;
  }
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  return tpt::tc_gemm_test(precision, M, N, K, A, B, D, work, dev, static_cast<cudaStream_t>(stream), tile, pair);
}

int tpt_tc_gemm_out(int precision, int M, int N, int K, const double* A, const double* B, int out_kind, int rm,
                    long long sm, long long sn, void* out0, void* out1, void* work, void* stream, int tile,
                    int tma_out, int pair) {
  if (tile != 0 && tile != 32 && tile != 64 && tile != 128 && tile != 256) return TPT_ERR_INVALID_ARG;
  if (pair < 0 || pair > 2) return TPT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_CUDA;
  }
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  return tpt::tc_gemm_out_test(precision, M, N, K, A, B, out_kind, rm, sm, sn, out0, out1, work, dev,
                               static_cast<cudaStream_t>(stream), tile, tma_out != 0, pair);
}

int tpt_set_stage_timing(tpt_plan p, int enable) {
  if (!p) return TPT_ERR_INVALID_ARG;
  p->stage_timing = enable ? 1 : 0;
  return TPT_OK;
}

int tpt_plan_transforms(tpt_plan p, int* xform) {
  if (!p || !xform) return TPT_ERR_INVALID_ARG;
  xform[0] = p->xform[0];
  xform[1] = p->xform[1];
  return TPT_OK;
}

int tpt_plan_eigenvalues(tpt_plan p, int dir, double* lam) {
  if (!p || !lam || (dir != 0 && dir != 1)) return TPT_ERR_INVALID_ARG;
  std::copy(p->eig[dir].lam.begin(), p->eig[dir].lam.end(), lam);
  return TPT_OK;
}

int tpt_plan_rows(tpt_plan p, int dir, double* a, double* b, double* c) {
  if (!p || !a || !b || !c || dir < 0 || dir > 2) return TPT_ERR_INVALID_ARG;
  const Dir1D& d = p->dir[dir];
  std::copy(d.a.begin(), d.a.end(), a);
  std::copy(d.b.begin(), d.b.end(), b);
  std::copy(d.c.begin(), d.c.end(), c);
  return TPT_OK;
}

}  // extern "C"
