// Batched solves of independent instances of uneven size (Sec. 2.2: each
// instance is its own tensor-product-Thomas solve, so a batch has no data
// dependence between instances).  The batch is recorded once as a CUDA graph:
// the instances are spread over several capture streams (longest first onto
// the least-loaded stream) whose chains become independent graph branches,
// so small instances that fill only part of the GPU overlap with others, and
// one graph launch replays the whole batch.  Declarations: include/tpt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "tpt_internal.h"

struct tpt_batch_s {
  int dev = 0;
  int count = 0;
  std::vector<tpt_plan> plans;
  std::vector<std::vector<int>> lanes;   // capture stream -> instances in issue order
  std::vector<size_t> lane_off;          // capture stream -> workspace offset
  size_t ws_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;         // stream the graph is captured on
  double* d_scal = nullptr;              // count x 16: each instance's final sums
  double* h_scal = nullptr;              // pinned copy, written at the end of a solve
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;          // buffers the graph was captured with
  std::vector<unsigned> gens;            // plan generations at capture
  unsigned long long launches = 0;       // kernels per replay
  bool solved = false;
  // grouped mode: one kernel per stage over every instance (when the plans
  // qualify; see tpt::group_create), instead of per-instance kernels spread
  // over the capture streams
  tpt::GroupSolve* group = nullptr;
  bool grouped = false;
  size_t ws_streams = 0;                 // workspace of the stream mode
};

namespace {

constexpr int kScal = 16;

struct DeviceScope {   // restores the caller's current device
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  tpt::note_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

#define BT_TRY(expr)               \
  do {                             \
    const int st_ = (expr);        \
    if (st_ != TPT_OK) return st_; \
  } while (0)
#define BT_CUDA(expr) BT_TRY(cuda_st(expr))

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

void release(tpt_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  tpt::group_destroy(b->group);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->d_scal) cudaFree(b->d_scal);
  if (b->h_scal) cudaFreeHost(b->h_scal);
  for (tpt_plan p : b->plans)
    if (p) tpt_plan_destroy(p);
  delete b;
}

// Work estimate of one instance for the stream assignment: the transform
// GEMMs dominate, 2 n_x n_y n_z (n_x + n_y) per correction.
double cost_of(const tpt_plan_s* p) {
  const double nx = p->n[0], ny = p->n[1], nz = p->n[2];
  return (1.0 + p->max_refine) * nx * ny * nz * (nx + ny + 16.0);
}

// Fork onto the capture streams, solve every instance, join, and copy the
// per-instance sums to the pinned host array (grouped mode: the grouped
// launches on s).
int enqueue(tpt_batch b, const double* const* f, double* const* phi, char* work, cudaStream_t s) {
  if (b->grouped) {
    BT_TRY(tpt::group_enqueue(b->group, b->d_scal, s));
    BT_CUDA(cudaMemcpyAsync(b->h_scal, b->d_scal, static_cast<size_t>(b->count) * kScal * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    return TPT_OK;
  }
  BT_CUDA(cudaEventRecord(b->fork, s));
  for (cudaStream_t ls : b->streams) BT_CUDA(cudaStreamWaitEvent(ls, b->fork, 0));
  for (size_t k = 0; k < b->lanes.size(); ++k) {
    char* w = work + b->lane_off[k];
    for (int i : b->lanes[k]) {
      BT_TRY(tpt::solve_enqueue(b->plans[i], f[i], phi[i], w, b->streams[k]));
      BT_CUDA(cudaMemcpyAsync(b->d_scal + static_cast<size_t>(i) * kScal, w, kScal * sizeof(double),
                              cudaMemcpyDeviceToDevice, b->streams[k]));
    }
  }
  for (size_t k = 0; k < b->streams.size(); ++k) {
    BT_CUDA(cudaEventRecord(b->joins[k], b->streams[k]));
    BT_CUDA(cudaStreamWaitEvent(s, b->joins[k], 0));
  }
  BT_CUDA(cudaMemcpyAsync(b->h_scal, b->d_scal, static_cast<size_t>(b->count) * kScal * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  return TPT_OK;
}

// Records the batch into a graph on the origin stream and instantiates it.
int capture(tpt_batch b, const double* const* f, double* const* phi, char* work) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const unsigned long long before = tpt::launch_count();
  BT_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
  const int st = enqueue(b, f, phi, work, b->origin);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
  const unsigned long long recorded = tpt::launch_count() - before;
  tpt::forget_launches(recorded);   // recorded, not run
  if (st != TPT_OK || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != TPT_OK ? st : TPT_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    b->exec = nullptr;
    return cuda_st(ie);
  }
  b->launches = recorded;
  return TPT_OK;
}

bool same_key(const tpt_batch b, const std::vector<const void*>& key) {
  if (!b->exec || key != b->key) return false;
  for (int i = 0; i < b->count; ++i)
    if (b->gens[i] != b->plans[i]->generation) return false;
  return true;
}

}  // namespace

extern "C" {

int tpt_batch_create(const tpt_desc* descs, int count, int cuda_device, int nstreams, tpt_batch* out) {
  if (!descs || count <= 0 || cuda_device < 0 || nstreams < 0 || !out) return TPT_ERR_INVALID_ARG;
  *out = nullptr;
  tpt_batch b = new (std::nothrow) tpt_batch_s;
  if (!b) return TPT_ERR_OOM;
  b->dev = cuda_device;
  b->count = count;
  b->plans.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    const int st = tpt_plan_create(&descs[i], cuda_device, &b->plans[i]);
    if (st != TPT_OK) {
      release(b);
      return st;
    }
  }
  DeviceScope scope(cuda_device);
  const int lanes = std::min(count, nstreams > 0 ? nstreams : 8);
  // longest processing time first onto the least-loaded lane
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return cost_of(b->plans[a]) > cost_of(b->plans[c]); });
  b->lanes.assign(lanes, {});
  std::vector<double> load(lanes, 0.0);
  for (int i : order) {
    const int k = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
    b->lanes[k].push_back(i);
    load[k] += cost_of(b->plans[i]);
  }
  b->lane_off.assign(lanes, 0);
  for (int k = 0; k < lanes; ++k) {
    size_t need = 256;
    for (int i : b->lanes[k]) {
      size_t w = 0;
      tpt_workspace_bytes(b->plans[i], &w);
      need = std::max(need, align256(w));
    }
    b->lane_off[k] = b->ws_bytes;
    b->ws_bytes += need;
  }
  int st = TPT_OK;
  b->streams.assign(lanes, nullptr);
  b->joins.assign(lanes, nullptr);
  for (int k = 0; k < lanes && st == TPT_OK; ++k) {
    st = cuda_st(cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking));
    if (st == TPT_OK) st = cuda_st(cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming));
  }
  if (st == TPT_OK) st = cuda_st(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  if (st == TPT_OK) st = cuda_st(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
  const size_t sb = static_cast<size_t>(count) * kScal * sizeof(double);
  if (st == TPT_OK) st = cuda_st(cudaMalloc(reinterpret_cast<void**>(&b->d_scal), sb));
  if (st == TPT_OK) st = cuda_st(cudaMallocHost(reinterpret_cast<void**>(&b->h_scal), sb));
  if (st != TPT_OK) {
    release(b);
    return st;
  }
  std::memset(b->h_scal, 0, sb);
  b->ws_streams = b->ws_bytes;
  b->group = tpt::group_create(b->plans.data(), count);
  if (b->group) {
    b->grouped = true;
    b->ws_bytes = tpt::group_workspace_bytes(b->group);
  }
  *out = b;
  return TPT_OK;
}

int tpt_batch_set_grouped(tpt_batch b, int grouped) {
  if (!b || grouped < 0 || grouped > 1) return TPT_ERR_INVALID_ARG;
  if (grouped && !b->group) {
    // the plans' refinement settings may have changed since creation
    b->group = tpt::group_create(b->plans.data(), b->count);
    if (!b->group) return TPT_ERR_UNSUPPORTED;
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->key.clear();
  b->grouped = grouped != 0;
  b->ws_bytes = b->grouped ? tpt::group_workspace_bytes(b->group) : b->ws_streams;
  return TPT_OK;
}

int tpt_batch_get_grouped(tpt_batch b, int* grouped) {
  if (!b || !grouped) return TPT_ERR_INVALID_ARG;
  *grouped = b->grouped ? 1 : 0;
  return TPT_OK;
}

int tpt_batch_workspace_bytes(tpt_batch b, size_t* bytes) {
  if (!b || !bytes) return TPT_ERR_INVALID_ARG;
  *bytes = b->ws_bytes;
  return TPT_OK;
}

int tpt_batch_plan(tpt_batch b, int i, tpt_plan* out) {
  if (!b || !out || i < 0 || i >= b->count) return TPT_ERR_INVALID_ARG;
  *out = b->plans[i];
  return TPT_OK;
}

int tpt_batch_autotune(tpt_batch b, void* work, void* stream) {
  if (!b || !work || reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  std::vector<int> done;   // instances whose shape is tuned
  for (int i = 0; i < b->count; ++i) {
    tpt_plan p = b->plans[i];
    if (p->precision == TPT_PREC_FP64) continue;
    int tiles[4] = {0, 0, 0, 0}, pairs[4] = {0, 0, 0, 0};
    bool found = false;
    for (int j : done) {
      const tpt_plan q = b->plans[j];
      if (q->precision == p->precision && q->n[0] == p->n[0] && q->n[1] == p->n[1] && q->n[2] == p->n[2]) {
        tpt_plan_get_tiles(q, tiles);
        tpt_plan_get_pairing(q, pairs);
        found = true;
        break;
      }
    }
    if (found) {
      BT_TRY(tpt_plan_set_tiles(p, tiles));
      BT_TRY(tpt_plan_set_pairing(p, pairs));
      continue;
    }
    BT_TRY(tpt_plan_autotune(p, work, stream, nullptr));   // the batch workspace holds any one plan's
    done.push_back(i);
  }
  return TPT_OK;
}

int tpt_batch_infos(tpt_batch b, tpt_info* infos, int* statuses) {
  if (!b) return TPT_ERR_INVALID_ARG;
  if (!b->solved) return TPT_ERR_INVALID_ARG;
  int first = TPT_OK;
  for (int i = 0; i < b->count; ++i) {
    const int st = tpt::solve_info(b->plans[i], b->h_scal + static_cast<size_t>(i) * kScal,
                                   infos ? &infos[i] : nullptr);
    if (statuses) statuses[i] = st;
    if (first == TPT_OK) first = st;
  }
  return first;
}

int tpt_batch_solve(tpt_batch b, const double* const* f, double* const* phi, void* work, void* stream,
                    tpt_info* infos, int* statuses) {
  if (!b || !f || !phi || !work || reinterpret_cast<uintptr_t>(work) % 256 != 0) return TPT_ERR_INVALID_ARG;
  std::vector<const void*> key;
  key.reserve(2 * b->count + 1);
  for (int i = 0; i < b->count; ++i) {
    if (!f[i] || !phi[i]) return TPT_ERR_INVALID_ARG;
    key.push_back(f[i]);
    key.push_back(phi[i]);
  }
  key.push_back(work);
  DeviceScope scope(b->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(work);
  b->solved = false;
  if (b->grouped) {
    const int st = tpt::group_prepare(b->group, f, phi, work, s);   // tables for these buffers
    if (st == TPT_ERR_UNSUPPORTED) {
      BT_TRY(tpt_batch_set_grouped(b, 0));   // buffers the grouped kernels cannot take
      return TPT_ERR_UNSUPPORTED;
    }
    BT_TRY(st);
  }
  if (same_key(b, key)) {
    BT_CUDA(cudaGraphLaunch(b->exec, s));
    tpt::note_launch(b->launches);
  } else {
    // the eager run is this call's solve; the capture serves the next calls
    BT_TRY(enqueue(b, f, phi, w, s));
    BT_TRY(capture(b, f, phi, w));
    b->key = key;
    b->gens.resize(b->count);
    for (int i = 0; i < b->count; ++i) b->gens[i] = b->plans[i]->generation;
  }
  b->solved = true;
  if (!infos && !statuses) return TPT_OK;
  BT_CUDA(cudaStreamSynchronize(s));
  return tpt_batch_infos(b, infos, statuses);
}

int tpt_batch_launches(tpt_batch b, unsigned long long* count) {
  if (!b || !count) return TPT_ERR_INVALID_ARG;
  *count = b->launches;
  return TPT_OK;
}

int tpt_batch_destroy(tpt_batch b) {
  if (!b) return TPT_ERR_INVALID_ARG;
  DeviceScope scope(b->dev);
  release(b);
  return TPT_OK;
}

}  // extern "C"
