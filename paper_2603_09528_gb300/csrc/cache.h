// Shared eigenbases of 1D directions and their device tables (cache.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "tpt_internal.h"

namespace tpt {

// Eigenbasis of one direction, keyed by (n, boundary pair, transform kind,
// cell widths, centre spacings), with device tables built on first use.
struct DirEntry {
  int n = 0, bc[2] = {0, 0}, xform = 0;
  std::vector<double> dxf, dxc;
  size_t hash = 0;
  Eigen1D eig;
  int fft_kind = 0;
  double null_g = 0.0;
  uint64_t stamp = 0;                    // last use, for eviction
  std::mutex mu;                         // guards the device tables below
  DevArena arena;
  bool fp64_ready[2] = {false, false};   // float64 GEMM operands per role (x, y)
  DevDir fp64[2];
  bool fft_ready = false;
  FftTables fft;
  double* lam = nullptr;
  bool mixed_ready[3] = {false, false, false};
  void* q[3][2][2] = {};                 // [format][forward | inverse][plane]
  float* lam_f[3] = {nullptr, nullptr, nullptr};
};

class BasisCache {
 public:
  BasisCache(int dev, size_t budget);
  ~BasisCache();
  int init();
  int device() const { return dev_; }
  cudaMemPool_t pool() const { return pool_; }
  // Pool of the request buffers (fields and workspaces): kept apart from the
  // tables so that a small table never splits a freed field-sized block and
  // same-shape requests reuse whole blocks.
  cudaMemPool_t buffer_pool() const { return buf_pool_; }
  cudaStream_t stream() const { return stream_; }
  // The entry of direction d with transform kind xform; computed on a miss.
  std::shared_ptr<DirEntry> get(const Dir1D& d, int xform, int* status);
  int device_fp64(DirEntry& e, int role, DevDir* out, FftTables* fft);
  // Evict least recently used entries no plan holds while over the budget.
  void trim();
  void stats(unsigned long long* hits, unsigned long long* misses, size_t* bytes, size_t* entries);

 private:
  int dev_;
  size_t budget_;
  cudaMemPool_t pool_ = nullptr;
  cudaMemPool_t buf_pool_ = nullptr;
  cudaStream_t stream_ = nullptr;
  std::mutex mu_;
  std::unordered_multimap<size_t, std::shared_ptr<DirEntry>> map_;
  uint64_t clock_ = 0;
  unsigned long long hits_ = 0, misses_ = 0, evictions_ = 0;
};

// Plan creation through an optional cache (capi.cu).
int create_plan(const tpt_desc* desc, int cuda_device, BasisCache* cache, tpt_plan* out);

// Tensor-core operand tables of a cached direction in format fmt, built on
// first use (mixed.cu calls this from the plan's mixed setup).
int entry_mixed_tables(DirEntry& e, int fmt, int dev, void* q[2][2], float** lam_f);

// Shared table builders (cache.cu, mixed.cu).
int upload_fp64_basis(DevArena& a, const Eigen1D& e, const std::vector<double>& dxf, int role, DevDir* out);
int upload_fft_tables(DevArena& a, int n, const Eigen1D& e, FftTables* t, double** lam);
double null_fhat(const Dir1D& d, const Eigen1D& e, bool fft);
// Tensor-core operand planes of one direction in format fmt: q[0] = Q^{-1}
// rows (forward), q[1] = Q rows (inverse), row stride n rounded up to 8.
int mixed_pack_basis(DevArena& a, int fmt, const Eigen1D& e, const std::vector<double>& dxf, int dev,
                     void* q[2][2], float** lam_f);

}  // namespace tpt

struct tpt_cache_s {
  tpt_cache_s(int dev, size_t budget) : impl(dev, budget) {}
  tpt::BasisCache impl;
};
