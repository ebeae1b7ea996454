// Device memory arenas, the device tables of a diagonalised direction, and
// the cache of shared eigenbases.
//
// The eigendecomposition of a direction (Sec. 2.2.1) depends only on its cell
// widths, centre spacings, boundary pair and transform kind -- not on the
// coefficients alpha, beta (Sec. 2.2.2: Poisson and Helmholtz share
// eigenvectors) nor on the other directions -- so plans with a direction in
// common can share its host eigenbasis and its device tables.  Building one
// costs O(n^3) on the host (the eigenvector accumulation of the QL
// iteration); the cache pays it once per distinct direction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "cache.h"
#include "tpt_internal.h"

namespace tpt {

namespace {
struct PinnedSlots {
  std::mutex mu;
  std::vector<std::pair<double*, double*>> free;   // (host, device)
  std::unordered_map<double*, double*> dev_of;
};
PinnedSlots& pinned_slots() {
  static PinnedSlots* s = new PinnedSlots();   // lives to process exit
  return *s;
}
}  // namespace

double* pinned_slot_acquire(double** dev) {
  PinnedSlots& ps = pinned_slots();
  std::lock_guard<std::mutex> g(ps.mu);
  if (ps.free.empty()) {
    constexpr int kSlots = 256, kDoubles = 16;
    void* blk = nullptr;
    if (cudaHostAlloc(&blk, kSlots * kDoubles * sizeof(double), cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    void* dblk = nullptr;
    if (cudaHostGetDevicePointer(&dblk, blk, 0) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;   // the block stays allocated (never freed), unused
    }
    std::memset(blk, 0, kSlots * kDoubles * sizeof(double));
    for (int i = kSlots - 1; i >= 0; --i)
      ps.free.emplace_back(static_cast<double*>(blk) + i * kDoubles, static_cast<double*>(dblk) + i * kDoubles);
  }
  const auto slot = ps.free.back();
  ps.free.pop_back();
  ps.dev_of[slot.first] = slot.second;
  *dev = slot.second;
  return slot.first;
}

void pinned_slot_release(double* host) {
  if (!host) return;
  PinnedSlots& ps = pinned_slots();
  std::lock_guard<std::mutex> g(ps.mu);
  auto it = ps.dev_of.find(host);
  if (it == ps.dev_of.end()) return;
  ps.free.emplace_back(host, it->second);
  ps.dev_of.erase(it);
}

namespace {

int st_of(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  tpt::note_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}

size_t hash_bytes(const void* p, size_t n, size_t h) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;   // FNV-1a
  return h;
}

}  // namespace

// ----------------------------------------------------------------- DevArena

int DevArena::alloc(size_t n, void** out) {
  void* ptr = nullptr;
  const size_t sz = n ? n : 16;
  if (injected_alloc_failure()) return TPT_ERR_OOM;
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&ptr, sz, pool, stream) : cudaMalloc(&ptr, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_OOM;
  }
  allocs.push_back(ptr);
  bytes += sz;
  *out = ptr;
  return TPT_OK;
}

int DevArena::upload(const void* h, size_t n, void** out) {
  const int st = alloc(n, out);
  if (st != TPT_OK || n == 0) return st;
  return st_of(cudaMemcpyAsync(*out, h, n, cudaMemcpyHostToDevice, stream));
}

void DevArena::release() {
  for (void* a : allocs) {
    if (pool) cudaFreeAsync(a, stream);
    else cudaFree(a);
  }
  cudaGetLastError();
  allocs.clear();
  bytes = 0;
}

// ------------------------------------------------------- direction tables

void fp64_operands(const Eigen1D& e, const std::vector<double>& dxf, int role, std::vector<double>* fwd,
                   std::vector<double>* inv) {
  const int n = static_cast<int>(dxf.size());
  fwd->assign(static_cast<size_t>(n) * n, 0.0);
  inv->assign(static_cast<size_t>(n) * n, 0.0);
  for (int m = 0; m < n; ++m) {        // mode
    for (int i = 0; i < n; ++i) {      // grid point
      const double s = std::sqrt(dxf[i]);
      const double q = e.qt[static_cast<size_t>(m) * n + i];
      const double qinv_mi = q * s;    // Q^{-1}(m, i) = Q~(i, m) sqrt(dx_i)
      const double q_im = q / s;       // Q(i, m) = Q~(i, m) / sqrt(dx_i)
      if (role == 0) {
        (*fwd)[m + static_cast<size_t>(n) * i] = qinv_mi;   // A(m, i), column-major
        (*inv)[i + static_cast<size_t>(n) * m] = q_im;      // A(i, m)
      } else {
        (*fwd)[i + static_cast<size_t>(n) * m] = qinv_mi;   // B(k = i, n = m) = Q^{-1}(m, i)
        (*inv)[m + static_cast<size_t>(n) * i] = q_im;      // B(k = m, n = i) = Q(i, m)
      }
    }
  }
}

int upload_fp64_basis(DevArena& a, const Eigen1D& e, const std::vector<double>& dxf, int role, DevDir* out) {
  std::vector<double> fwd, inv;
  fp64_operands(e, dxf, role, &fwd, &inv);
  void* p = nullptr;
  int st = a.upload(fwd.data(), fwd.size() * sizeof(double), &p);
  if (st != TPT_OK) return st;
  out->fwd = static_cast<double*>(p);
  st = a.upload(inv.data(), inv.size() * sizeof(double), &p);
  if (st != TPT_OK) return st;
  out->inv = static_cast<double*>(p);
  st = a.upload(e.lam.data(), e.lam.size() * sizeof(double), &p);
  if (st != TPT_OK) return st;
  out->lam = static_cast<double*>(p);
  // the host vectors die here: wait for the copies from pageable memory
  return st_of(cudaStreamSynchronize(a.stream));
}

int upload_fft_tables(DevArena& a, int n, const Eigen1D& e, FftTables* t, double** lam) {
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<double> twc(n / 2 > 0 ? n / 2 : 1, 1.0), tws(twc.size(), 0.0), hc(n), hs(n);
  for (int m = 0; m < n / 2; ++m) {
    twc[m] = static_cast<double>(std::cos(2.0L * pi * m / n));
    tws[m] = static_cast<double>(std::sin(2.0L * pi * m / n));
  }
  for (int k = 0; k < n; ++k) {
    hc[k] = static_cast<double>(std::cos(pi * k / (2.0L * n)));
    hs[k] = static_cast<double>(std::sin(pi * k / (2.0L * n)));
  }
  double** dst[5] = {&t->twc, &t->tws, &t->hc, &t->hs, lam};
  const std::vector<double>* src[5] = {&twc, &tws, &hc, &hs, &e.lam};
  for (int i = 0; i < 5; ++i) {
    void* p = nullptr;
    const int st = a.upload(src[i]->data(), src[i]->size() * sizeof(double), &p);
    if (st != TPT_OK) return st;
    *dst[i] = static_cast<double*>(p);
  }
  return st_of(cudaStreamSynchronize(a.stream));
}

double null_fhat(const Dir1D& d, const Eigen1D& e, bool fft) {
  // f-hat of the constant 1 on the null mode: N for the Fourier transforms,
  // sum_i Q~[i, null] sqrt(dx_i) for the eigenbasis
  if (fft) return d.n;
  double g = 0.0;
  for (int i = 0; i < d.n; ++i) g += e.qt[i] * std::sqrt(d.dxf[i]);
  return g;
}

// ------------------------------------------------------------- the cache

BasisCache::BasisCache(int dev, size_t budget) : dev_(dev), budget_(budget) {}

int BasisCache::init() {
  if (dev_ < 0) return TPT_OK;   // host-only: eigenbases without device tables
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev_;
  for (cudaMemPool_t* pl : {&pool_, &buf_pool_}) {
    int st = st_of(cudaMemPoolCreate(pl, &props));
    if (st != TPT_OK) return st;
    uint64_t keep = ~0ULL;   // keep freed memory in the pool: no release to the driver
    st = st_of(cudaMemPoolSetAttribute(*pl, cudaMemPoolAttrReleaseThreshold, &keep));
    if (st != TPT_OK) return st;
    // an allocation on one stream must not reuse a block freed on another
    // stream by waiting for that stream (requests on different slots would
    // then run one after another); it reuses blocks whose free has completed
    // and grows the pool otherwise
    int no = 0;
    st = st_of(cudaMemPoolSetAttribute(*pl, cudaMemPoolReuseAllowInternalDependencies, &no));
    if (st != TPT_OK) return st;
  }
  return st_of(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
}

BasisCache::~BasisCache() {
  if (dev_ >= 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev_);
    for (auto& kv : map_) kv.second->arena.release();
    map_.clear();
    if (stream_) {
      cudaStreamSynchronize(stream_);
      cudaStreamDestroy(stream_);
    }
    if (pool_) cudaMemPoolDestroy(pool_);
    if (buf_pool_) cudaMemPoolDestroy(buf_pool_);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
  }
}

std::shared_ptr<DirEntry> BasisCache::get(const Dir1D& d, int xform, int* status) {
  size_t h = 1469598103934665603ULL;
  const int key_ints[4] = {d.n, d.bc[0], d.bc[1], xform};
  h = hash_bytes(key_ints, sizeof(key_ints), h);
  h = hash_bytes(d.dxf.data(), d.dxf.size() * sizeof(double), h);
  h = hash_bytes(d.dxc.data(), d.dxc.size() * sizeof(double), h);
  auto same = [&](const DirEntry& e) {
    return e.n == d.n && e.bc[0] == d.bc[0] && e.bc[1] == d.bc[1] && e.xform == xform && e.dxf == d.dxf &&
           e.dxc == d.dxc;
  };
  {
    std::lock_guard<std::mutex> g(mu_);
    auto range = map_.equal_range(h);
    for (auto it = range.first; it != range.second; ++it)
      if (same(*it->second)) {
        it->second->stamp = ++clock_;
        ++hits_;
        *status = TPT_OK;
        return it->second;
      }
  }
  // miss: the eigendecomposition runs outside the lock, so distinct
  // directions are built in parallel by concurrent callers
  auto e = std::make_shared<DirEntry>();
  e->n = d.n;
  e->bc[0] = d.bc[0];
  e->bc[1] = d.bc[1];
  e->xform = xform;
  e->dxf = d.dxf;
  e->dxc = d.dxc;
  e->hash = h;
  e->arena.pool = pool_;
  e->arena.stream = stream_;
  const int st = (xform == TPT_XFORM_FFT) ? fft_dir(d, &e->eig, &e->fft_kind) : eigen_dir(d, &e->eig);
  if (st != TPT_OK) {
    *status = st;
    return nullptr;
  }
  e->null_g = null_fhat(d, e->eig, xform == TPT_XFORM_FFT);
  std::lock_guard<std::mutex> g(mu_);
  auto range = map_.equal_range(h);
  for (auto it = range.first; it != range.second; ++it)
    if (same(*it->second)) {   // built concurrently by another caller: keep theirs
      it->second->stamp = ++clock_;
      ++hits_;
      *status = TPT_OK;
      return it->second;
    }
  e->stamp = ++clock_;
  ++misses_;
  map_.emplace(h, e);
  *status = TPT_OK;
  return e;
}

int BasisCache::device_fp64(DirEntry& e, int role, DevDir* out, FftTables* fft) {
  std::lock_guard<std::mutex> g(e.mu);
  if (e.xform == TPT_XFORM_FFT) {
    if (!e.fft_ready) {
      const int st = upload_fft_tables(e.arena, e.n, e.eig, &e.fft, &e.lam);
      if (st != TPT_OK) return st;
      e.fft.kind = e.fft_kind;
      e.fft_ready = true;
    }
    out->fwd = out->inv = nullptr;
    out->lam = e.lam;
    *fft = e.fft;
    return TPT_OK;
  }
  if (!e.fp64_ready[role]) {
    const int st = upload_fp64_basis(e.arena, e.eig, e.dxf, role, &e.fp64[role]);
    if (st != TPT_OK) return st;
    e.fp64_ready[role] = true;
  }
  *out = e.fp64[role];
  return TPT_OK;
}

int entry_mixed_tables(DirEntry& e, int fmt, int dev, void* q[2][2], float** lam_f) {
  std::lock_guard<std::mutex> g(e.mu);
  if (!e.mixed_ready[fmt]) {
    const int st = mixed_pack_basis(e.arena, fmt, e.eig, e.dxf, dev, e.q[fmt], &e.lam_f[fmt]);
    if (st != TPT_OK) return st;
    const cudaError_t ce = cudaStreamSynchronize(e.arena.stream);
    if (ce != cudaSuccess) return st_of(ce);
    e.mixed_ready[fmt] = true;
  }
  for (int r = 0; r < 2; ++r)
    for (int pl = 0; pl < 2; ++pl) q[r][pl] = e.q[fmt][r][pl];
  *lam_f = e.lam_f[fmt];
  return TPT_OK;
}

void BasisCache::trim() {
  std::lock_guard<std::mutex> g(mu_);
  for (;;) {
    size_t total = 0;
    for (auto& kv : map_) total += kv.second->arena.bytes;
    if (total <= budget_) return;
    // least recently used entry that no plan holds
    auto victim = map_.end();
    for (auto it = map_.begin(); it != map_.end(); ++it)
      if (it->second.use_count() == 1 && (victim == map_.end() || it->second->stamp < victim->second->stamp))
        victim = it;
    if (victim == map_.end()) return;
    victim->second->arena.release();
    map_.erase(victim);
    ++evictions_;
  }
}

void BasisCache::stats(unsigned long long* hits, unsigned long long* misses, size_t* bytes, size_t* entries) {
  std::lock_guard<std::mutex> g(mu_);
  if (hits) *hits = hits_;
  if (misses) *misses = misses_;
  size_t total = 0;
  for (auto& kv : map_) total += kv.second->arena.bytes;
  if (bytes) *bytes = total;
  if (entries) *entries = map_.size();
}

}  // namespace tpt
