// Mixed-precision solve: low-precision correction solves on the tensor cores
// with float64-accurate iterative refinement.
//
// Each correction applies the paper's procedure (Sec. 2.2.2, solution steps
// 2.1-2.5) to the current residual with the transforms on tcgen05 (bf16, split
// bf16 or tf32 operands, float32 accumulation; gemm_tc.cu), a float32 Thomas
// sweep (float64 on the singular null line), and accumulates the correction
// into phi held as an unevaluated float pair (hi + lo, ~48 significant bits).
// The residual r = f - (alpha I + beta L) phi is evaluated in float-pair
// arithmetic with the 7-point stencil of the float64 rows, which keeps it
// accurate to ~1e-13 of f while running on the float32 pipe (GB300's float64
// rate is ~1/55 of its float32 rate).
//
// Intermediate layouts (every GEMM operand K-major, every store coalesced):
//   R  (i, j, k)  rows (j,k) of ldx   -- residual, x-forward input
//   T1 (j, p, k)  rows (p,k) of ldy   -- x-forward output, y-forward input
//   T2 (q, p, k)  rows (p,k) of ldy   -- y-forward output, Thomas in/out (T3)
//   T4 (p, j, k)  rows (j,k) of ldx   -- y-inverse output, x-inverse input
// where p, q index x and y modes and ldx, ldy are Nx, Ny rounded up to 8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc.h"
#include "tpt_internal.h"

namespace tpt {
namespace {

// ------------------------------------------------------------ float pairs
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, {-y.hi, -y.lo}); }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_from_double(double v) {
  const float h = static_cast<float>(v);
  return {h, static_cast<float>(v - static_cast<double>(h))};
}

// ------------------------------------------------------ operand element I/O
template <int FMT>
struct Elem;
template <>
struct Elem<kFmtSplit> {
  static __device__ __forceinline__ float load(const void* p0, const void* p1, long long i) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(p0)[i]) +
           __bfloat162float(static_cast<const __nv_bfloat16*>(p1)[i]);
  }
  static __device__ __forceinline__ void store(void* p0, void* p1, long long i, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(p0)[i] = h;
    static_cast<__nv_bfloat16*>(p1)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
};
template <>
struct Elem<kFmtBF16> {
  static __device__ __forceinline__ float load(const void* p0, const void*, long long i) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(p0)[i]);
  }
  static __device__ __forceinline__ void store(void* p0, void*, long long i, float v) {
    static_cast<__nv_bfloat16*>(p0)[i] = __float2bfloat16_rn(v);
  }
};
template <>
struct Elem<kFmtF32> {
  static __device__ __forceinline__ float load(const void* p0, const void*, long long i) {
    return static_cast<const float*>(p0)[i];
  }
  static __device__ __forceinline__ void store(void* p0, void*, long long i, float v) {
    static_cast<float*>(p0)[i] = v;
  }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// f (float64, (Nx,Ny,Nz)) -> f as float pair, R = f in operand format, and the
// sums (sum f^2, sum f, sum vol*f) into sums[0..2].
template <int FMT>
__global__ void __launch_bounds__(256)
prepare_kernel(int nx, int ny, int nz, int ldx, const double* __restrict__ f, float* __restrict__ fh,
               float* __restrict__ fl, void* r0, void* r1, const double* __restrict__ dxf,
               const double* __restrict__ dyf, const double* __restrict__ dzf, double* sums) {
  const long long n = static_cast<long long>(nx) * ny * nz;
  double s2 = 0.0, s1 = 0.0, sv = 0.0;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < n;
       o += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(o % nx);
    const long long line = o / nx;
    const int j = static_cast<int>(line % ny), k = static_cast<int>(line / ny);
    const double v = f[o];
    const df d = df_from_double(v);
    fh[o] = d.hi;
    fl[o] = d.lo;
    Elem<FMT>::store(r0, r1, i + static_cast<long long>(ldx) * line, d.hi + d.lo);
    s2 = fma(v, v, s2);
    s1 += v;
    sv = fma(dxf[i] * dyf[j] * dzf[k], v, sv);
  }
  s2 = warp_sum_d(s2);
  s1 = warp_sum_d(s1);
  sv = warp_sum_d(sv);
  if (threadIdx.x % 32 == 0) {
    atomicAdd(&sums[0], s2);
    atomicAdd(&sums[1], s1);
    atomicAdd(&sums[2], sv);
  }
}

// Thomas sweep on T2 (q, p, k), rows of ldy: one thread per (q, p) line with
// q fastest.  float32 recurrence with c' in `scratch`; the singular null line
// (q, p) = (0, 0) is solved in float64 with the compatibility projection and
// the zero-mean gauge of the float64 path.
template <int FMT>
__global__ void __launch_bounds__(128)
thomas_mixed_kernel(int nx, int ny, int nz, int ldy, void* t0, void* t1, float* __restrict__ scratch,
                    double* __restrict__ nl_c, double* __restrict__ nl_d,
                    const float* __restrict__ lamx, const float* __restrict__ lamy,
                    const float* __restrict__ az, const float* __restrict__ bz,
                    const float* __restrict__ cz, const double* __restrict__ az64,
                    const double* __restrict__ bz64, const double* __restrict__ cz64,
                    const double* __restrict__ dz64, double alpha, double beta, int singular) {
  const long long lines = static_cast<long long>(nx) * ny;
  const long long line = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (line >= lines) return;
  const int q = static_cast<int>(line % ny), p = static_cast<int>(line / ny);
  const long long base = q + static_cast<long long>(ldy) * p;
  const long long stride = static_cast<long long>(ldy) * nx;
  if (singular && q == 0 && p == 0) {
    // float64 null line: project to compatible form, zero the last modal
    // unknown, shift to zero dz-weighted mean (c', d' kept in nl_c, nl_d)
    double s = 0.0, w = 0.0;
    for (int k = 0; k < nz; ++k) {
      s = fma(dz64[k], static_cast<double>(Elem<FMT>::load(t0, t1, base + k * stride)), s);
      w += dz64[k];
    }
    const double fshift = s / w;
    double cp = 0.0, dp = 0.0;
    for (int k = 0; k < nz; ++k) {
      const double sub = (k > 0) ? beta * az64[k] : 0.0;
      const double m = beta * bz64[k] - sub * cp;   // alpha = 0 and lambda = 0 on this line
      const double rhs = (static_cast<double>(Elem<FMT>::load(t0, t1, base + k * stride)) - fshift) - sub * dp;
      if (k == nz - 1) {
        dp = 0.0;
      } else {
        const double inv = 1.0 / m;
        cp = beta * cz64[k] * inv;
        dp = rhs * inv;
      }
      nl_c[k] = cp;
      nl_d[k] = dp;
    }
    double x = dp, xs = dz64[nz - 1] * dp;
    for (int k = nz - 2; k >= 0; --k) {
      x = nl_d[k] - nl_c[k] * x;
      nl_d[k] = x;
      xs = fma(dz64[k], x, xs);
    }
    const double mean = xs / w;
    for (int k = 0; k < nz; ++k)
      Elem<FMT>::store(t0, t1, base + k * stride, static_cast<float>(nl_d[k] - mean));
    return;
  }
  const float fb = static_cast<float>(beta);
  const float shift = static_cast<float>(alpha) + fb * (lamx[p] + lamy[q]);
  float cp = 0.0f, dp = 0.0f;
  for (int k = 0; k < nz; ++k) {
    const long long o = base + k * stride;
    const float sub = (k > 0) ? fb * az[k] : 0.0f;
    const float m = fmaf(-sub, cp, fmaf(fb, bz[k], shift));
    const float inv = 1.0f / m;
    cp = (k < nz - 1) ? fb * cz[k] * inv : 0.0f;
    dp = fmaf(-sub, dp, Elem<FMT>::load(t0, t1, o)) * inv;
    scratch[o] = cp;
    Elem<FMT>::store(t0, t1, o, dp);
  }
  float x = dp;
  for (int k = nz - 2; k >= 0; --k) {
    const long long o = base + k * stride;
    x = fmaf(-scratch[o], x, Elem<FMT>::load(t0, t1, o));
    Elem<FMT>::store(t0, t1, o, x);
  }
}

// Float-pair coefficient tables of one direction: a, c and the diagonal
// remainder w = -(a + b + c) of the float64 rows, so that
//   a phi_{i-1} + b phi_i + c phi_{i+1} = a (phi_{i-1} - phi_i) + c (phi_{i+1} - phi_i) - w phi_i.
struct DFRows {
  const float *ah, *al, *ch, *cl, *wh, *wl;
};

__device__ __forceinline__ df ld_df(const float* h, const float* l, long long i) { return {h[i], l[i]}; }

__device__ __forceinline__ df flux3(const DFRows& R, int i, df pm, df p0, df pp) {
  const df t1 = df_mul({R.ah[i], R.al[i]}, df_sub(pm, p0));
  const df t2 = df_mul({R.ch[i], R.cl[i]}, df_sub(pp, p0));
  const df t3 = df_mul({R.wh[i], R.wl[i]}, p0);
  return df_sub(df_add(t1, t2), t3);
}

// r = (f - fshift) - alpha phi - beta L phi in float-pair arithmetic; r goes to
// R (operand format, rows of ldx) and sum r^2 to sums[0].  One thread per
// (i, j), marching along k.
template <int FMT>
__global__ void __launch_bounds__(128)
residual_df_kernel(int nx, int ny, int nz, int ldx, const float* __restrict__ fh,
                   const float* __restrict__ fl, const float* __restrict__ ph,
                   const float* __restrict__ pl, void* r0, void* r1, DFRows RX, DFRows RY, DFRows RZ,
                   double alpha, double beta, const double* __restrict__ fsums, double inv_vol,
                   int singular, double* sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double s2 = 0.0;
  if (i < nx && j < ny) {
    const long long sy = nx, sz = static_cast<long long>(nx) * ny;
    const long long base = i + sy * j;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const df dalpha = df_from_double(alpha), dbeta = df_from_double(beta);
    const df fshift = df_from_double(singular ? fsums[2] * inv_vol : 0.0);
    df pm = ld_df(ph, pl, base + sz * (nz - 1));
    df p0 = ld_df(ph, pl, base);
    float acc = 0.0f;
    for (int k = 0; k < nz; ++k) {
      const long long o = base + sz * k;
      const df pp = ld_df(ph, pl, base + sz * ((k == nz - 1) ? 0 : k + 1));
      const df lx = flux3(RX, i, ld_df(ph, pl, im + sy * j + sz * k), p0, ld_df(ph, pl, ip + sy * j + sz * k));
      const df ly = flux3(RY, j, ld_df(ph, pl, i + sy * jm + sz * k), p0, ld_df(ph, pl, i + sy * jp + sz * k));
      const df lz = flux3(RZ, k, pm, p0, pp);
      const df lap = df_add(df_add(lx, ly), lz);
      const df ap = df_add(df_mul(dalpha, p0), df_mul(dbeta, lap));
      const df r = df_sub(df_sub(ld_df(fh, fl, o), fshift), ap);
      const float rv = r.hi + r.lo;
      Elem<FMT>::store(r0, r1, i + static_cast<long long>(ldx) * (j + static_cast<long long>(ny) * k), rv);
      acc = fmaf(rv, rv, acc);
      pm = p0;
      p0 = pp;
    }
    s2 = acc;
  }
  s2 = warp_sum_d(s2);
  if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == 0) atomicAdd(&sums[0], s2);
}

// sum of cell volume times phi (float pair) into *out, for the exact gauge
__global__ void __launch_bounds__(256)
wsum_df_kernel(int nx, int ny, int nz, const float* __restrict__ h, const float* __restrict__ l,
               const double* __restrict__ dxf, const double* __restrict__ dyf,
               const double* __restrict__ dzf, double* out) {
  const long long n = static_cast<long long>(nx) * ny * nz;
  double s = 0.0;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < n;
       o += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(o % nx);
    const long long line = o / nx;
    const int j = static_cast<int>(line % ny), k = static_cast<int>(line / ny);
    s = fma(dxf[i] * dyf[j] * dzf[k], static_cast<double>(h[o]) + static_cast<double>(l[o]), s);
  }
  s = warp_sum_d(s);
  if (threadIdx.x % 32 == 0) atomicAdd(out, s);
}

// phi = hi + lo - shift, shift = (*wsum) * inv_vol when wsum is given (the
// singular problem's zero volume-weighted-mean gauge, applied exactly)
__global__ void __launch_bounds__(256)
df_to_f64_kernel(long long n, const float* __restrict__ h, const float* __restrict__ l,
                 const double* __restrict__ wsum, double inv_vol, double* out) {
  const double shift = wsum ? *wsum * inv_vol : 0.0;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < n;
       o += static_cast<long long>(gridDim.x) * blockDim.x)
    out[o] = (static_cast<double>(h[o]) + static_cast<double>(l[o])) - shift;
}

// rows x K float64 (row-major, stride K) -> operand planes with row stride ld
template <int FMT>
__global__ void __launch_bounds__(256)
pack_kernel(int rows, int K, int ld, const double* __restrict__ src, void* d0, void* d1) {
  const long long n = static_cast<long long>(rows) * K;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < n;
       o += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = o / K;
    const int k = static_cast<int>(o % K);
    const double v = src[o];
    const long long di = r * ld + k;
    if (FMT == kFmtSplit) {
      const __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(v));
      static_cast<__nv_bfloat16*>(d0)[di] = h;
      static_cast<__nv_bfloat16*>(d1)[di] =
          __float2bfloat16_rn(static_cast<float>(v - static_cast<double>(__bfloat162float(h))));
    } else if (FMT == kFmtBF16) {
      static_cast<__nv_bfloat16*>(d0)[di] = __float2bfloat16_rn(static_cast<float>(v));
    } else {
      static_cast<float*>(d0)[di] = static_cast<float>(v);
    }
  }
}

int grid_for(long long n, int bs, int dev) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long nb = (n + bs - 1) / bs;
  const long long cap = 8LL * sms;
  return static_cast<int>(nb < 1 ? 1 : (nb > cap ? cap : nb));
}

}  // namespace

// ------------------------------------------------------------------ host side

int fmt_of(int precision) {
  return precision == TPT_PREC_MIXED_BF16X3 ? kFmtSplit
                                            : (precision == TPT_PREC_MIXED_TF32 ? kFmtF32 : kFmtBF16);
}
int elem_bytes(int fmt) { return fmt == kFmtF32 ? 4 : 2; }
int nplanes(int fmt) { return fmt == kFmtSplit ? 2 : 1; }
int kind_of(int fmt) { return fmt == kFmtF32 ? tc::kKindTF32 : tc::kKindBF16; }

cudaError_t pack_operand(int fmt, int rows, int K, int ld, const double* src, void* d0, void* d1,
                         int dev, cudaStream_t s) {
  const long long n = static_cast<long long>(rows) * K;
  const int nb = grid_for(n, 256, dev);
  note_launch(1);
  if (fmt == kFmtSplit) pack_kernel<kFmtSplit><<<nb, 256, 0, s>>>(rows, K, ld, src, d0, d1);
  else if (fmt == kFmtBF16) pack_kernel<kFmtBF16><<<nb, 256, 0, s>>>(rows, K, ld, src, d0, d1);
  else pack_kernel<kFmtF32><<<nb, 256, 0, s>>>(rows, K, ld, src, d0, d1);
  return cudaGetLastError();
}

}  // namespace tpt

namespace tpt {
namespace {

int st_of(cudaError_t e) {
  if (e == cudaSuccess) return TPT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}
#define MX_TRY(expr)               \
  do {                             \
    int st_ = (expr);              \
    if (st_ != TPT_OK) return st_; \
  } while (0)
#define MX_CUDA(expr) MX_TRY(st_of(expr))

int dev_alloc(tpt_plan_s* p, size_t bytes, void** out) {
  void* ptr = nullptr;
  if (cudaMalloc(&ptr, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_OOM;
  }
  p->allocs.push_back(ptr);
  *out = ptr;
  return TPT_OK;
}

template <typename T>
int upload_vec(tpt_plan_s* p, const std::vector<T>& h, T** d) {
  void* ptr = nullptr;
  MX_TRY(dev_alloc(p, h.size() * sizeof(T), &ptr));
  *d = static_cast<T*>(ptr);
  if (!h.empty()) MX_CUDA(cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TPT_OK;
}

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

void split_ld(long double v, float* h, float* l) {
  const float hi = static_cast<float>(v);
  *h = hi;
  *l = static_cast<float>(v - static_cast<long double>(hi));
}

// Workspace regions of the mixed path.
struct MixedWork {
  double* scal;        // 16 doubles: [1] sum r^2, [2] sum vol*phi, [5..7] sums of f, [15] error flag
  double* nl;          // 2 * Nz doubles: c', d' of the null line
  float *fh, *fl, *ph, *pl;
  void* R[2];
  void* A[2];
  void* B[2];
  float* scratch;
};

struct MixedSizes {
  size_t nf, nr, nab, nscr, eb, np;
};

MixedSizes sizes_of(const tpt_plan_s* p) {
  const MixedTables& m = p->mixed;
  const size_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
  MixedSizes s;
  s.nf = nx * ny * nz;
  s.nr = static_cast<size_t>(m.ldx) * ny * nz;
  s.nab = std::max(static_cast<size_t>(m.ldy) * nx, static_cast<size_t>(m.ldx) * ny) * nz;
  s.nscr = static_cast<size_t>(m.ldy) * nx * nz;
  s.eb = elem_bytes(m.fmt);
  s.np = nplanes(m.fmt);
  return s;
}

MixedWork carve(const tpt_plan_s* p, void* work) {
  const MixedSizes z = sizes_of(p);
  char* w = static_cast<char*>(work);
  MixedWork mw;
  mw.scal = reinterpret_cast<double*>(w);
  w += 256;
  mw.nl = reinterpret_cast<double*>(w);
  w += align256(2 * sizeof(double) * p->n[2]);
  float** fl[4] = {&mw.fh, &mw.fl, &mw.ph, &mw.pl};
  for (float** f : fl) {
    *f = reinterpret_cast<float*>(w);
    w += align256(z.nf * sizeof(float));
  }
  for (int pl = 0; pl < 2; ++pl) {
    mw.R[pl] = (pl < static_cast<int>(z.np)) ? static_cast<void*>(w) : nullptr;
    if (pl < static_cast<int>(z.np)) w += align256(z.nr * z.eb);
  }
  for (int pl = 0; pl < 2; ++pl) {
    mw.A[pl] = (pl < static_cast<int>(z.np)) ? static_cast<void*>(w) : nullptr;
    if (pl < static_cast<int>(z.np)) w += align256(z.nab * z.eb);
  }
  for (int pl = 0; pl < 2; ++pl) {
    mw.B[pl] = (pl < static_cast<int>(z.np)) ? static_cast<void*>(w) : nullptr;
    if (pl < static_cast<int>(z.np)) w += align256(z.nab * z.eb);
  }
  mw.scratch = reinterpret_cast<float*>(w);
  return mw;
}

int out_mode(int fmt) {
  return fmt == kFmtSplit ? tc::kOutSplitBF16 : (fmt == kFmtBF16 ? tc::kOutBF16 : tc::kOutF32);
}

tc::Operand operand(void* const pl[2], int rows, int K, int ld) {
  tc::Operand o;
  o.plane[0] = pl[0];
  o.plane[1] = pl[1];
  o.rows = rows;
  o.K = K;
  o.ld = ld;
  return o;
}

tc::GemmOut gout(int M, int N, int K, int rm, long long sm, long long sn, void* o0, void* o1, int mode,
                 int acc, int n_fastest, int* err) {
  tc::GemmOut g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.rm = rm;
  g.sm = sm;
  g.sn = sn;
  g.out0 = o0;
  g.out1 = o1;
  g.mode = mode;
  g.accumulate = acc;
  g.n_fastest = n_fastest;
  g.err = err;
  return g;
}

constexpr int kBig = 1 << 30;

template <int FMT>
cudaError_t launch_prepare(const tpt_plan_s* p, const double* f, const MixedWork& w, cudaStream_t s) {
  const long long n = static_cast<long long>(p->n[0]) * p->n[1] * p->n[2];
  note_launch(1);
  prepare_kernel<FMT><<<grid_for(n, 256, p->dev), 256, 0, s>>>(
      p->n[0], p->n[1], p->n[2], p->mixed.ldx, f, w.fh, w.fl, w.R[0], w.R[1], p->d_dxf[0], p->d_dxf[1],
      p->d_dxf[2], w.scal + 5);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_thomas(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  const MixedTables& m = p->mixed;
  const int nz = p->n[2];
  const long long lines = static_cast<long long>(p->n[0]) * p->n[1];
  const double* rz = p->d_rows[2];
  note_launch(1);
  thomas_mixed_kernel<FMT><<<static_cast<unsigned>((lines + 127) / 128), 128, 0, s>>>(
      p->n[0], p->n[1], nz, m.ldy, w.B[0], w.B[1], w.scratch, w.nl, w.nl + nz, m.lam_f[0], m.lam_f[1],
      m.zrows_f, m.zrows_f + nz, m.zrows_f + 2 * nz, rz, rz + nz, rz + 2 * nz, p->d_dxf[2], p->alpha,
      p->beta, p->singular ? 1 : 0);
  return cudaGetLastError();
}

DFRows rows_of(const float* t, int n) {
  return DFRows{t, t + n, t + 2 * n, t + 3 * n, t + 4 * n, t + 5 * n};
}

template <int FMT>
cudaError_t launch_residual(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  dim3 block(32, 4), grid((nx + 31) / 32, (ny + 3) / 4);
  note_launch(1);
  residual_df_kernel<FMT><<<grid, block, 0, s>>>(
      nx, ny, nz, p->mixed.ldx, w.fh, w.fl, w.ph, w.pl, w.R[0], w.R[1], rows_of(p->mixed.dfrows[0], nx),
      rows_of(p->mixed.dfrows[1], ny), rows_of(p->mixed.dfrows[2], nz), p->alpha, p->beta, w.scal + 5,
      1.0 / p->vol, p->singular ? 1 : 0, w.scal + 1);
  return cudaGetLastError();
}

template <int FMT>
int correction(tpt_plan_s* p, const MixedWork& w, bool accumulate, cudaStream_t s) {
  const MixedTables& m = p->mixed;
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int kind = kind_of(FMT), npl = nplanes(FMT), om = out_mode(FMT);
  int* err = reinterpret_cast<int*>(w.scal + 15);
  // step 2.1: x forward.  A = R rows (j,k), B = Q_x^{-1} rows p -> T1 (j, p, k)
  MX_CUDA(tc::gemm(kind, npl, operand(w.R, ny * nz, nx, m.ldx), operand(m.q[0][0], nx, nx, m.ldx),
                   gout(ny * nz, nx, nx, ny, static_cast<long long>(m.ldy) * nx, m.ldy, w.A[0], w.A[1], om,
                        0, 1, err),
                   s));
  // step 2.2: y forward.  A = Q_y^{-1} rows q, B = T1 rows (p,k) -> T2 (q, p, k)
  MX_CUDA(tc::gemm(kind, npl, operand(m.q[1][0], ny, ny, m.ldy), operand(w.A, nx * nz, ny, m.ldy),
                   gout(ny, nx * nz, ny, kBig, 0, m.ldy, w.B[0], w.B[1], om, 0, 0, err), s));
  // step 2.3: modal Thomas along z, in place on T2
  MX_CUDA(launch_thomas<FMT>(p, w, s));
  // step 2.4: y inverse.  A = T3 rows (p,k), B = Q_y rows j -> T4 (p, j, k)
  MX_CUDA(tc::gemm(kind, npl, operand(w.B, nx * nz, ny, m.ldy), operand(m.q[1][1], ny, ny, m.ldy),
                   gout(nx * nz, ny, ny, nx, static_cast<long long>(m.ldx) * ny, m.ldx, w.A[0], w.A[1], om,
                        0, 1, err),
                   s));
  // step 2.5: x inverse.  A = Q_x rows i, B = T4 rows (j,k) -> phi (float pair) (+)= result
  MX_CUDA(tc::gemm(kind, npl, operand(m.q[0][1], nx, nx, m.ldx), operand(w.A, ny * nz, nx, m.ldx),
                   gout(nx, ny * nz, nx, kBig, 0, nx, w.ph, w.pl, tc::kOutDF, accumulate ? 1 : 0, 0, err),
                   s));
  return TPT_OK;
}

double proj_norm2(const double* h, double npts, double vol, bool singular) {
  if (!singular) return h[5];
  const double c = h[7] / vol;
  return h[5] - 2.0 * c * h[6] + npts * c * c;
}

template <int FMT>
int solve_fmt(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s, tpt_info* info) {
  const MixedWork w = carve(p, work);
  MX_CUDA(cudaMemsetAsync(w.scal, 0, 16 * sizeof(double), s));
  MX_CUDA(launch_prepare<FMT>(p, f, w, s));
  const int corrections = 1 + p->max_refine;
  const bool adaptive = p->rtol > 0.0;
  const double np = static_cast<double>(npts(p));
  double h[16] = {0.0};
  double rel = -1.0;
  int iters = 0, status = TPT_OK;
  bool converged = false;
  for (;;) {
    MX_TRY(correction<FMT>(p, w, iters > 0, s));
    ++iters;
    const bool need_residual = iters < corrections || adaptive || info;
    if (!need_residual) break;
    MX_CUDA(cudaMemsetAsync(w.scal + 1, 0, sizeof(double), s));
    MX_CUDA(launch_residual<FMT>(p, w, s));
    if (adaptive) {
      MX_CUDA(cudaMemcpyAsync(h, w.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MX_CUDA(cudaStreamSynchronize(s));
      int errflag = 0;
      std::memcpy(&errflag, &h[15], sizeof(int));
      if (errflag) return TPT_ERR_TIMEOUT;
      const double fn2 = proj_norm2(h, np, p->vol, p->singular);
      if (!std::isfinite(h[1]) || !std::isfinite(fn2)) return TPT_ERR_NONFINITE;
      rel = fn2 > 0.0 ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
      if (rel <= p->rtol) {
        converged = true;
        break;
      }
    }
    if (iters >= corrections) break;
  }
  const long long n = static_cast<long long>(np);
  if (p->singular) {
    MX_CUDA(cudaMemsetAsync(w.scal + 2, 0, sizeof(double), s));
    note_launch(1);
    wsum_df_kernel<<<grid_for(n, 256, p->dev), 256, 0, s>>>(p->n[0], p->n[1], p->n[2], w.ph, w.pl, p->d_dxf[0],
                                                            p->d_dxf[1], p->d_dxf[2], w.scal + 2);
    MX_CUDA(cudaGetLastError());
  }
  note_launch(1);
  df_to_f64_kernel<<<grid_for(n, 256, p->dev), 256, 0, s>>>(n, w.ph, w.pl, p->singular ? w.scal + 2 : nullptr,
                                                            1.0 / p->vol, phi);
  MX_CUDA(cudaGetLastError());
  if (adaptive && !converged) status = TPT_ERR_NOT_CONVERGED;
  if (info) {
    if (!adaptive) {
      MX_CUDA(cudaMemcpyAsync(h, w.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MX_CUDA(cudaStreamSynchronize(s));
      const double fn2 = proj_norm2(h, np, p->vol, p->singular);
      rel = fn2 > 0.0 ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
    }
    info->iters = iters;
    info->rel_residual = rel;
    info->compat_defect = p->singular ? h[7] / p->vol : 0.0;
    for (float& t : info->ms_stage) t = 0.0f;
  }
  return status;
}

}  // namespace

int mixed_setup(tpt_plan_s* p) {
  MixedTables& m = p->mixed;
  m.fmt = fmt_of(p->precision);
  m.ldx = (p->n[0] + 7) & ~7;
  m.ldy = (p->n[1] + 7) & ~7;
  const int np = nplanes(m.fmt);
  const size_t eb = elem_bytes(m.fmt);
  for (int d = 0; d < 2; ++d) {
    const int n = p->n[d];
    const int ld = d == 0 ? m.ldx : m.ldy;
    const std::vector<double>& qt = p->eig[d].qt;
    const std::vector<double>& dxf = p->dir[d].dxf;
    std::vector<double> fwd(static_cast<size_t>(n) * n), inv(static_cast<size_t>(n) * n);
    for (int mode = 0; mode < n; ++mode)
      for (int i = 0; i < n; ++i) {
        const double s = std::sqrt(dxf[i]);
        const double q = qt[static_cast<size_t>(mode) * n + i];
        fwd[static_cast<size_t>(mode) * n + i] = q * s;   // Q^{-1}(mode, i), row-major
        inv[static_cast<size_t>(i) * n + mode] = q / s;   // Q(i, mode), row-major
      }
    for (int role = 0; role < 2; ++role) {
      double* stage = nullptr;
      MX_TRY(upload_vec(p, role == 0 ? fwd : inv, &stage));
      for (int pl = 0; pl < np; ++pl) MX_TRY(dev_alloc(p, eb * static_cast<size_t>(n) * ld, &m.q[d][role][pl]));
      MX_CUDA(cudaMemset(m.q[d][role][0], 0, eb * static_cast<size_t>(n) * ld));
      if (np == 2) MX_CUDA(cudaMemset(m.q[d][role][1], 0, eb * static_cast<size_t>(n) * ld));
      MX_CUDA(pack_operand(m.fmt, n, n, ld, stage, m.q[d][role][0], m.q[d][role][1], p->dev, 0));
    }
    std::vector<float> lf(p->eig[d].lam.begin(), p->eig[d].lam.end());
    MX_TRY(upload_vec(p, lf, &m.lam_f[d]));
  }
  {
    const Dir1D& z = p->dir[2];
    std::vector<float> zr(3 * static_cast<size_t>(z.n));
    for (int k = 0; k < z.n; ++k) {
      zr[k] = static_cast<float>(z.a[k]);
      zr[z.n + k] = static_cast<float>(z.b[k]);
      zr[2 * z.n + k] = static_cast<float>(z.c[k]);
    }
    MX_TRY(upload_vec(p, zr, &m.zrows_f));
  }
  for (int d = 0; d < 3; ++d) {
    const Dir1D& dd = p->dir[d];
    const int n = dd.n;
    std::vector<float> t(6 * static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) {
      const long double a = dd.a[i], b = dd.b[i], c = dd.c[i];
      split_ld(a, &t[i], &t[n + i]);
      split_ld(c, &t[2 * n + i], &t[3 * n + i]);
      split_ld(-(a + b + c), &t[4 * n + i], &t[5 * n + i]);
    }
    MX_TRY(upload_vec(p, t, &m.dfrows[d]));
  }
  MX_CUDA(cudaDeviceSynchronize());
  return TPT_OK;
}

size_t mixed_workspace_bytes(const tpt_plan_s* p) {
  const MixedSizes z = sizes_of(p);
  size_t b = 256 + align256(2 * sizeof(double) * p->n[2]);
  b += 4 * align256(z.nf * sizeof(float));
  b += z.np * align256(z.nr * z.eb);
  b += 2 * z.np * align256(z.nab * z.eb);
  b += align256(z.nscr * sizeof(float));
  return b;
}

int mixed_solve(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s, tpt_info* info) {
  switch (p->mixed.fmt) {
    case kFmtSplit: return solve_fmt<kFmtSplit>(p, f, phi, work, s, info);
    case kFmtBF16: return solve_fmt<kFmtBF16>(p, f, phi, work, s, info);
    default: return solve_fmt<kFmtF32>(p, f, phi, work, s, info);
  }
}

int tc_gemm_test(int precision, int M, int N, int K, const double* A, const double* B, double* D,
                 void* work, int dev, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !D || !work) return TPT_ERR_INVALID_ARG;
  if (precision < TPT_PREC_MIXED_BF16 || precision > TPT_PREC_MIXED_TF32) return TPT_ERR_INVALID_ARG;
  const int fmt = fmt_of(precision);
  const int ld = (K + 7) & ~7;
  const size_t eb = elem_bytes(fmt);
  char* w = static_cast<char*>(work);
  void* pa[2] = {w, w + align256(eb * static_cast<size_t>(M) * ld)};
  char* wb = w + 2 * align256(eb * static_cast<size_t>(M) * ld);
  void* pb[2] = {wb, wb + align256(eb * static_cast<size_t>(N) * ld)};
  if (nplanes(fmt) == 1) {
    pa[1] = nullptr;
    pb[1] = nullptr;
  }
  MX_CUDA(pack_operand(fmt, M, K, ld, A, pa[0], pa[1], dev, s));
  MX_CUDA(pack_operand(fmt, N, K, ld, B, pb[0], pb[1], dev, s));
  MX_CUDA(tc::gemm(kind_of(fmt), nplanes(fmt), operand(pa, M, K, ld), operand(pb, N, K, ld),
                   gout(M, N, K, kBig, 0, M, D, nullptr, tc::kOutF64, 0, 0, nullptr), s));
  return TPT_OK;
}

}  // namespace tpt
