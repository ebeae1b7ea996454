// Float64-accurate transform GEMMs on the bf16 tensor cores by the Ozaki
// scheme (error-free splitting of the operands into slices whose products sum
// exactly in the float32 accumulator; Ozaki, Ogita, Oishi and Rump 2012, and
// its tensor-core form of Ootomo, Ozaki and Yokota 2024).  It replaces the
// float64 DGEMM of the eigenbasis transforms (Sec. 2.2.2 solution steps 2.1,
// 2.2, 2.4, 2.5; Algorithm 1 steps 1, 3, 7, 9) of a TPT_PREC_FP64_OZAKI plan.
//
// Slicing.  Each row x of an operand (the K values one output element
// contracts with) is split into kOzS slices
//     x = sum_{t=1..S} q_t 2^(e - beta t) + r,   |r| <= 2^(e - beta S - 1),
// with 2^e > max |x| (one exponent per row), q_t integers, |q_1| <= 2^beta + 1
// and |q_t| <= 2^(beta-1) after it; each q_t 2^(e - beta t) has at most seven
// significant bits and is exact in bf16.
//
// Levels.  A product of slices s and t of two rows is an integer times
// 2^(e_m + e_n - beta (s + t)); all pairs with s + t = L share that scale, so
// their sums over K are integers times it.  With beta = 6 a level's products
// are at most 65^2 units (level 2, one pair) or 2 x 65 x 32 + 5 x 32^2 units
// (later levels), so with K <= 576 every partial sum stays below 2^24 units:
// the float32 accumulator of one level is exact whatever the order.  Level L is
// one plain bf16 GEMM over the slices laid side by side along K, the first
// operand's slices 1..L-1 against the second's L-1..1; the second operand is
// therefore stored with its slices in reverse order, so that every level reads
// a prefix of the first operand's row and a suffix of the second's.  All
// levels run in one launch of the transform GEMM: each output tile takes the
// levels in turn (double-buffered accumulators in tensor memory), and the
// epilogue adds each level into the float64 output while the tile is still in
// L2, so the output crosses DRAM once.  Levels 2..S+1 are kept
// (pairs with s + t > S + 1 are below 2^-(beta (S+1)) of the scale); with
// S = 7 the product is accurate to ~1e-13 of sum_k |a_k||b_k|, and the float64
// refinement of the solve removes the rest.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "tc.h"
#include "tpt_internal.h"

namespace tpt {
namespace {

constexpr int kOzS = 7;       // slices per operand row
constexpr int kOzBeta = 6;    // bits per slice
constexpr int kOzMaxK = 576;  // contraction length that keeps a level's sums exact

size_t al256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Slices of one value x of a row with exponent e (2^e > max |x|), by integer
// arithmetic only: X = round(x 2^(beta S - e)) (|X| <= 2^(beta S)), written in
// balanced base-2^beta digits d_S .. d_2 in [-2^(beta-1), 2^(beta-1)) and a top
// digit d_1 (|d_1| <= 2^beta + 1); slice t is d_t 2^(e - beta t), exact in
// float32 and in bf16 (at most seven significant bits).  The dropped part of x
// is at most 2^(e - beta S - 1).
__host__ __device__ inline void slice_value(double x, int e, float* q) {
  uint64_t bits;
#ifdef __CUDA_ARCH__
  bits = static_cast<uint64_t>(__double_as_longlong(x));
#else
  std::memcpy(&bits, &x, sizeof(bits));
#endif
  const int ex = static_cast<int>((bits >> 52) & 0x7ff);
  long long X = 0;
  if (ex != 0) {   // zero and subnormal values give zero digits
    const long long mant = static_cast<long long>((bits & ((1ull << 52) - 1)) | (1ull << 52));
    const int sh = 1075 + e - kOzBeta * kOzS - ex;   // x = mant 2^(ex - 1075)
    if (sh <= 0) X = mant << (-sh);                     // not reached for |x| < 2^e
    else if (sh < 62) X = (mant + (1LL << (sh - 1))) >> sh;
    if (bits >> 63) X = -X;
  }
  for (int t = kOzS; t >= 2; --t) {
    const long long d = ((X + (1LL << (kOzBeta - 1))) & ((1LL << kOzBeta) - 1)) - (1LL << (kOzBeta - 1));
    X = (X - d) >> kOzBeta;
    q[t - 1] = ldexpf(static_cast<float>(d), e - kOzBeta * t);
  }
  q[0] = ldexpf(static_cast<float>(X), e - kOzBeta);
}

// The row exponent: e with 2^(e-1) <= m < 2^e for the row maximum m > 0, as
// frexp gives it; 0 for m = 0 or subnormal (the row's digits are then zero).
__host__ __device__ inline int row_exponent(double m) {
  uint64_t bits;
#ifdef __CUDA_ARCH__
  bits = static_cast<uint64_t>(__double_as_longlong(m));
#else
  std::memcpy(&bits, &m, sizeof(bits));
#endif
  const int ex = static_cast<int>((bits >> 52) & 0x7ff);
  return ex == 0 ? 0 : ex - 1022;
}

// The digits of slice_value for one value given its bits, with each slice
// d_t 2^(e - beta t) formed as float(d_t) times a power of two built from its
// bits (the caller checks that 2^(e - beta S) and 2^(e - beta) are normal
// floats, so the products are the exact values ldexpf gives).  Integer and
// float32 operations only: GB300's float64 pipe is ~1/64 of the float32 rate.
__device__ __forceinline__ void slice_value_dev(unsigned long long bits, int e, float* q) {
  const int ex = static_cast<int>((bits >> 52) & 0x7ff);
  long long X = 0;
  if (ex != 0) {
    const long long mant = static_cast<long long>((bits & ((1ull << 52) - 1)) | (1ull << 52));
    const int sh = 1075 + e - kOzBeta * kOzS - ex;
    if (sh <= 0) X = mant << (-sh);
    else if (sh < 62) X = (mant + (1LL << (sh - 1))) >> sh;
    if (bits >> 63) X = -X;
  }
  for (int t = kOzS; t >= 2; --t) {
    const long long d = ((X + (1LL << (kOzBeta - 1))) & ((1LL << kOzBeta) - 1)) - (1LL << (kOzBeta - 1));
    X = (X - d) >> kOzBeta;
    q[t - 1] = static_cast<float>(static_cast<int>(d)) * __int_as_float((127 + e - kOzBeta * t) << 23);
  }
  q[0] = static_cast<float>(static_cast<int>(X)) * __int_as_float((127 + e - kOzBeta) << 23);
}

// Rows x K float64 (element (r, k) at src[r rs + k]) into kOzS bf16 slices per
// row at dst[r ld + pos Kp + k], ld = kOzS Kp, pos = t - 1 (reversed: kOzS - t);
// columns K..Kp-1 are zero.  One warp per row; the row maximum is taken on
// the bit patterns (for non-negative doubles they order as the values do).
__global__ void __launch_bounds__(256)
ozaki_slice_kernel(long long rows, int K, int Kp, long long rs, const double* __restrict__ src,
                   __nv_bfloat16* __restrict__ dst, int reversed) {
  const int lane = threadIdx.x % 32;
  const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x / 32);
  for (long long r = blockIdx.x * static_cast<long long>(blockDim.x / 32) + threadIdx.x / 32; r < rows;
       r += warps) {
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(src + r * rs);
    unsigned long long m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, row[k] & 0x7fffffffffffffffull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = row_exponent(__longlong_as_double(static_cast<long long>(m)));
    // 2^(e - beta S) .. 2^(e - beta) normal: the fast slices (uniform over the warp)
    const bool fast = e - kOzBeta * kOzS >= -126 && e - kOzBeta <= 127;
    __nv_bfloat16* out = dst + r * static_cast<long long>(kOzS) * Kp;
    for (int k = lane; k < Kp; k += 32) {
      float q[kOzS];
      if (k < K) {
        if (fast) slice_value_dev(row[k], e, q);
        else slice_value(__longlong_as_double(static_cast<long long>(row[k])), e, q);
      } else {
#pragma unroll
        for (int t = 0; t < kOzS; ++t) q[t] = 0.0f;
      }
#pragma unroll
      for (int t = 1; t <= kOzS; ++t) {
        const int pos = reversed ? kOzS - t : t - 1;
        out[static_cast<long long>(pos) * Kp + k] = __float2bfloat16_rn(q[t - 1]);
      }
    }
  }
}

// (Nx, Ny, Nz) field -> rows (i, k) of Ny values: out[(i + Nx k) Ny + j] = in[i + Nx j + Nx Ny k],
// through 32 x 32 shared-memory tiles of each z-slab.
__global__ void __launch_bounds__(256)
transpose_xy_kernel(int nx, int ny, int nz, const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;
  for (int k = blockIdx.z; k < nz; k += gridDim.z) {
    const double* src = in + static_cast<long long>(nx) * ny * k;
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int i = bi + threadIdx.x, j = bj + r;
      tile[r][threadIdx.x] = (i < nx && j < ny) ? src[i + static_cast<long long>(nx) * j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int i = bi + r, j = bj + threadIdx.x;
      if (i < nx && j < ny) out[(i + static_cast<long long>(nx) * k) * ny + j] = tile[threadIdx.x][r];
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

// bf16 bits of a float with at most eight significant bits (exact)
uint16_t bf16_bits(float v) {
  uint32_t b;
  std::memcpy(&b, &v, sizeof(b));
  return static_cast<uint16_t>(b >> 16);
}

// rows x K matrix (element (r, k) at m[r rs + k cs]) into slices as the
// kernel writes them; uploaded into the plan's arena.
int slice_matrix_host(tpt_plan_s* p, const std::vector<double>& m, int rows, int K, long long rs, long long cs,
                      int Kp, bool reversed, void** out) {
  std::vector<uint16_t> h(static_cast<size_t>(rows) * kOzS * Kp, 0);
  for (int r = 0; r < rows; ++r) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::fmax(mx, std::fabs(m[r * rs + k * cs]));
    const int e = row_exponent(mx);
    for (int k = 0; k < K; ++k) {
      float q[kOzS];
      slice_value(m[r * rs + k * cs], e, q);
      for (int t = 1; t <= kOzS; ++t) {
        const int pos = reversed ? kOzS - t : t - 1;
        h[(static_cast<size_t>(r) * kOzS + pos) * Kp + k] = bf16_bits(q[t - 1]);
      }
    }
  }
  return p->arena.upload(h.data(), h.size() * sizeof(uint16_t), out);
}

}  // namespace

bool ozaki_supported(const tpt_plan_s* p) {
  for (int d = 0; d < 2; ++d)
    if (!p->dir[d].excluded() && p->xform[d] == TPT_XFORM_GEMM && p->n[d] > kOzMaxK) return false;
  return true;
}

int ozaki_setup(tpt_plan_s* p) {
  if (!ozaki_supported(p)) return TPT_ERR_UNSUPPORTED;
  for (int d = 0; d < 2; ++d) {
    if (p->dir[d].excluded() || p->xform[d] != TPT_XFORM_GEMM) continue;
    const int n = p->n[d];
    const int kp = (n + 63) & ~63;   // whole 64-element K chunks per slice (zero padded)
    p->oz_kp[d] = kp;
    for (int inv = 0; inv < 2; ++inv) {
      // the float64 DGEMM's matrix (column-major n x n): x transforms use it as
      // the first operand, rows = output modes (A[r][k] = mat[r + n k]); y
      // transforms as the second, rows = output modes (B[r][k] = mat[k + n r])
      std::vector<double> mat(static_cast<size_t>(n) * n);
      const double* src = inv ? p->ddir[d].inv : p->ddir[d].fwd;
      if (cudaMemcpy(mat.data(), src, mat.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return TPT_ERR_CUDA;
      }
      const int st = d == 0 ? slice_matrix_host(p, mat, n, n, 1, n, kp, false, &p->oz_tab[2 * d + inv])
                            : slice_matrix_host(p, mat, n, n, n, 1, kp, true, &p->oz_tab[2 * d + inv]);
      if (st != TPT_OK) return st;
    }
  }
  p->ozaki = true;
  return TPT_OK;
}

size_t ozaki_scratch_bytes(const tpt_plan_s* p) {
  const size_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const size_t sx = al256(ny * nz * kOzS * static_cast<size_t>(p->oz_kp[0]) * 2);
  const size_t sy = al256(nx * ny * nz * sizeof(double)) + al256(nx * nz * kOzS * static_cast<size_t>(p->oz_kp[1]) * 2);
  return 256 + (sx > sy ? sx : sy);
}

cudaError_t ozaki_transform(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                            bool accumulate, void* scratch, int* err, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int kp = p->oz_kp[d];
  const int ld = kOzS * kp;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev);
  char* w = static_cast<char*>(scratch) + 256;
  const __nv_bfloat16* tab = static_cast<const __nv_bfloat16*>(p->oz_tab[2 * d + (inverse ? 1 : 0)]);
  __nv_bfloat16* sl;
  long long rows;
  if (d == 0) {   // rows (j, k) of the field, K = x: the second operand, slices reversed
    rows = static_cast<long long>(ny) * nz;
    sl = reinterpret_cast<__nv_bfloat16*>(w);
    const long long blocks = (rows + 7) / 8;
    note_launch(1);
    ozaki_slice_kernel<<<static_cast<unsigned>(blocks < 16LL * sms ? blocks : 16LL * sms), 256, 0, s>>>(
        rows, nx, kp, nx, in, sl, 1);
  } else {        // rows (i, k), K = y: the first operand, after a transpose of each z-slab
    rows = static_cast<long long>(nx) * nz;
    double* xt = reinterpret_cast<double*>(w);
    sl = reinterpret_cast<__nv_bfloat16*>(w + al256(static_cast<size_t>(nx) * ny * nz * sizeof(double)));
    note_launch(2);
    transpose_xy_kernel<<<dim3((nx + 31) / 32, (ny + 31) / 32, nz < 64 ? nz : 64), dim3(32, 8), 0, s>>>(nx, ny, nz,
                                                                                                   in, xt);
    const long long blocks = (rows + 7) / 8;
    ozaki_slice_kernel<<<static_cast<unsigned>(blocks < 16LL * sms ? blocks : 16LL * sms), 256, 0, s>>>(
        rows, ny, kp, ny, xt, sl, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // one launch for the seven levels: every output tile takes level L = 2..8
  // (slices 1..L-1 of A against L-1..1 of B, K = (L - 1) Kp) in turn, the
  // first written (or added, when accumulating) and the rest added in float64
  // while the tile is still in L2
  const int kall = kOzS * kp;
  tc::Operand a, b;
  tc::GemmOut g;
  std::memset(&g, 0, sizeof(g));
  if (d == 0) {
    a = tc::Operand{{tab, nullptr}, nx, kall, ld};
    b = tc::Operand{{sl, nullptr}, static_cast<int>(rows), kall, ld};
    g.M = nx;
    g.N = static_cast<int>(rows);
    g.rm = nx;
    g.sm = 0;
    g.sn = nx;
  } else {
    a = tc::Operand{{sl, nullptr}, static_cast<int>(rows), kall, ld};
    b = tc::Operand{{tab, nullptr}, ny, kall, ld};
    g.M = static_cast<int>(rows);
    g.N = ny;
    g.rm = nx;
    g.sm = static_cast<long long>(nx) * ny;
    g.sn = nx;
  }
  g.K = kall;
  g.out0 = out;
  g.mode = tc::kOutF64;
  g.accumulate = accumulate ? 1 : 0;
  g.levels = kOzS;
  g.level_k = kp;
  // consecutive CTAs share the data tile: x (data second) walks the few
  // m-tiles of the matrix fastest, y (data first) the few n-tiles
  g.n_fastest = d == 0 ? 0 : 1;
  g.err = err;
  g.tma_out = 0;
  return tc::gemm(tc::kKindBF16, 1, a, b, g, s);
}

}  // namespace tpt
