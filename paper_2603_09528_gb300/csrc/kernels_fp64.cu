// float64 kernels of the solve: the eigenbasis-transform GEMM (Sec. 2.2.2,
// Eq. forward-xy / inverse-xy; lines stacked as one GEMM), the modal Thomas
// sweep along z (solution step 2.3, with the gauge of Sec. 3), and the
// 7-point residual r = f - (alpha I + beta L) phi (Sec. 4.1).
//
// float64 arithmetic on GB300 runs at about 1 TFLOP/s (FMA and DMMA alike), so
// these kernels are bound by the float64 pipe, not by HBM; the layouts below
// keep every global access coalesced so that the float64 units stay fed.
#include <cuda_runtime.h>

#include <cmath>

#include "tpt_internal.h"

namespace tpt {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;   // block tile and k-step
constexpr int TX = 16, TY = 16;            // 256 threads, 4 x 4 outputs each

// C_b = A_b B_b (+ C_b): column-major, ragged edges zero-filled in shared memory.
__global__ void __launch_bounds__(TX * TY)
dgemm_cm_kernel(int M, int N, int K, const double* __restrict__ A, int lda, long long sA,
                const double* __restrict__ B, int ldb, long long sB, double* __restrict__ C,
                int ldc, long long sC, int accumulate) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const long long b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int r = 0; r < (TM * TK) / (TX * TY); ++r) {   // A tile, coalesced along m
      const int e = tid + r * TX * TY, m = e % TM, k = e / TM;
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < M && gk < K) ? A[gm + static_cast<long long>(gk) * lda] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < (TN * TK) / (TX * TY); ++r) {   // B tile, coalesced along k
      const int e = tid + r * TX * TY, k = e % TK, n = e / TK;
      const int gk = k0 + k, gn = n0 + n;
      Bs[k][n] = (gk < K && gn < N) ? B[gk + static_cast<long long>(gn) * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][tx + TX * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + TY * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gn = n0 + ty + TY * c;
    if (gn >= N) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gm = m0 + tx + TX * r;
      if (gm >= M) continue;
      double* p = C + gm + static_cast<long long>(gn) * ldc;
      *p = accumulate ? *p + acc[r][c] : acc[r][c];
    }
  }
}

// 1 / m in float64 without a division: the float32 reciprocal as the seed
// (relative error below 2^-21) and two Newton steps r <- r + r (1 - m r), each
// of which squares the relative error (2^-42, then below the float64
// rounding).  Pivots outside the float32 range take the division.
__device__ __forceinline__ double recip_fp64(double m) {
  const float rf = __fdividef(1.0f, static_cast<float>(m));
  if (!(fabsf(rf) < 1.0e37f && fabsf(rf) > 1.0e-37f)) return 1.0 / m;
  double r = static_cast<double>(rf);
  r = fma(r, fma(-m, r, 1.0), r);
  return fma(r, fma(-m, r, 1.0), r);
}

// One thread per (i, j) line.  Forward elimination keeps c' in `scratch`
// and d' in `out`; back substitution overwrites `out`.  The singular line
// (null_i, null_j) is first projected to compatible form (its dz-weighted
// mean removed, recorded in *defect), its last modal unknown is set to zero,
// and the result is shifted to zero dz-weighted mean.  The beta-scaled z rows
// are staged in shared memory once per block (3 Nz doubles, dynamic) when
// ROWS is set; the pipe that bounds the kernel is GB300's float64 pipe, so
// the per-point work is kept to two DFMA, the reciprocal and two multiplies
// forward and one DFMA back.  f may alias out (each element is read before
// the same thread writes it).
template <bool ROWS>
__global__ void __launch_bounds__(128)
thomas_fp64_kernel(int nx, int ny, int nz, const double* f, double* out,
                   double* __restrict__ scratch, const double* __restrict__ lamx,
                   const double* __restrict__ lamy, const double* __restrict__ az,
                   const double* __restrict__ bz, const double* __restrict__ cz,
                   const double* __restrict__ dz, double alpha, double beta, int null_i,
                   int null_j, double null_scale, double* defect) {
  extern __shared__ double zrow[];   // beta a, beta b, beta c (ROWS)
  if (ROWS) {
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
      zrow[k] = k > 0 ? beta * az[k] : 0.0;
      zrow[nz + k] = beta * bz[k];
      zrow[2 * nz + k] = k < nz - 1 ? beta * cz[k] : 0.0;
    }
    __syncthreads();
  }
  auto ra = [&](int k) { return ROWS ? zrow[k] : (k > 0 ? beta * az[k] : 0.0); };
  auto rb = [&](int k) { return ROWS ? zrow[nz + k] : beta * bz[k]; };
  auto rc = [&](int k) { return ROWS ? zrow[2 * nz + k] : (k < nz - 1 ? beta * cz[k] : 0.0); };
  const long long lines = static_cast<long long>(nx) * ny;
  const long long line = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (line >= lines) return;
  const int i = static_cast<int>(line % nx), j = static_cast<int>(line / nx);
  const bool is_null = (i == null_i && j == null_j);
  const double shift = alpha + beta * (lamx[i] + lamy[j]);
  double fshift = 0.0;
  if (is_null) {
    double s = 0.0, w = 0.0;
    for (int k = 0; k < nz; ++k) {
      s = fma(dz[k], f[line + k * lines], s);
      w += dz[k];
    }
    fshift = s / w;
    if (defect) *defect = fshift * null_scale;
  }
  double cp = 0.0, dp = 0.0;
  for (int k = 0; k < nz; ++k) {
    const long long o = line + k * lines;
    const double sub = ra(k);
    const double m = fma(-sub, cp, rb(k) + shift);
    double fo = f[o];
    if (is_null) fo -= fshift;
    const double rhs = fma(-sub, dp, fo);
    if (is_null && k == nz - 1) {
      dp = 0.0;   // vanishing final pivot: the modal unknown is set to zero
    } else {
      const double inv = recip_fp64(m);
      cp = rc(k) * inv;
      dp = rhs * inv;
    }
    scratch[o] = cp;
    out[o] = dp;
  }
  double x = dp;
  for (int k = nz - 2; k >= 0; --k) {
    const long long o = line + k * lines;
    x = fma(-scratch[o], x, out[o]);
    out[o] = x;
  }
  if (is_null) {
    double xs = 0.0, w = 0.0;
    for (int k = 0; k < nz; ++k) {
      xs = fma(dz[k], out[line + k * lines], xs);
      w += dz[k];
    }
    const double mean = xs / w;
    for (int k = 0; k < nz; ++k) out[line + k * lines] -= mean;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = (f - fshift) - (alpha phi + beta (Lx + Ly + Lz) phi); one thread per
// (i, j) marching along k.  End couplings of non-periodic directions are zero,
// so wrapped neighbour indices only ever meet a zero coefficient.  The
// beta-scaled rows are formed once (x and y per thread, z per block in shared
// memory when ROWS, with alpha folded into the z diagonal), so that a point
// costs six FMAs for the neighbours, one for the diagonal and one subtraction
// on GB300's float64 pipe (~1/64 of the float32 rate, the bound of this
// kernel).  sums[0] += sum r^2; with ALL also sums[1] += sum r and sums[2] +=
// sum vol*r.
template <bool ROWS, bool ALL>
__global__ void __launch_bounds__(128)
residual_fp64_kernel(int nx, int ny, int nz, const double* __restrict__ f,
                     const double* __restrict__ phi, double* __restrict__ r,
                     const double* __restrict__ rx, const double* __restrict__ ry,
                     const double* __restrict__ rz, const double* __restrict__ dxf,
                     const double* __restrict__ dyf, const double* __restrict__ dzf,
                     double alpha, double beta, const double* __restrict__ fshift_p,
                     double* sums) {
  extern __shared__ double zrow[];   // beta a_k, beta b_k + alpha, beta c_k (ROWS)
  if (ROWS) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    for (int k = tid; k < nz; k += nt) {
      zrow[k] = beta * rz[k];
      zrow[nz + k] = fma(beta, rz[nz + k], alpha);
      zrow[2 * nz + k] = beta * rz[2 * nz + k];
    }
    __syncthreads();
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double s2 = 0.0, s1 = 0.0, sv = 0.0;
  if (i < nx && j < ny) {
    const long long sy = nx, sz = static_cast<long long>(nx) * ny;
    const long long base = i + sy * j;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const double ax = beta * rx[i], cx = beta * rx[2 * nx + i];
    const double ay = beta * ry[j], cy = beta * ry[2 * ny + j];
    const double bxy = beta * (rx[nx + i] + ry[ny + j]);
    const double fshift = fshift_p ? *fshift_p : 0.0;
    const double vxy = ALL ? dxf[i] * dyf[j] : 0.0;
    double pm = phi[base + sz * (nz - 1)];   // wrap partner, multiplied by a_0 = 0
    double p0 = phi[base];
    for (int k = 0; k < nz; ++k) {
      const long long o = base + sz * k;
      const double pp = phi[base + sz * ((k == nz - 1) ? 0 : k + 1)];
      const double az = ROWS ? zrow[k] : beta * rz[k];
      const double bz = ROWS ? zrow[nz + k] : fma(beta, rz[nz + k], alpha);
      const double cz = ROWS ? zrow[2 * nz + k] : beta * rz[2 * nz + k];
      double acc = ax * phi[im + sy * j + sz * k];
      acc = fma(cx, phi[ip + sy * j + sz * k], acc);
      acc = fma(ay, phi[i + sy * jm + sz * k], acc);
      acc = fma(cy, phi[i + sy * jp + sz * k], acc);
      acc = fma(az, pm, acc);
      acc = fma(cz, pp, acc);
      acc = fma(bxy + bz, p0, acc);
      const double val = (fshift_p ? f[o] - fshift : f[o]) - acc;
      r[o] = val;
      s2 = fma(val, val, s2);
      if (ALL) {
        s1 += val;
        sv = fma(vxy * dzf[k], val, sv);
      }
      pm = p0;
      p0 = pp;
    }
  }
  if (sums) {
    s2 = warp_sum(s2);
    if (ALL) {
      s1 = warp_sum(s1);
      sv = warp_sum(sv);
    }
    if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == 0) {
      atomicAdd(&sums[0], s2);
      if (ALL) {
        atomicAdd(&sums[1], s1);
        atomicAdd(&sums[2], sv);
      }
    }
  }
}

// sums[0] += sum f^2, sums[1] += sum f, sums[2] += sum vol*f  (grid-stride)
__global__ void __launch_bounds__(256)
field_sums_kernel(int nx, int ny, int nz, const double* __restrict__ f, const double* __restrict__ dxf,
                  const double* __restrict__ dyf, const double* __restrict__ dzf, double* sums) {
  const long long n = static_cast<long long>(nx) * ny * nz;
  double s2 = 0.0, s1 = 0.0, sv = 0.0;
  for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < n;
       o += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(o % nx);
    const long long jk = o / nx;
    const int j = static_cast<int>(jk % ny), k = static_cast<int>(jk / ny);
    const double v = f[o];
    s2 = fma(v, v, s2);
    s1 += v;
    sv = fma(dxf[i] * dyf[j] * dzf[k], v, sv);
  }
  s2 = warp_sum(s2);
  s1 = warp_sum(s1);
  sv = warp_sum(sv);
  if (threadIdx.x % 32 == 0) {
    atomicAdd(&sums[0], s2);
    atomicAdd(&sums[1], s1);
    atomicAdd(&sums[2], sv);
  }
}

// Canonical gauge (reading R4): the volume-weighted mean of phi, summed
// with error-free additions (TwoSum) so that the mean is exact to a few ulps
// of the sum of |vol phi| whatever the cancellation, in two deterministic
// levels: block partial sums as (hi, lo) pairs, then one block over them.
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void pair_add_d(double& hi, double& lo, double h2, double l2) {
  double s, e;
  two_sum_d(hi, h2, s, e);
  hi = s;
  lo += e + l2;
}

__global__ void __launch_bounds__(256)
wsum_partial_fp64_kernel(int nx, int ny, int nz, const double* __restrict__ phi, const double* __restrict__ dxf,
                         const double* __restrict__ dyf, const double* __restrict__ dzf, double2* partial) {
  const long long lines = static_cast<long long>(ny) * nz;
  double hi = 0.0, lo = 0.0;
  for (long long L = blockIdx.x; L < lines; L += gridDim.x) {   // x-line (j, k) = L
    const int j = static_cast<int>(L % ny), k = static_cast<int>(L / ny);
    const double wyz = dyf[j] * dzf[k];
    const double* row = phi + static_cast<long long>(nx) * L;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = (dxf[i] * wyz) * row[i];
      double s, e;
      two_sum_d(hi, v, s, e);
      hi = s;
      lo += e;
    }
  }
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = hi;
  sh[1][threadIdx.x] = lo;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double h = sh[0][threadIdx.x], l = sh[1][threadIdx.x];
      pair_add_d(h, l, sh[0][threadIdx.x + w], sh[1][threadIdx.x + w]);
      sh[0][threadIdx.x] = h;
      sh[1][threadIdx.x] = l;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = make_double2(sh[0][0], sh[1][0]);
}

// mean = (sum of the partial pairs) / volume, one block
__global__ void __launch_bounds__(256)
wsum_final_fp64_kernel(int nb, const double2* __restrict__ partial, double inv_vol, double* mean) {
  double hi = 0.0, lo = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) pair_add_d(hi, lo, partial[b].x, partial[b].y);
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = hi;
  sh[1][threadIdx.x] = lo;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double h = sh[0][threadIdx.x], l = sh[1][threadIdx.x];
      pair_add_d(h, l, sh[0][threadIdx.x + w], sh[1][threadIdx.x + w]);
      sh[0][threadIdx.x] = h;
      sh[1][threadIdx.x] = l;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *mean = (sh[0][0] + sh[1][0]) * inv_vol;
}

__global__ void __launch_bounds__(256) sub_scalar_kernel(long long n, const double* __restrict__ c,
                                                          double* __restrict__ x) {
  const double v = *c;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride)
    x[i] -= v;
}

}  // namespace

namespace {
__global__ void __launch_bounds__(256) add_kernel(long long n, const double* __restrict__ in, double* __restrict__ out) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride)
    out[i] += in[i];
}
}  // namespace

cudaError_t add_fp64(long long n, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  note_launch(1);
  add_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(n, in, out);
  return cudaGetLastError();
}

cudaError_t remove_weighted_mean(const tpt_plan_s* p, double* phi, void* scratch, size_t scratch_bytes,
                                 double* mean, cudaStream_t s) {
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->dev);
  const long long lines = static_cast<long long>(p->n[1]) * p->n[2];
  long long cap = static_cast<long long>(scratch_bytes / sizeof(double2));
  if (cap > 4LL * dev_sms) cap = 4LL * dev_sms;
  if (cap < 1) return cudaErrorInvalidValue;
  const int nb = static_cast<int>(lines < cap ? lines : cap);
  double2* partial = static_cast<double2*>(scratch);
  note_launch(3);
  wsum_partial_fp64_kernel<<<nb, 256, 0, s>>>(p->n[0], p->n[1], p->n[2], phi, p->d_dxf[0], p->d_dxf[1],
                                              p->d_dxf[2], partial);
  wsum_final_fp64_kernel<<<1, 256, 0, s>>>(nb, partial, 1.0 / p->vol, mean);
  const long long n = static_cast<long long>(p->n[0]) * p->n[1] * p->n[2];
  long long g = (n + 255) / 256;
  if (g > 16LL * dev_sms) g = 16LL * dev_sms;
  sub_scalar_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(n, mean, phi);
  return cudaGetLastError();
}

cudaError_t field_sums(const tpt_plan_s* p, const double* f, double* sums, cudaStream_t s) {
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, p->dev);
  const long long n = static_cast<long long>(p->n[0]) * p->n[1] * p->n[2];
  long long nb = (n + 255) / 256;
  if (nb > 8LL * dev_sms) nb = 8LL * dev_sms;
  note_launch();
  field_sums_kernel<<<static_cast<unsigned>(nb), 256, 0, s>>>(p->n[0], p->n[1], p->n[2], f, p->d_dxf[0],
                                                              p->d_dxf[1], p->d_dxf[2], sums);
  return cudaGetLastError();
}

cudaError_t dgemm_cm(int M, int N, int K, const double* A, int lda, long long sA,
                     const double* B, int ldb, long long sB, double* C, int ldc, long long sC,
                     int batch, bool accumulate, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidConfiguration;
  // split N so that the grid's y extent stays within the hardware limit
  const int nchunk = 65535 * TN;
  for (int n0 = 0; n0 < N; n0 += nchunk) {
    const int nn = (N - n0 < nchunk) ? N - n0 : nchunk;
    dim3 grid((M + TM - 1) / TM, (nn + TN - 1) / TN, batch);
    note_launch();
    dgemm_cm_kernel<<<grid, dim3(TX, TY), 0, s>>>(M, nn, K, A, lda, sA,
                                                  B + static_cast<long long>(n0) * ldb, ldb, sB,
                                                  C + static_cast<long long>(n0) * ldc, ldc, sC,
                                                  accumulate ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t thomas_fp64(const tpt_plan_s* p, const double* fhat, double* phihat, double* scratch,
                        double* defect, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const long long lines = static_cast<long long>(nx) * ny;
  const int bs = 128;
  const long long nb = (lines + bs - 1) / bs;
  const double* rz = p->d_rows[2];
  // f-hat of the null line equals (g_x g_y) times the physical constant
  const double null_scale = p->singular ? 1.0 / (p->null_g[0] * p->null_g[1]) : 0.0;
  const size_t rows_bytes = 3 * static_cast<size_t>(nz) * sizeof(double);
  const bool rows = rows_bytes <= 48 * 1024;   // within the default dynamic limit
  note_launch();
  auto kern = rows ? thomas_fp64_kernel<true> : thomas_fp64_kernel<false>;
  kern<<<static_cast<unsigned>(nb), bs, rows ? rows_bytes : 0, s>>>(
      nx, ny, nz, fhat, phihat, scratch, p->ddir[0].lam, p->ddir[1].lam, rz, rz + nz, rz + 2 * nz,
      p->d_dxf[2], p->alpha, p->beta, p->singular ? p->null_i : -1, p->singular ? p->null_j : -1,
      null_scale, p->singular ? defect : nullptr);
  return cudaGetLastError();
}

cudaError_t residual_fp64(const tpt_plan_s* p, const double* f, const double* phi, double* r,
                          double* sums, const double* fshift, cudaStream_t s, bool all_sums) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  dim3 block(32, 4);
  dim3 grid((nx + 31) / 32, (ny + 3) / 4);
  const size_t rows_bytes = 3 * static_cast<size_t>(nz) * sizeof(double);
  const bool rows = rows_bytes <= 48 * 1024;   // within the default dynamic limit
  auto kern = rows ? (all_sums ? residual_fp64_kernel<true, true> : residual_fp64_kernel<true, false>)
                   : (all_sums ? residual_fp64_kernel<false, true> : residual_fp64_kernel<false, false>);
  note_launch();
  kern<<<grid, block, rows ? rows_bytes : 0, s>>>(nx, ny, nz, f, phi, r, p->d_rows[0], p->d_rows[1], p->d_rows[2],
                                                 p->d_dxf[0], p->d_dxf[1], p->d_dxf[2], p->alpha, p->beta,
                                                 fshift, sums);
  return cudaGetLastError();
}

}  // namespace tpt
