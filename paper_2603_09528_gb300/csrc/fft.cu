// Fourier-based transforms of a uniform diagonalised direction (Sec. 2.2.1:
// on a uniform grid the eigenbasis projections are discrete trigonometric
// transforms evaluated with FFTs; Algorithm 1 steps 1, 3, 7, 9, "U Grid").
//
//   periodic  (real DFT):  forward  c_0 = sum f_i, c_{2k-1} = sum f_i cos(2 pi i k / N),
//                          c_{2k} = sum f_i sin(2 pi i k / N) (1 <= k < N/2),
//                          c_{N-1} = sum f_i (-1)^i; the inverse rebuilds f with 1/N.
//   Neumann   (DCT-II / DCT-III): forward X_k = sum x_i cos(pi k (2i + 1) / 2N), the
//                          inverse is its exact inverse; both through one complex FFT
//                          of length N with Makhoul's even/odd reordering.
//
// Mode p of the forward output is an eigenvector of the 1D operator with the
// plan's eigenvalue lam[p]; mode 0 is the constant (null) mode.  N is a power
// of two.  A block transforms `tl` lines held as complex arrays in shared
// memory: iterative radix-2 butterflies on bit-reversed input, one barrier per
// stage.  Line l of the field starts at (l % L1) * s1 + (l / L1) * s2 and has
// element stride es; lines with es > 1 are loaded across consecutive lines so
// that global accesses stay coalesced in both the x and the y direction.
#include <cuda_runtime.h>

#include "tpt_internal.h"

namespace tpt {
namespace {

__device__ __forceinline__ int bitrev(int v, int logn) {
  return logn == 0 ? 0 : static_cast<int>(__brev(static_cast<unsigned>(v)) >> (32 - logn));
}

template <typename R, int KIND, bool INV>
__global__ void __launch_bounds__(256)
fft_lines_kernel(int N, int logN, long long nlines, int tl, long long L1, long long s1, long long s2,
                 long long es, const R* __restrict__ in, R* __restrict__ out, int accumulate,
                 const R* __restrict__ twc, const R* __restrict__ tws, const R* __restrict__ hc,
                 const R* __restrict__ hs) {
  extern __shared__ unsigned char smem_raw[];
  R* re = reinterpret_cast<R*>(smem_raw);
  R* im = re + static_cast<size_t>(tl) * N;
  const long long l0 = static_cast<long long>(blockIdx.x) * tl;
  const int total = tl * N;
  const bool contiguous = (es == 1);
  auto base_of = [&](long long l) { return (l % L1) * s1 + (l / L1) * s2; };
  auto coords = [&](int e, int& line, int& t) {
    line = contiguous ? e / N : e % tl;
    t = contiguous ? e % N : e / tl;
  };

  // ---- load, pre-process, place at bit-reversed positions
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int line, t;
    coords(e, line, t);
    const long long l = l0 + line;
    const bool ok = l < nlines;
    const long long b = ok ? base_of(l) : 0;
    R fr = R(0), fi = R(0);
    int pos = t;
    if (!INV) {
      const R x = ok ? in[b + t * es] : R(0);
      fr = x;
      if (KIND == 1) pos = (t % 2 == 0) ? t / 2 : N - 1 - t / 2;   // v_n = x_2n, v_{N-1-n} = x_{2n+1}
    } else if (ok) {
      const int k = t;
      if (KIND == 0) {
        // F_0 = c_0, F_{N/2} = c_{N-1}, F_k = c_{2k-1} - i c_{2k}, F_{N-k} = conj(F_k)
        if (k == 0) {
          fr = in[b];
        } else if (2 * k == N) {
          fr = in[b + (N - 1) * es];
        } else if (2 * k < N) {
          fr = in[b + (2 * k - 1) * es];
          fi = -in[b + (2 * k) * es];
        } else {
          const int kk = N - k;
          fr = in[b + (2 * kk - 1) * es];
          fi = in[b + (2 * kk) * es];
        }
      } else {
        // V_k = e^{i pi k / 2N} (X_k - i X_{N-k}), X_N = 0
        const R xr = in[b + k * es];
        const R xi = (k == 0) ? R(0) : -in[b + (N - k) * es];
        fr = hc[k] * xr - hs[k] * xi;
        fi = hc[k] * xi + hs[k] * xr;
      }
    }
    re[static_cast<size_t>(line) * N + bitrev(pos, logN)] = fr;
    im[static_cast<size_t>(line) * N + bitrev(pos, logN)] = fi;
  }
  __syncthreads();

  // ---- radix-2 butterflies; forward uses e^{-2 pi i m / N}, inverse e^{+...}
  const int half = N / 2;
  for (int s = 0; s < logN; ++s) {
    const int h = 1 << s;
    const int tstep = N / (2 * h);
    for (int bfly = threadIdx.x; bfly < tl * half; bfly += blockDim.x) {
      const int line = bfly / half, j = bfly % half;
      const int grp = j >> s, pos = j & (h - 1);
      const int i0 = line * N + grp * 2 * h + pos, i1 = i0 + h;
      const R c = twc[pos * tstep], sn = tws[pos * tstep];
      const R vr = re[i1], vi = im[i1];
      const R tr = INV ? c * vr - sn * vi : c * vr + sn * vi;
      const R ti = INV ? c * vi + sn * vr : c * vi - sn * vr;
      const R ur = re[i0], ui = im[i0];
      re[i0] = ur + tr;
      im[i0] = ui + ti;
      re[i1] = ur - tr;
      im[i1] = ui - ti;
    }
    __syncthreads();
  }

  // ---- post-process and store
  const R invN = R(1) / static_cast<R>(N);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int line, t;
    coords(e, line, t);
    const long long l = l0 + line;
    if (l >= nlines) continue;
    const R* lr = re + static_cast<size_t>(line) * N;
    const R* li = im + static_cast<size_t>(line) * N;
    R val;
    if (!INV) {
      if (KIND == 0) {
        if (t == 0) val = lr[0];
        else if (t == N - 1) val = lr[N / 2];
        else if (t % 2 == 1) val = lr[(t + 1) / 2];
        else val = -li[t / 2];
      } else {
        val = lr[t] * hc[t] + li[t] * hs[t];   // Re(e^{-i pi t / 2N} V_t)
      }
    } else {
      if (KIND == 0) val = lr[t] * invN;
      else val = lr[(t % 2 == 0) ? t / 2 : N - 1 - t / 2] * invN;
    }
    const long long o = base_of(l) + t * es;
    out[o] = accumulate ? out[o] + val : val;
  }
}

template <typename R>
cudaError_t launch_fft(int kind, bool inverse, int N, long long nlines, long long L1, long long s1,
                       long long s2, long long es, const R* in, R* out, bool accumulate, const R* twc,
                       const R* tws, const R* hc, const R* hs, cudaStream_t s) {
  int logN = 0;
  while ((1 << logN) < N) ++logN;
  int tl = 4096 / N;
  tl = tl < 1 ? 1 : (tl > 32 ? 32 : tl);
  const size_t smem = 2 * static_cast<size_t>(tl) * N * sizeof(R);
  const long long blocks = (nlines + tl - 1) / tl;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int acc = accumulate ? 1 : 0;
  const unsigned g = static_cast<unsigned>(blocks);
  int dev = 0, cap = 48 * 1024;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    cap = 48 * 1024;
  }
#define TPT_FFT_LAUNCH(K, I)                                                                       \
  do {                                                                                             \
    auto kern = fft_lines_kernel<R, K, I>;                                                         \
    if (smem > 48 * 1024) {                                                                        \
      /* the device's cap, the same for every launch: a per-launch value could */                 \
      /* be lowered by another thread between setting it and launching */                        \
      if (static_cast<int>(smem) > cap) return cudaErrorInvalidConfiguration;                      \
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap); \
      if (e != cudaSuccess) return e;                                                              \
    }                                                                                              \
    note_launch(1);                                                                                \
    kern<<<g, 256, smem, s>>>(N, logN, nlines, tl, L1, s1, s2, es, in, out, acc, twc, tws, hc, hs); \
  } while (0)
  if (kind == 0 && !inverse) TPT_FFT_LAUNCH(0, false);
  else if (kind == 0) TPT_FFT_LAUNCH(0, true);
  else if (!inverse) TPT_FFT_LAUNCH(1, false);
  else TPT_FFT_LAUNCH(1, true);
#undef TPT_FFT_LAUNCH
  return cudaGetLastError();
}

}  // namespace

cudaError_t fft_fp64(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                     bool accumulate, cudaStream_t s) {
  const FftTables& t = p->fft[d];
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  if (d == 0) {
    const long long lines = static_cast<long long>(ny) * nz;
    return launch_fft<double>(t.kind, inverse, nx, lines, lines, nx, 0, 1, in, out, accumulate, t.twc,
                              t.tws, t.hc, t.hs, s);
  }
  const long long lines = static_cast<long long>(nx) * nz;
  return launch_fft<double>(t.kind, inverse, ny, lines, nx, 1, static_cast<long long>(nx) * ny, nx, in,
                            out, accumulate, t.twc, t.tws, t.hc, t.hs, s);
}

}  // namespace tpt
