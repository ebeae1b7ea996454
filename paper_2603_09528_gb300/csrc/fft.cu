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
// memory, two real lines per complex array (as its real and imaginary parts):
// iterative radix-2 butterflies on bit-reversed input, one barrier per stage.  Line l of the field starts at (l % L1) * s1 + (l / L1) * s2 and has
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
  // tl lines (even) in tl / 2 complex slots: lines 2c and 2c + 1 of the block
  // are the real and imaginary parts of slot c, so one complex FFT of length N
  // transforms two real lines (forward), or two Hermitian spectra whose
  // transforms are real (inverse)
  extern __shared__ unsigned char smem_raw[];
  const int ts = tl / 2;
  R* re = reinterpret_cast<R*>(smem_raw);
  R* im = re + static_cast<size_t>(ts) * N;
  const long long l0 = static_cast<long long>(blockIdx.x) * tl;
  const int total = tl * N;
  const bool contiguous = (es == 1);
  auto base_of = [&](long long l) { return (l % L1) * s1 + (l / L1) * s2; };
  auto coords = [&](int e, int& line, int& t) {
    line = contiguous ? e / N : e % tl;
    t = contiguous ? e % N : e / tl;
  };

  if (!INV) {
    // ---- load real lines, place at bit-reversed positions of their part
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int line, t;
      coords(e, line, t);
      const long long l = l0 + line;
      const R x = l < nlines ? in[base_of(l) + t * es] : R(0);
      int pos = t;
      if (KIND == 1) pos = (t % 2 == 0) ? t / 2 : N - 1 - t / 2;   // v_n = x_2n, v_{N-1-n} = x_{2n+1}
      (line % 2 == 0 ? re : im)[static_cast<size_t>(line / 2) * N + bitrev(pos, logN)] = x;
    }
  } else {
    // ---- load both spectra of a slot, combine Z = V_a + i V_b
    const int tot2 = ts * N;
    for (int e = threadIdx.x; e < tot2; e += blockDim.x) {
      const int c = contiguous ? e / N : e % ts;
      const int k = contiguous ? e % N : e / ts;
      R vr[2], vi[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long l = l0 + 2 * c + h;
        R fr = R(0), fi = R(0);
        if (l < nlines) {
          const long long b = base_of(l);
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
        vr[h] = fr;
        vi[h] = fi;
      }
      const size_t o = static_cast<size_t>(c) * N + bitrev(k, logN);
      re[o] = vr[0] - vi[1];
      im[o] = vi[0] + vr[1];
    }
  }
  __syncthreads();

  // ---- radix-2 butterflies; forward uses e^{-2 pi i m / N}, inverse e^{+...}
  const int half = N / 2;
  for (int st = 0; st < logN; ++st) {
    const int h = 1 << st;
    const int tstep = N / (2 * h);
    for (int bfly = threadIdx.x; bfly < ts * half; bfly += blockDim.x) {
      const int slot = bfly / half, j = bfly % half;
      const int grp = j >> st, pos = j & (h - 1);
      const int i0 = slot * N + grp * 2 * h + pos, i1 = i0 + h;
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
    const R* zr = re + static_cast<size_t>(line / 2) * N;
    const R* zi = im + static_cast<size_t>(line / 2) * N;
    const int part = line % 2;
    R val;
    if (!INV) {
      // the transform of this line: (Z_k + conj Z_{N-k}) / 2, or (Z_k - conj Z_{N-k}) / 2i
      auto spec = [&](int k, R& xr, R& xi) {
        const int kn = (N - k) & (N - 1);
        if (part == 0) {
          xr = R(0.5) * (zr[k] + zr[kn]);
          xi = R(0.5) * (zi[k] - zi[kn]);
        } else {
          xr = R(0.5) * (zi[k] + zi[kn]);
          xi = R(0.5) * (zr[kn] - zr[k]);
        }
      };
      R xr, xi;
      if (KIND == 0) {
        if (t == 0) {
          spec(0, xr, xi);
          val = xr;
        } else if (t == N - 1) {
          spec(N / 2, xr, xi);
          val = xr;
        } else if (t % 2 == 1) {
          spec((t + 1) / 2, xr, xi);
          val = xr;
        } else {
          spec(t / 2, xr, xi);
          val = -xi;
        }
      } else {
        spec(t, xr, xi);
        val = xr * hc[t] + xi * hs[t];   // Re(e^{-i pi t / 2N} V_t)
      }
    } else {
      const R* z = part == 0 ? zr : zi;   // the real transform of this line
      if (KIND == 0) val = z[t] * invN;
      else val = z[(t % 2 == 0) ? t / 2 : N - 1 - t / 2] * invN;
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
  int tl = 8192 / N;                       // lines per block, two per complex slot
  tl = tl < 2 ? 2 : (tl > 64 ? 64 : tl);
  const size_t smem = 2 * static_cast<size_t>(tl / 2) * N * sizeof(R);
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
