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
// iterative radix-2 butterflies on bit-reversed input, one barrier per stage.
// The same kernel serves two precisions through its line-access policy: the
// float64 path's fields in the natural layout (any line stride), and the
// float32 transforms inside the mixed-precision corrections, which read the
// correction's operand formats and write the next stage's layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tc.h"
#include "tpt_internal.h"

namespace tpt {
namespace {

__device__ __forceinline__ int bitrev(int v, int logn) {
  return logn == 0 ? 0 : static_cast<int>(__brev(static_cast<unsigned>(v)) >> (32 - logn));
}

// ------------------------------------------------------------ line access
// The float64 kernel reads and writes its lines through an access policy IO: element
// t of input line l is at in_base(l) + t * in_step(), element t of output
// line l at out_base(l) + t * out_step() (the bases are computed once per
// line of a block and kept in shared memory), and
//   load(o)           the input element at offset o, as R;
//   store(o, v)       the output element at offset o (with the policy's
//                     format and accumulation);
//   stopped()         the solve this launch belongs to has stopped: return.
// Lines whose step is 1 are swept with t fastest across the threads of a
// block, the others with the line index fastest, so that global accesses
// stay coalesced either way.

// float64 field in the natural layout: line l starts at (l % L1) * s1 +
// (l / L1) * s2 with element stride es, in and out alike; out (+)= result.
struct StridedF64 {
  const double* in;
  double* out;
  long long L1, s1, s2, es;
  int accumulate;
  __device__ __forceinline__ long long in_base(long long l) const { return (l % L1) * s1 + (l / L1) * s2; }
  __device__ __forceinline__ long long out_base(long long l) const { return in_base(l); }
  __device__ __forceinline__ long long in_step() const { return es; }
  __device__ __forceinline__ long long out_step() const { return es; }
  __device__ __forceinline__ bool stopped() const { return false; }
  __device__ __forceinline__ double load(long long o) const { return in[o]; }
  __device__ __forceinline__ void store(long long o, double v) const { out[o] = accumulate ? out[o] + v : v; }
};

// Elements of one complex slot's part in shared memory: N plus one padding
// element per 128 bytes, rounded up to an odd count.
template <typename R>
__host__ __device__ __forceinline__ int slot_stride(int N) {
  const int s = N + N / (128 / static_cast<int>(sizeof(R)));
  return s | 1;
}

template <typename R, int KIND, bool INV, typename IO>
__global__ void __launch_bounds__(256)
fft_lines_kernel(int N, int logN, long long nlines, int tl, const IO io, const R* __restrict__ twc,
                 const R* __restrict__ tws, const R* __restrict__ hc, const R* __restrict__ hs) {
  // tl lines (even) in tl / 2 complex slots: lines 2c and 2c + 1 of the block
  // are the real and imaginary parts of slot c, so one complex FFT of length N
  // transforms two real lines (forward), or two Hermitian spectra whose
  // transforms are real (inverse)
  if (io.stopped()) return;
  extern __shared__ unsigned char smem_raw[];
  const int ts = tl / 2;
  // shared-memory layout: slot c at c * S, element i of a slot at i + i / P
  // (one padding element per 128 bytes) with S odd in elements: the
  // bit-reversed scatter, the butterflies of small span and the
  // line-by-line accesses of strided lines all spread over the banks
  constexpr int P = 128 / static_cast<int>(sizeof(R));
  const int S = slot_stride<R>(N);
  auto at = [&](int c, int i) { return c * S + i + i / P; };
  R* re = reinterpret_cast<R*>(smem_raw);
  R* im = re + static_cast<size_t>(ts) * S;
  // the block's line bases (tl <= 64) behind the two arrays
  long long* ibase = reinterpret_cast<long long*>(smem_raw + ((2 * static_cast<size_t>(ts) * S * sizeof(R) + 15) & ~15));
  long long* obase = ibase + 64;
  // twiddles cos, sin of 2 pi m / N (m < N/2) behind the line bases
  R* stc = reinterpret_cast<R*>(obase + 64);
  R* sts = stc + (N / 2 > 0 ? N / 2 : 1);
  for (int m = threadIdx.x; m < N / 2; m += blockDim.x) {
    stc[m] = twc[m];
    sts[m] = tws[m];
  }
  const long long l0 = static_cast<long long>(blockIdx.x) * tl;
  const int total = tl * N;
  const long long istep = io.in_step(), ostep = io.out_step();
  const bool icontig = istep == 1, ocontig = ostep == 1;
  for (int line = threadIdx.x; line < tl; line += blockDim.x) {
    const long long l = l0 + line < nlines ? l0 + line : 0;
    ibase[line] = io.in_base(l);
    obase[line] = io.out_base(l);
  }
  __syncthreads();

  if (!INV) {
    // ---- load real lines, place at bit-reversed positions of their part
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int line = icontig ? e / N : e % tl;
      const int t = icontig ? e % N : e / tl;
      const long long l = l0 + line;
      const R x = l < nlines ? io.load(ibase[line] + t * istep) : R(0);
      int pos = t;
      if (KIND == 1) pos = (t % 2 == 0) ? t / 2 : N - 1 - t / 2;   // v_n = x_2n, v_{N-1-n} = x_{2n+1}
      (line % 2 == 0 ? re : im)[at(line / 2, bitrev(pos, logN))] = x;
    }
  } else {
    // ---- load both spectra of a slot, combine Z = V_a + i V_b
    const int tot2 = ts * N;
    for (int e = threadIdx.x; e < tot2; e += blockDim.x) {
      const int c = icontig ? e / N : e % ts;
      const int k = icontig ? e % N : e / ts;
      R vr[2], vi[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long l = l0 + 2 * c + h;
        const long long b = ibase[2 * c + h];
        auto ld = [&](int t) { return io.load(b + t * istep); };
        R fr = R(0), fi = R(0);
        if (l < nlines) {
          if (KIND == 0) {
            // F_0 = c_0, F_{N/2} = c_{N-1}, F_k = c_{2k-1} - i c_{2k}, F_{N-k} = conj(F_k)
            if (k == 0) {
              fr = ld(0);
            } else if (2 * k == N) {
              fr = ld(N - 1);
            } else if (2 * k < N) {
              fr = ld(2 * k - 1);
              fi = -ld(2 * k);
            } else {
              const int kk = N - k;
              fr = ld(2 * kk - 1);
              fi = ld(2 * kk);
            }
          } else {
            // V_k = e^{i pi k / 2N} (X_k - i X_{N-k}), X_N = 0
            const R xr = ld(k);
            const R xi = (k == 0) ? R(0) : -ld(N - k);
            fr = hc[k] * xr - hs[k] * xi;
            fi = hc[k] * xi + hs[k] * xr;
          }
        }
        vr[h] = fr;
        vi[h] = fi;
      }
      const int o = at(c, bitrev(k, logN));
      re[o] = vr[0] - vi[1];
      im[o] = vi[0] + vr[1];
    }
  }
  __syncthreads();

  // ---- radix-2 butterflies; forward uses e^{-2 pi i m / N}, inverse e^{+...}
  const int half = N / 2;
  for (int st = 0; st < logN; ++st) {
    const int h = 1 << st;
    const int tsh = logN - 1 - st;   // twiddle index pos * N / (2h) as a shift
    for (int bfly = threadIdx.x; bfly < ts * half; bfly += blockDim.x) {
      const int slot = bfly >> (logN - 1), j = bfly & (half - 1);
      const int grp = j >> st, pos = j & (h - 1);
      const int i0 = at(slot, grp * 2 * h + pos), i1 = at(slot, grp * 2 * h + pos + h);
      const R c = stc[pos << tsh], sn = sts[pos << tsh];
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
    const int line = ocontig ? e / N : e % tl;
    const int t = ocontig ? e % N : e / tl;
    const long long l = l0 + line;
    if (l >= nlines) continue;
    const R* zr = re + at(line / 2, 0);
    const R* zi = im + at(line / 2, 0);
    auto pd = [&](int i) { return i + i / P; };   // padded offset inside the slot
    const int part = line % 2;
    R val;
    if (!INV) {
      // the transform of this line: (Z_k + conj Z_{N-k}) / 2, or (Z_k - conj Z_{N-k}) / 2i
      auto spec = [&](int k, R& xr, R& xi) {
        const int kn = (N - k) & (N - 1);
        if (part == 0) {
          xr = R(0.5) * (zr[pd(k)] + zr[pd(kn)]);
          xi = R(0.5) * (zi[pd(k)] - zi[pd(kn)]);
        } else {
          xr = R(0.5) * (zi[pd(k)] + zi[pd(kn)]);
          xi = R(0.5) * (zr[pd(kn)] - zr[pd(k)]);
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
      if (KIND == 0) val = z[pd(t)] * invN;
      else val = z[pd((t % 2 == 0) ? t / 2 : N - 1 - t / 2)] * invN;
    }
    io.store(obase[line] + t * ostep, val);
  }
}

int dev_smem_cap() {
  int dev = 0, cap = 48 * 1024;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    cap = 48 * 1024;
  }
  return cap;
}

// Launches fft_lines_kernel<R, KIND, INV, IO> over nlines lines of length N,
// `line_budget` / N lines per block (two per complex slot, 2 to 64).
template <typename R, int KIND, bool INV, typename IO>
cudaError_t launch_lines(int N, long long nlines, int line_budget, const IO& io, const R* twc, const R* tws,
                         const R* hc, const R* hs, cudaStream_t s) {
  int logN = 0;
  while ((1 << logN) < N) ++logN;
  int tl = line_budget / N;
  tl = tl < 2 ? 2 : (tl > 64 ? 64 : tl & ~1);
  const size_t smem = ((2 * static_cast<size_t>(tl / 2) * slot_stride<R>(N) * sizeof(R) + 15) & ~static_cast<size_t>(15)) +
                      2 * 64 * sizeof(long long) + 2 * static_cast<size_t>(N / 2 > 0 ? N / 2 : 1) * sizeof(R);
  const long long blocks = (nlines + tl - 1) / tl;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto kern = fft_lines_kernel<R, KIND, INV, IO>;
  if (smem > 48 * 1024) {
    // the device's cap, the same for every launch: a per-launch value could
    // be lowered by another thread between setting it and launching
    const int cap = dev_smem_cap();
    if (static_cast<int>(smem) > cap) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
  }
  note_launch(1);
  kern<<<static_cast<unsigned>(blocks), 256, smem, s>>>(N, logN, nlines, tl, io, twc, tws, hc, hs);
  return cudaGetLastError();
}

template <typename R, typename IO>
cudaError_t launch_kind(int kind, bool inverse, int N, long long nlines, int line_budget, const IO& io,
                        const R* twc, const R* tws, const R* hc, const R* hs, cudaStream_t s) {
  if (kind == 0 && !inverse) return launch_lines<R, 0, false>(N, nlines, line_budget, io, twc, tws, hc, hs, s);
  if (kind == 0) return launch_lines<R, 0, true>(N, nlines, line_budget, io, twc, tws, hc, hs, s);
  if (!inverse) return launch_lines<R, 1, false>(N, nlines, line_budget, io, twc, tws, hc, hs, s);
  return launch_lines<R, 1, true>(N, nlines, line_budget, io, twc, tws, hc, hs, s);
}

cudaError_t launch_fft_f64(int kind, bool inverse, int N, long long nlines, long long L1, long long s1,
                           long long s2, long long es, const double* in, double* out, bool accumulate,
                           const double* twc, const double* tws, const double* hc, const double* hs,
                           cudaStream_t s) {
  StridedF64 io;
  io.in = in;
  io.out = out;
  io.L1 = L1;
  io.s1 = s1;
  io.s2 = s2;
  io.es = es;
  io.accumulate = accumulate ? 1 : 0;
  return launch_kind<double>(kind, inverse, N, nlines, 8192, io, twc, tws, hc, hs, s);
}

// ------------------------------------------------- float32 (mixed path)
// Float32 transforms inside a mixed-precision correction.  Input rows are
// contiguous (line l at l * ldi) in the correction's operand format FMT and
// are read 16 bytes at a time; the output is one of
//   STAGE 0  forward, transposed (element t of line a + L1 * b at
//            b * ldo * N + t * ldo + a), operand format of FMT;
//   STAGE 1  forward, contiguous rows (l * ldo), float32;
//   STAGE 2  inverse, transposed, operand format of FMT;
//   STAGE 3  inverse, contiguous rows, the float-pair phi update (+)= or =.
// The two lines of a complex slot are finished by one thread: their values
// at the same t come from the same four spectrum entries, and in a
// transposed output they are neighbours (one paired store).  Inverse kernels
// first stage their input rows in shared memory (the spectra of a slot's two
// lines are read at mirrored positions k and N - k).
template <int FMT>
struct InVec;
template <>
struct InVec<kFmtSplit> {   // hi + lo planes of bf16
  static constexpr int V = 8;
  __device__ __forceinline__ static void load(const void* p0, const void* p1, long long o, float (&v)[V]) {
    const uint4 h = *reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(p0) + o);
    const uint4 l = *reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(p1) + o);
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[q]));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&lw[q]));
      v[2 * q] = a.x + b.x;
      v[2 * q + 1] = a.y + b.y;
    }
  }
};
template <>
struct InVec<kFmtBF16> {
  static constexpr int V = 8;
  __device__ __forceinline__ static void load(const void* p0, const void*, long long o, float (&v)[V]) {
    const uint4 h = *reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(p0) + o);
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[q]));
      v[2 * q] = a.x;
      v[2 * q + 1] = a.y;
    }
  }
};
template <>
struct InVec<kFmtF32> {
  static constexpr int V = 4;
  __device__ __forceinline__ static void load(const void* p0, const void*, long long o, float (&v)[V]) {
    const float4 h = *reinterpret_cast<const float4*>(static_cast<const float*>(p0) + o);
    v[0] = h.x;
    v[1] = h.y;
    v[2] = h.z;
    v[3] = h.w;
  }
};

// Values of lines (a, a + 1) at output offsets o0 and o1 in the operand
// format of FMT: one paired store when they are neighbours at an even
// offset, two single stores otherwise (b: line a + 1 exists).
template <int FMT>
__device__ __forceinline__ void store_two(void* out0, void* out1, long long o0, long long o1, bool b, float va,
                                          float vb) {
  const bool paired = b && o1 == o0 + 1 && (o0 & 1) == 0;
  if (FMT == kFmtF32) {
    float* q = static_cast<float*>(out0);
    if (paired) {
      *reinterpret_cast<float2*>(q + o0) = make_float2(va, vb);
    } else {
      q[o0] = va;
      if (b) q[o1] = vb;
    }
    return;
  }
  const __nv_bfloat16 ha = __float2bfloat16_rn(va), hb = __float2bfloat16_rn(vb);
  __nv_bfloat16* qh = static_cast<__nv_bfloat16*>(out0);
  __nv_bfloat16* ql = static_cast<__nv_bfloat16*>(out1);
  if (paired) {
    *reinterpret_cast<__nv_bfloat162*>(qh + o0) = __halves2bfloat162(ha, hb);
    if (FMT == kFmtSplit)
      *reinterpret_cast<__nv_bfloat162*>(ql + o0) = __halves2bfloat162(
          __float2bfloat16_rn(va - __bfloat162float(ha)), __float2bfloat16_rn(vb - __bfloat162float(hb)));
    return;
  }
  qh[o0] = ha;
  if (FMT == kFmtSplit) ql[o0] = __float2bfloat16_rn(va - __bfloat162float(ha));
  if (b) {
    qh[o1] = hb;
    if (FMT == kFmtSplit) ql[o1] = __float2bfloat16_rn(vb - __bfloat162float(hb));
  }
}

// (h, l) += v (exactly, Knuth's two-sum, then the lo parts), or = v
__device__ __forceinline__ void df_update(float& h, float& l, float v, bool acc) {
  if (!acc) {
    h = v;
    l = 0.0f;
    return;
  }
  const float s = h + v;
  const float bb = s - h;
  float e = (h - (s - bb)) + (v - bb);
  e += l;
  const float hi = s + e;
  l = e - (hi - s);
  h = hi;
}

// Elements of each padded twiddle table (cos, sin of 2 pi m / N, m < N/2).
__host__ __device__ __forceinline__ int tw_stride(int N) { return N / 2 + N / 64 + 1; }

// Byte offset of the output line bases in a mixed kernel's shared memory:
// behind the two slot arrays and the twiddles, 16-byte aligned.
__host__ __device__ __forceinline__ size_t mixed_obase_off(int ts, int N) {
  const size_t b = (2 * static_cast<size_t>(ts) * slot_stride<float>(N) + 2 * static_cast<size_t>(tw_stride(N))) *
                   sizeof(float);
  return (b + 15) & ~static_cast<size_t>(15);
}

struct MixedFftArgs {
  int N, logN, tl, lg_ts;   // tl = 2 ts lines per block, ts a power of two
  long long nlines;
  const void* in0;
  const void* in1;
  void* out0;
  void* out1;
  long long ldi, ldo, L1;
  int accumulate;
  const int* stop;
};

// R consecutive radix-2 DIT stages ST0 .. ST0 + R - 1 (span h = 2^s, forward
// twiddle e^{-2 pi i pos / 2h}, inverse e^{+...}) of every slot, in
// registers: the 2^R elements base + m 2^ST0 (m < 2^R; base = hi 2^(ST0+R)
// + lo, lo < 2^ST0) are closed under these stages, so a thread loads them
// once, applies the 2^(R-1) R butterflies in stage order and stores them
// back.  Each butterfly is the same operation as in a stage-by-stage sweep
// (a unit twiddle, which the first pass has for pos = 0, is applied as the
// exact product it is), so results do not depend on the grouping.  ST0 is a
// template parameter so that the padded shared-memory offsets of the 2^R
// elements are fixed offsets from the first (ST0 = 0: consecutive elements
// of one 32-element row; ST0 >= 5: whole rows apart).
template <int R, int ST0, bool INV>
__device__ __forceinline__ void fft_pass(float* re, float* im, const float* stc, const float* sts, int ts, int N,
                                         int logN, int S) {
  constexpr int G = 1 << R;
  static_assert(ST0 == 0 || ST0 == 3 || ST0 >= 5, "pass origins");
  const int per_slot = N >> R;
  const int items = ts * per_slot;
  // padded offset of element m relative to element 0 (ST0 == 3: 8 m plus one
  // padding element per four m, the row of element 0 starting at a multiple
  // of 64 plus lo < 8)
  auto moff = [](int m) {
    return ST0 == 0 ? m : (ST0 == 3 ? 8 * m + m / 4 : m * ((1 << ST0) + (1 << ST0) / 32));
  };
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int slot = it >> (logN - R), w = it & (per_slot - 1);
    const int lo = w & ((1 << ST0) - 1), hi = w >> ST0;
    const int base = (hi << (ST0 + R)) + lo;
    const int o0 = slot * S + base + base / 32;
    float xr[G], xi[G];
#pragma unroll
    for (int m = 0; m < G; ++m) {
      xr[m] = re[o0 + moff(m)];
      xi[m] = im[o0 + moff(m)];
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int hq = 1 << q;
      const int tsh = logN - 1 - (ST0 + q);   // twiddle index pos * N / 2h
      float cw[G / 2], sw[G / 2];
#pragma unroll
      for (int j = 0; j < G / 2; ++j) {
        if (j < hq) {
          const int tw = ((j << ST0) + lo) << tsh;
          cw[j] = stc[tw + tw / 32];   // padded like the slots (see fft_mixed_kernel)
          sw[j] = sts[tw + tw / 32];
        }
      }
#pragma unroll
      for (int m = 0; m < G; ++m) {
        if (m & hq) continue;
        const int j = m & (hq - 1);
        const float vr = xr[m + hq], vi = xi[m + hq];
        float tr, ti;
        if (ST0 == 0 && j == 0) {   // pos = 0: the twiddle is 1
          tr = vr;
          ti = vi;
        } else {
          const float c = cw[j], sn = sw[j];
          tr = INV ? c * vr - sn * vi : c * vr + sn * vi;
          ti = INV ? c * vi + sn * vr : c * vi - sn * vr;
        }
        const float ur = xr[m], ui = xi[m];
        xr[m] = ur + tr;
        xi[m] = ui + ti;
        xr[m + hq] = ur - tr;
        xi[m + hq] = ui - ti;
      }
    }
#pragma unroll
    for (int m = 0; m < G; ++m) {
      re[o0 + moff(m)] = xr[m];
      im[o0 + moff(m)] = xi[m];
    }
  }
}

// Passes of three stages from stage 0, the last one shorter (logN <= 12).
template <bool INV>
__device__ __forceinline__ void fft_passes(float* re, float* im, const float* stc, const float* sts, int ts, int N,
                                           int logN, int S) {
#define TPT_PASS(ST0)                                                                                    \
  if (logN > ST0) {                                                                                      \
    const int r = logN - ST0;                                                                            \
    if (r >= 3) fft_pass<3, ST0, INV>(re, im, stc, sts, ts, N, logN, S);                                 \
    else if (r == 2) fft_pass<2, ST0, INV>(re, im, stc, sts, ts, N, logN, S);                            \
    else fft_pass<1, ST0, INV>(re, im, stc, sts, ts, N, logN, S);                                        \
    __syncthreads();                                                                                     \
  }
  TPT_PASS(0)
  TPT_PASS(3)
  TPT_PASS(6)
  TPT_PASS(9)
#undef TPT_PASS
}

template <int KIND, int STAGE, int FMT>
__global__ void __launch_bounds__(256)
fft_mixed_kernel(const MixedFftArgs A, const float* __restrict__ twc, const float* __restrict__ tws,
                 const float* __restrict__ hc, const float* __restrict__ hs) {
  constexpr bool INV = STAGE >= 2;
  constexpr bool TRANS = STAGE == 0 || STAGE == 2;
  constexpr int V = InVec<FMT>::V;
  if (A.stop != nullptr && *A.stop != 0) return;   // the refinement has stopped
  extern __shared__ unsigned char smem_raw[];
  const int N = A.N, logN = A.logN, tl = A.tl, ts = tl / 2;
  constexpr int P = 32;
  const int S = slot_stride<float>(N);
  auto at = [&](int c, int i) { return c * S + i + i / P; };
  // shared memory: re | im (ts slots of S) | two padded twiddle tables |
  // output line bases (64) | staged input rows (inverse: tl rows of N + 4)
  float* re = reinterpret_cast<float*>(smem_raw);
  float* im = re + static_cast<size_t>(ts) * S;
  float* stc = im + static_cast<size_t>(ts) * S;
  float* sts = stc + tw_stride(N);
  long long* obase = reinterpret_cast<long long*>(smem_raw + mixed_obase_off(ts, N));
  const int SL = N + 4;
  float* stg = reinterpret_cast<float*>(obase + 64);
  const long long l0 = static_cast<long long>(blockIdx.x) * tl;
  for (int m = threadIdx.x; m < N / 2; m += blockDim.x) {
    // one padding element per 32: the passes read twiddles at strides of
    // 4 to 32 elements across a warp
    stc[m + m / 32] = twc[m];
    sts[m + m / 32] = tws[m];
  }
  for (int line = threadIdx.x; line < tl; line += blockDim.x) {
    const long long l = l0 + line < A.nlines ? l0 + line : 0;
    obase[line] = TRANS ? (l / A.L1) * A.ldo * N + (l % A.L1) : l * A.ldo;
  }

  // Thread mappings below keep what depends on a thread's position along the
  // line (t, k) in registers and walk the lines or slots: a slot is shared
  // by kper = min(N, 256) consecutive threads (by N / V of them when rows are
  // read V at a time), so each thread serves a fixed set of positions.

  // ---- input: rows read V elements at a time
  const int npv = N / V;
  if (npv <= 256) {
    const int t0 = (threadIdx.x % npv) * V;
    const int lstep = 256 / npv;
    int off[V];   // forward: padded bit-reversed position of each element in its slot
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const int t = t0 + q;
      const int pos = KIND == 1 ? ((t % 2 == 0) ? t / 2 : N - 1 - t / 2) : t;   // v_n = x_2n, v_{N-1-n} = x_{2n+1}
      const int br = bitrev(pos, logN);
      off[q] = br + br / P;
    }
    constexpr int U = 4;
    for (int line0 = threadIdx.x / npv; line0 < tl; line0 += U * lstep) {
      float v[U][V];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int line = line0 + u * lstep;
        const long long l = l0 + line;
        if (line < tl && l < A.nlines) {
          InVec<FMT>::load(A.in0, A.in1, l * A.ldi + t0, v[u]);
        } else {
#pragma unroll
          for (int q = 0; q < V; ++q) v[u][q] = 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int line = line0 + u * lstep;
        if (line >= tl) break;
        if (!INV) {
          float* part = ((line & 1) ? im : re) + (line >> 1) * S;
#pragma unroll
          for (int q = 0; q < V; ++q) part[off[q]] = v[u][q];
        } else {
          float* row = stg + static_cast<size_t>(line) * SL + t0;
#pragma unroll
          for (int q = 0; q < V; q += 4)
            *reinterpret_cast<float4*>(row + q) = make_float4(v[u][q], v[u][q + 1], v[u][q + 2], v[u][q + 3]);
        }
      }
    }
  } else {   // lines longer than 256 vectors: one vector at a time
    for (int g = threadIdx.x; g < tl * npv; g += blockDim.x) {
      const int line = g / npv, t0 = (g % npv) * V;
      const long long l = l0 + line;
      float v[V];
      if (l < A.nlines) {
        InVec<FMT>::load(A.in0, A.in1, l * A.ldi + t0, v);
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = 0.0f;
      }
      if (!INV) {
        float* part = (line & 1) ? im : re;
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int t = t0 + q;
          const int pos = KIND == 1 ? ((t % 2 == 0) ? t / 2 : N - 1 - t / 2) : t;
          part[at(line >> 1, bitrev(pos, logN))] = v[q];
        }
      } else {
        float* row = stg + static_cast<size_t>(line) * SL + t0;
#pragma unroll
        for (int q = 0; q < V; q += 4)
          *reinterpret_cast<float4*>(row + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  }
  __syncthreads();
  const int kper = N < 256 ? N : 256;
  const int c0 = threadIdx.x / kper, cstep = 256 / kper;
  if (INV) {
    // ---- both spectra of a slot, combined Z = V_a + i V_b at bit-reversed k
    for (int k = threadIdx.x % kper; k < N; k += kper) {
      const int o = bitrev(k, logN);
      const int ob = o + o / P;
      // where the spectrum at k comes from: DFT F_0 = c_0, F_{N/2} = c_{N-1},
      // F_k = c_{2k-1} - i c_{2k}, F_{N-k} = conj(F_k); DCT V_k = e^{i pi k / 2N}
      // (X_k - i X_{N-k}), X_N = 0
      int ir, ii;
      float sr = 1.0f, si = 0.0f, c = 1.0f, sn = 0.0f;
      if (KIND == 0) {
        const int kk = 2 * k <= N ? k : N - k;
        ir = kk == 0 ? 0 : (2 * kk == N ? N - 1 : 2 * kk - 1);
        ii = (kk == 0 || 2 * kk == N) ? -1 : 2 * kk;
        si = 2 * k < N ? -1.0f : 1.0f;
      } else {
        ir = k;
        ii = k == 0 ? -1 : N - k;
        si = -1.0f;
        c = hc[k];
        sn = hs[k];
      }
      for (int cc = c0; cc < ts; cc += cstep) {
        float vr[2], vi[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float* x = stg + static_cast<size_t>(2 * cc + h) * SL;
          const float xr = sr * x[ir];
          const float xi = ii >= 0 ? si * x[ii] : 0.0f;
          if (KIND == 0) {
            vr[h] = xr;
            vi[h] = xi;
          } else {
            vr[h] = c * xr - sn * xi;
            vi[h] = c * xi + sn * xr;
          }
        }
        re[cc * S + ob] = vr[0] - vi[1];
        im[cc * S + ob] = vi[0] + vr[1];
      }
    }
    __syncthreads();
  }

  // ---- radix-2 stages, three at a time in registers
  fft_passes<INV>(re, im, stc, sts, ts, N, logN, S);

  // ---- output: both lines of a slot per thread
  auto pd = [&](int i) { return i + i / P; };
  if (TRANS) {
    // slot-fastest (neighbouring lines of a row block next to each other)
    const int c = threadIdx.x & (ts - 1);
    const long long la = l0 + 2 * c;
    if (la < A.nlines) {
      const bool has_b = la + 1 < A.nlines;
      const long long oa0 = obase[2 * c], ob0 = obase[2 * c + 1];
      const float* zr = re + c * S;
      const float* zi = im + c * S;
      const float invN = 1.0f / static_cast<float>(N);
      for (int t = threadIdx.x >> A.lg_ts; t < N; t += 256 >> A.lg_ts) {
        float va, vb;
        if (!INV) {
          int k;
          if (KIND == 0) k = (t == 0) ? 0 : (t == N - 1 ? N / 2 : (t + 1) / 2);
          else k = t;
          const int kn = (N - k) & (N - 1);
          const float zrk = zr[pd(k)], zrn = zr[pd(kn)], zik = zi[pd(k)], zin = zi[pd(kn)];
          // spectra of the two lines: (Z_k + conj Z_{N-k}) / 2 and (Z_k - conj Z_{N-k}) / 2i
          const float ar = 0.5f * (zrk + zrn), ai = 0.5f * (zik - zin);
          const float br = 0.5f * (zik + zin), bi = 0.5f * (zrn - zrk);
          if (KIND == 0) {
            const bool imag = t != 0 && t != N - 1 && t % 2 == 0;
            va = imag ? -ai : ar;
            vb = imag ? -bi : br;
          } else {
            va = ar * hc[t] + ai * hs[t];   // Re(e^{-i pi t / 2N} V_t)
            vb = br * hc[t] + bi * hs[t];
          }
        } else {
          const int o = pd(KIND == 0 ? t : ((t % 2 == 0) ? t / 2 : N - 1 - t / 2));
          va = zr[o] * invN;
          vb = zi[o] * invN;
        }
        const long long tt = static_cast<long long>(t) * A.ldo;
        store_two<FMT>(A.out0, A.out1, oa0 + tt, ob0 + tt, has_b, va, vb);
      }
    }
  } else if (!INV) {
    // float32 rows: fixed positions t per thread, the slots in turn
    float* q = static_cast<float*>(A.out0);
    for (int t = threadIdx.x % kper; t < N; t += kper) {
      int k;
      if (KIND == 0) k = (t == 0) ? 0 : (t == N - 1 ? N / 2 : (t + 1) / 2);
      else k = t;
      const int pk = pd(k), pkn = pd((N - k) & (N - 1));
      const bool imag = KIND == 0 && t != 0 && t != N - 1 && t % 2 == 0;
      const float hct = KIND == 1 ? hc[t] : 0.0f, hst = KIND == 1 ? hs[t] : 0.0f;
      for (int c = c0; c < ts; c += cstep) {
        const long long la = l0 + 2 * c;
        if (la >= A.nlines) break;
        const float* zr = re + c * S;
        const float* zi = im + c * S;
        const float zrk = zr[pk], zrn = zr[pkn], zik = zi[pk], zin = zi[pkn];
        const float ar = 0.5f * (zrk + zrn), ai = 0.5f * (zik - zin);
        const float br = 0.5f * (zik + zin), bi = 0.5f * (zrn - zrk);
        float va, vb;
        if (KIND == 0) {
          va = imag ? -ai : ar;
          vb = imag ? -bi : br;
        } else {
          va = ar * hct + ai * hst;
          vb = br * hct + bi * hst;
        }
        q[obase[2 * c] + t] = va;
        if (la + 1 < A.nlines) q[obase[2 * c + 1] + t] = vb;
      }
    }
  } else {
    // the float-pair phi update: four consecutive points of both lines, fixed
    // positions per thread, the slots in turn
    float* ph = static_cast<float*>(A.out0);
    float* pl = static_cast<float*>(A.out1);
    const bool acc = A.accumulate != 0;
    const float invN = 1.0f / static_cast<float>(N);
    const int gper = N / 4 < 256 ? N / 4 : 256;
    const int g0 = threadIdx.x / gper, gstep = 256 / gper;
    for (int t0 = (threadIdx.x % gper) * 4; t0 < N; t0 += 4 * gper) {
      int so[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = t0 + q;
        so[q] = pd(KIND == 0 ? t : ((t % 2 == 0) ? t / 2 : N - 1 - t / 2));
      }
      for (int c = g0; c < ts; c += gstep) {
        const long long la = l0 + 2 * c;
        if (la >= A.nlines) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && la + 1 >= A.nlines) break;
          const float* z = (h == 0 ? re : im) + c * S;
          const long long o = obase[2 * c + h] + t0;
          float4 H = acc ? *reinterpret_cast<const float4*>(ph + o) : make_float4(0.f, 0.f, 0.f, 0.f);
          float4 L = acc ? *reinterpret_cast<const float4*>(pl + o) : make_float4(0.f, 0.f, 0.f, 0.f);
          df_update(H.x, L.x, z[so[0]] * invN, acc);
          df_update(H.y, L.y, z[so[1]] * invN, acc);
          df_update(H.z, L.z, z[so[2]] * invN, acc);
          df_update(H.w, L.w, z[so[3]] * invN, acc);
          *reinterpret_cast<float4*>(ph + o) = H;
          *reinterpret_cast<float4*>(pl + o) = L;
        }
      }
    }
  }
}

template <int KIND, int STAGE, int FMT>
cudaError_t launch_mixed_stage(const FftMixedArgs& a, cudaStream_t s) {
  MixedFftArgs A;
  A.N = a.N;
  int logN = 0;
  while ((1 << logN) < a.N) ++logN;
  A.logN = logN;
  // lines per block: 16384 (forward) / 8192 (inverse, which also stages its
  // input rows) elements, 2 to 64 lines, even
  int tl = (STAGE >= 2 ? 8192 : 16384) / a.N;
  tl = tl < 2 ? 2 : (tl > 64 ? 64 : tl & ~1);
  A.tl = tl;
  A.lg_ts = 0;
  while ((2 << A.lg_ts) < tl) ++A.lg_ts;
  A.nlines = a.nlines;
  A.in0 = a.in0;
  A.in1 = a.in1;
  A.out0 = a.out0;
  A.out1 = a.out1;
  A.ldi = a.ldi;
  A.ldo = a.ldo;
  A.L1 = a.L1 > 0 ? a.L1 : 1;
  A.accumulate = a.accumulate;
  A.stop = a.stop;
  const size_t smem = mixed_obase_off(tl / 2, a.N) + 64 * sizeof(long long) +
                      (STAGE >= 2 ? static_cast<size_t>(tl) * (a.N + 4) * sizeof(float) : 0);
  const long long blocks = (a.nlines + tl - 1) / tl;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto kern = fft_mixed_kernel<KIND, STAGE, FMT>;
  if (smem > 48 * 1024) {
    const int cap = dev_smem_cap();
    if (static_cast<int>(smem) > cap) return cudaErrorInvalidConfiguration;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
  }
  note_launch(1);
  kern<<<static_cast<unsigned>(blocks), 256, smem, s>>>(A, a.tw[0], a.tw[1], a.tw[2], a.tw[3]);
  return cudaGetLastError();
}

template <int STAGE, int FMT>
cudaError_t launch_mixed_kind(const FftMixedArgs& a, cudaStream_t s) {
  return a.kind == 0 ? launch_mixed_stage<0, STAGE, FMT>(a, s) : launch_mixed_stage<1, STAGE, FMT>(a, s);
}

template <int FMT>
cudaError_t launch_mixed_fmt(const FftMixedArgs& a, cudaStream_t s) {
  // the output each stage writes: transposed rows in the operand format,
  // float32 rows (forward) or the float-pair update (inverse)
  const int om = FMT == kFmtSplit ? tc::kOutSplitBF16 : (FMT == kFmtBF16 ? tc::kOutBF16 : tc::kOutF32);
  const bool tr = a.L1 > 0;
  if (tr && a.out_mode != om) return cudaErrorInvalidValue;
  if (!tr && a.out_mode != (a.inverse ? tc::kOutDF : tc::kOutF32)) return cudaErrorInvalidValue;
  if (!a.inverse) return tr ? launch_mixed_kind<0, FMT>(a, s) : launch_mixed_kind<1, FMT>(a, s);
  return tr ? launch_mixed_kind<2, FMT>(a, s) : launch_mixed_kind<3, FMT>(a, s);
}

}  // namespace

cudaError_t fft_fp64(const tpt_plan_s* p, int d, bool inverse, const double* in, double* out,
                     bool accumulate, cudaStream_t s) {
  const FftTables& t = p->fft[d];
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  if (d == 0) {
    const long long lines = static_cast<long long>(ny) * nz;
    return launch_fft_f64(t.kind, inverse, nx, lines, lines, nx, 0, 1, in, out, accumulate, t.twc, t.tws, t.hc,
                          t.hs, s);
  }
  const long long lines = static_cast<long long>(nx) * nz;
  return launch_fft_f64(t.kind, inverse, ny, lines, nx, 1, static_cast<long long>(nx) * ny, nx, in, out,
                        accumulate, t.twc, t.tws, t.hc, t.hs, s);
}

cudaError_t fft_mixed(const FftMixedArgs& a, cudaStream_t s) {
  // 16-byte row accesses: N >= 16, row strides of whole 16-byte units
  const int eb = a.in_fmt == kFmtF32 ? 4 : 2;
  if (a.N < 16 || a.N > 4096 || (a.N & (a.N - 1)) != 0 || a.nlines < 0 || (a.ldi * eb) % 16 != 0)
    return cudaErrorInvalidValue;
  if (a.L1 == 0 && a.inverse && a.ldo % 4 != 0) return cudaErrorInvalidValue;
  switch (a.in_fmt) {
    case kFmtSplit: return launch_mixed_fmt<kFmtSplit>(a, s);
    case kFmtBF16: return launch_mixed_fmt<kFmtBF16>(a, s);
    case kFmtF32: return launch_mixed_fmt<kFmtF32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tpt
