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

#include "cache.h"
#include "ptx.h"
#include "df.h"
#include "tc.h"
#include "tpt_internal.h"

namespace tpt {
namespace {

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

// acc += coef * (x - y) with float pairs; acc stays unnormalised (hi, lo)
__device__ __forceinline__ void acc_flux(df& acc, float ch, float cl, df x, df y) {
  df d = two_sum(x.hi, -y.hi);
  d.lo += x.lo - y.lo;
  const float pr = ch * d.hi;
  float pe = fmaf(ch, d.hi, -pr);
  pe = fmaf(ch, d.lo, pe);
  pe = fmaf(cl, d.hi, pe);
  const df t = two_sum(acc.hi, pr);
  acc.hi = t.hi;
  acc.lo += t.lo + pe;
}
// acc += coef * x
__device__ __forceinline__ void acc_mul(df& acc, float ch, float cl, df x) {
  const float pr = ch * x.hi;
  float pe = fmaf(ch, x.hi, -pr);
  pe = fmaf(ch, x.lo, pe);
  pe = fmaf(cl, x.hi, pe);
  const df t = two_sum(acc.hi, pr);
  acc.hi = t.hi;
  acc.lo += t.lo + pe;
}


// f (float64, (Nx,Ny,Nz)) -> f as float pair, R = f in operand format, and
// the sums sum f^2 (float), sum f and sum vol*f (float pairs) added to
// sums[0..2].  No float64 arithmetic per point.
template <int FMT>
__global__ void __launch_bounds__(256)
prepare_kernel(int nx, int ny, int nz, int ldx, int nbi, const double* __restrict__ f, float* __restrict__ fh,
               float* __restrict__ fl, void* r0, void* r1, const float* __restrict__ gx,
               const float* __restrict__ gy, const float* __restrict__ gz, double* sums) {
  // work item t covers x-line (j, k) = t / nbi, points (t % nbi) * 256 + 0..255;
  // one division per item (uniform over the block), none per element.
  // sum f^2 and sum f feed only the norm of f (float is enough); sum vol*f
  // fixes the compatibility constant and is kept as a float pair, with the
  // line weight dy_j dz_k applied once per item.
  const long long items = static_cast<long long>(nbi) * ny * nz;
  float s2 = 0.0f, s1f = 0.0f;
  df sv = {0.0f, 0.0f};
  constexpr int U = 4;   // items in flight per thread
  for (long long t0 = blockIdx.x; t0 < items; t0 += static_cast<long long>(U) * gridDim.x) {
    double v[U];
    long long line[U];
    int ii[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long t = t0 + static_cast<long long>(u) * gridDim.x;
      line[u] = t / nbi;
      ii[u] = static_cast<int>(t % nbi) * 256 + threadIdx.x;
      const bool ok = t < items && ii[u] < nx;
      if (!ok) ii[u] = -1;
      v[u] = ok ? f[ii[u] + static_cast<long long>(nx) * line[u]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = ii[u];
      if (i < 0) continue;
      const int j = static_cast<int>(line[u] % ny), k = static_cast<int>(line[u] / ny);
      const long long o = i + static_cast<long long>(nx) * line[u];
      const df d = split_double_int(v[u]);
      fh[o] = d.hi;
      fl[o] = d.lo;
      Elem<FMT>::store(r0, r1, i + static_cast<long long>(ldx) * line[u], d.hi + d.lo);
      s2 = fmaf(d.hi, d.hi, s2);
      s1f += d.hi;
      const df wline = df_mul({gy[j], gy[ny + j]}, {gz[k], gz[nz + k]});
      acc_mul(sv, wline.hi, wline.lo, df_mul({gx[i], gx[nx + i]}, d));
    }
  }
  df s1 = {s1f, 0.0f};
  sv = fast_two_sum(sv.hi, sv.lo);
  // block reduction in float pairs, one float64 atomic per block and sum
  __shared__ float red[3][2][8];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 = df_add(s1, {__shfl_xor_sync(0xffffffffu, s1.hi, o), __shfl_xor_sync(0xffffffffu, s1.lo, o)});
    sv = df_add(sv, {__shfl_xor_sync(0xffffffffu, sv.hi, o), __shfl_xor_sync(0xffffffffu, sv.lo, o)});
  }
  if (lane == 0) {
    red[0][0][w] = s2;
    red[1][0][w] = s1.hi;
    red[1][1][w] = s1.lo;
    red[2][0][w] = sv.hi;
    red[2][1][w] = sv.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < 8; ++q) {
      a += red[0][0][q];
      b += static_cast<double>(red[1][0][q]) + red[1][1][q];
      c += static_cast<double>(red[2][0][q]) + red[2][1][q];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
    atomicAdd(&sums[2], c);
  }
}

// ---------------------------------------------------------------- Thomas
// Tridiagonal solves along z (Algorithm 1 step 5) from T2 (float32, written by
// the y-forward GEMM) into T3 (the y-inverse GEMM operand format), by the
// partition method.  Line L = q + ldy p has its rows k at L + k ldy Nx, so
// for a fixed k all lines are contiguous; a tile is TLT consecutive lines
// times all rows.  The kernel is persistent (one CTA per SM): one thread
// claims tiles from a global counter and streams them into a ring of
// shared-memory input stages with 2D TMA loads (box TLT lines x up to 256
// rows, rows past Nz zero-filled) running ahead of the solve; the CTA solves
// a tile into an output tile that one thread stores with a TMA store.
// Claiming tiles dynamically lets a CTA that starts late (its SM busy with the
// null line) take fewer tiles.
//
// Per tile, warp s owns rows [sM, (s+1)M) of all TLT lines (lane l = line l),
// for s < nseg = ceil(Nz / M); further warps idle (identity rows of the
// reduced system).  Rows past Nz are identity rows (a = c = 0, diagonal 1,
// right side 0), folded into a per-row coefficient table in shared memory
// (beta a, beta b, beta c, and 1 or 0 for the modal shift).  The segment's
// last row is its interface unknown y_s.  One forward elimination over the
// interior rows, for the right side and for the coupling to y_{s-1}, gives
// with x_t = g_t + u_t y_{s-1} + v_t y_s the values the interface rows need
// (g, u of the last interior row, and g_0, u_0, v_0 of the first, accumulated
// during the sweep as sums with the running product of -c'_t, so no row is
// kept); the interface rows form a tridiagonal system in (y_0 .. y_{nseg-1})
// per line, solved by parallel cyclic reduction on nseg lanes; finally each
// segment is solved by Thomas with its two interface values as boundary
// values, the eliminated right side kept in place of the input.  Only the
// reciprocal pivots stay in registers.  float32 throughout.  The singular
// null line (q, p) = (0, 0) is taken by null_line_kernel (float64) on a
// second stream, which writes that line of T3 itself, so the tile holding it
// is stored with plain stores that skip it.  Lines with q >= Ny are padding:
// solved with a dummy shift and stored into the padding of T3, which no
// later step reads.
constexpr int kThomasThreads = 512;
constexpr int kThomasSmemBudget = 212 * 1024;   // dynamic shared memory of the kernel
constexpr int kThomasMaxStages = 8;

struct RowCoef {
  float a, b, c, m;   // beta a_k (0 at k = 0), beta b_k, beta c_k (0 from Nz - 1), shift factor
};

// Geometry of one launch (host and device): stage rows SR = nb * rb >= nseg * M.
struct ThomasGeom {
  int nseg, nb, rb, sr;
  int stages;
  int in_bytes, out_bytes, coef_bytes;   // one input stage, the output tile, the table
};

template <int FMT>
struct T3Fmt {
  static constexpr int NPL = (FMT == kFmtSplit) ? 2 : 1;
  static constexpr int EB = (FMT == kFmtF32) ? 4 : 2;
};

// Raw copy of element i of an output tile (planes s0, s1) to element j of T3.
template <int FMT>
__device__ __forceinline__ void copy_elem(const void* s0, const void* s1, int i, void* g0, void* g1, long long j) {
  if (FMT == kFmtF32) {
    static_cast<float*>(g0)[j] = static_cast<const float*>(s0)[i];
  } else {
    static_cast<uint16_t*>(g0)[j] = static_cast<const uint16_t*>(s0)[i];
    if (FMT == kFmtSplit) static_cast<uint16_t*>(g1)[j] = static_cast<const uint16_t*>(s1)[i];
  }
}

template <int FMT, int M, int TLT, int NT>
__global__ void __launch_bounds__(NT, kThomasThreads / NT)
thomas_tma_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_o0,
                  const __grid_constant__ CUtensorMap map_o1, ThomasGeom geo, int nx, int ny, int nz, int ldy,
                  int ntiles, int* next_tile, void* t3_0, void* t3_1, const float* __restrict__ lamx,
                  const float* __restrict__ lamy, const float* __restrict__ az, const float* __restrict__ bz,
                  const float* __restrict__ cz, float alpha, float beta, int singular, int* err,
                  const int* skip) {
  if (skip && *skip) return;   // the refinement has stopped
  using O = T3Fmt<FMT>;
  constexpr int NSEG = NT / TLT;   // segment slots per line (16 or 32)
  extern __shared__ __align__(128) uint8_t dsm_raw[];
  // 1024-byte aligned start, offset on the shared pointer itself so that every
  // access below stays a shared-memory (not generic) access
  uint8_t* dsm = dsm_raw + ((1024u - (ptx::smem_u32(dsm_raw) & 1023u)) & 1023u);
  RowCoef* coef = reinterpret_cast<RowCoef*>(dsm);
  uint8_t* in_base = dsm + geo.coef_bytes;
  uint8_t* ot = in_base + static_cast<size_t>(geo.stages) * geo.in_bytes;
  void* o0 = ot;
  void* o1 = ot + (O::NPL == 2 ? geo.out_bytes / 2 : 0);
  __shared__ float red[7 * NT];
  __shared__ __align__(8) uint64_t full[kThomasMaxStages];
  __shared__ int tile_of[kThomasMaxStages];   // tile loaded into each stage, -1: none left
  __shared__ int go;
  float* G0 = red;                       // [slot][TLT] g_0, u_0, v_0 of each segment
  float* U0 = G0 + NT;
  float* V0 = U0 + NT;
  float* RA = V0 + NT;                   // reduced rows
  float* RB = RA + NT;
  float* RC = RB + NT;
  float* RD = RC + NT;                   // right-hand side, then y
  const int tid = threadIdx.x;
  const int l = tid % TLT, s = tid / TLT;
  const int s0 = s * M;
  const bool active = s < geo.nseg;
  const int lines = ldy * nx;            // also the row stride of T2 / T3
  const int S = geo.stages;
  long long issued = 0;                  // (thread 0) local stages issued so far
  bool exhausted = false;                // (thread 0) the counter has run past ntiles
  int claim = -1;                        // (thread 0) next claimed tile, fetched a tile early

  auto issue = [&](long long i, int tile) {   // one thread: load claimed `tile` as local tile i
    const int st = static_cast<int>(i % S);
    const uint32_t bar = ptx::smem_u32(&full[st]);
    ++issued;
    if (tile >= ntiles) {                // none left: complete the phase without data
      exhausted = true;
      tile_of[st] = -1;
      ptx::mbar_arrive(bar);
      return;
    }
    tile_of[st] = tile;
    ptx::mbar_arrive_expect_tx(bar, static_cast<uint32_t>(geo.in_bytes));
    uint8_t* base = in_base + static_cast<size_t>(st) * geo.in_bytes;
    for (int b = 0; b < geo.nb; ++b)
      ptx::tma_load_2d(ptx::smem_u32(base + b * geo.rb * TLT * 4), &map_in, bar, tile * TLT, b * geo.rb);
  };

  for (int k = tid; k < geo.sr; k += blockDim.x) {
    RowCoef rc{0.0f, 1.0f, 0.0f, 0.0f};
    if (k < nz) {
      rc.a = k > 0 ? beta * az[k] : 0.0f;
      rc.b = beta * bz[k];
      rc.c = k < nz - 1 ? beta * cz[k] : 0.0f;
      rc.m = 1.0f;
    }
    coef[k] = rc;
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) ptx::mbar_init(ptx::smem_u32(&full[i]), 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&map_in);
    ptx::prefetch_tmap(&map_o0);
    if (O::NPL == 2) ptx::prefetch_tmap(&map_o1);
  }
  __syncthreads();
  if (tid == 0) {
    for (long long i = 0; i < S && !exhausted; ++i) issue(i, atomicAdd(next_tile, 1));
    if (!exhausted) claim = atomicAdd(next_tile, 1);   // its latency hides behind a tile
  }

  long long i = 0;
  bool ok = true;
  for (;; ++i) {
    const int st = static_cast<int>(i % S);
    const uint32_t bar = ptx::smem_u32(&full[st]);
    const uint32_t par = static_cast<uint32_t>((i / S) & 1);
    if (tid == 0) go = ptx::mbar_wait(bar, par, err, ptx::kErrWaitFull) ? 1 : 0;
    __syncthreads();
    if (!go) {
      ok = false;
      break;
    }
    const int tile = tile_of[st];
    if (tile < 0) break;
    for (int k = 0; k < 64 && !ptx::mbar_try_wait(bar, par); ++k) {
    }   // the phase is complete: this acquires the TMA writes for every thread
    float* in = reinterpret_cast<float*>(in_base + static_cast<size_t>(st) * geo.in_bytes);

    const int L = tile * TLT + l;
    int q = L % ldy, p = L / ldy;
    if (L >= lines || q >= ny) q = p = 0;        // padding line: dummy shift
    const float shift = alpha + beta * (lamx[p] + lamy[q]);
    const int o = s * TLT + l;

    // forward elimination of the interior rows t = 0 .. M-2 for the right
    // side (g) and the coupling to y_{s-1} (u); g_0, u_0 after the back
    // substitution are sum_t P_t g_t, sum_t P_t u_t with P_t = prod_{j<t} -c'_j
    float inv[M - 1];
    float cprev = 0.0f, gprev = 0.0f, uprev = 0.0f;
    if (active) {
      float P = 1.0f, Gs = 0.0f, Us = 0.0f;
#pragma unroll
      for (int t = 0; t < M - 1; ++t) {
        const RowCoef rc = coef[s0 + t];
        const float m = fmaf(-rc.a, cprev, fmaf(rc.m, shift, rc.b));
        const float iv = __fdividef(1.0f, m);
        const float d = in[(s0 + t) * TLT + l];
        inv[t] = iv;
        const float cp = rc.c * iv;
        const float g = fmaf(-rc.a, gprev, d) * iv;
        const float u = (t == 0 ? -rc.a : -rc.a * uprev) * iv;
        Gs = fmaf(P, g, Gs);
        Us = fmaf(P, u, Us);
        P *= -cp;
        cprev = cp;
        gprev = g;
        uprev = u;
      }
      G0[o] = Gs;
      U0[o] = Us;
      V0[o] = P;                         // v_0 = prod_t -c'_t
    } else {
      G0[o] = 0.0f;
      U0[o] = 0.0f;
      V0[o] = 0.0f;
    }
    __syncthreads();
    if (active) {
      const int k = s0 + M - 1;          // interface row of this segment
      const RowCoef rc = coef[k];
      const float dl = in[k * TLT + l];
      const float A = rc.a * uprev;
      float B = fmaf(-rc.a, cprev, fmaf(rc.m, shift, rc.b));
      float D = fmaf(-rc.a, gprev, dl);
      float Cc = 0.0f;
      if (s + 1 < NSEG) {
        const int on = o + TLT;
        B = fmaf(rc.c, U0[on], B);
        Cc = rc.c * V0[on];
        D = fmaf(-rc.c, G0[on], D);
      }
      RA[o] = A;
      RB[o] = B;
      RC[o] = Cc;
      RD[o] = D;
    } else {
      RA[o] = 0.0f;
      RB[o] = 1.0f;
      RC[o] = 0.0f;
      RD[o] = 0.0f;
    }
    __syncthreads();
    // Reduced system of every line by parallel cyclic reduction: NSEG lanes
    // per line (lane r holds interface row r), log2(NSEG) shuffle steps.
    {
      const int r = tid % NSEG, line = tid / NSEG;
      const int ix = r * TLT + line;
      float A = RA[ix], B = RB[ix], Cc = RC[ix], D = RD[ix];
#pragma unroll
      for (int dlt = 1; dlt < NSEG; dlt <<= 1) {
        const float Am = __shfl_up_sync(0xffffffffu, A, dlt, NSEG), Bm = __shfl_up_sync(0xffffffffu, B, dlt, NSEG);
        const float Cm = __shfl_up_sync(0xffffffffu, Cc, dlt, NSEG), Dm = __shfl_up_sync(0xffffffffu, D, dlt, NSEG);
        const float Ap = __shfl_down_sync(0xffffffffu, A, dlt, NSEG), Bp = __shfl_down_sync(0xffffffffu, B, dlt, NSEG);
        const float Cp = __shfl_down_sync(0xffffffffu, Cc, dlt, NSEG), Dp = __shfl_down_sync(0xffffffffu, D, dlt, NSEG);
        const bool hasm = r >= dlt, hasp = r + dlt < NSEG;
        const float k1 = hasm ? __fdividef(A, Bm) : 0.0f;
        const float k2 = hasp ? __fdividef(Cc, Bp) : 0.0f;
        const float nA = hasm ? -Am * k1 : 0.0f;
        const float nC = hasp ? -Cp * k2 : 0.0f;
        B = B - (hasm ? Cm * k1 : 0.0f) - (hasp ? Ap * k2 : 0.0f);
        D = D - (hasm ? Dm * k1 : 0.0f) - (hasp ? Dp * k2 : 0.0f);
        A = nA;
        Cc = nC;
      }
      RD[ix] = __fdividef(D, B);
    }
    if (tid == 0) {                      // the output tile of tile i-1 has been stored
      ptx::bulk_wait_read<0>();
    }
    __syncthreads();
    if (active) {
      // Thomas on the segment with boundary values y_{s-1} and y_s
      const float ys = RD[o];
      float gp = (s > 0) ? RD[o - TLT] : 0.0f;
#pragma unroll
      for (int t = 0; t < M - 1; ++t) {
        const int ix = (s0 + t) * TLT + l;
        gp = fmaf(-coef[s0 + t].a, gp, in[ix]) * inv[t];
        in[ix] = gp;
      }
      Elem<FMT>::store(o0, o1, (s0 + M - 1) * TLT + l, ys);
      float x = ys;
#pragma unroll
      for (int t = M - 2; t >= 0; --t) {
        const int ix = (s0 + t) * TLT + l;
        x = fmaf(-coef[s0 + t].c * inv[t], x, in[ix]);
        Elem<FMT>::store(o0, o1, ix, x);
      }
    }
    ptx::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && !exhausted) {        // the input stage is free: refill it
      issue(i + S, claim);
      if (!exhausted) claim = atomicAdd(next_tile, 1);
    }
    if (!(singular && tile == 0)) {
      if (tid == 0) {
        for (int b = 0; b < geo.nb; ++b) {
          const int off = b * geo.rb * TLT * O::EB;
          ptx::tma_store_2d(&map_o0, ptx::smem_u32(static_cast<uint8_t*>(o0) + off), tile * TLT, b * geo.rb);
          if (O::NPL == 2)
            ptx::tma_store_2d(&map_o1, ptx::smem_u32(static_cast<uint8_t*>(o1) + off), tile * TLT, b * geo.rb);
        }
        ptx::bulk_commit();
      }
    } else {                             // the null line is not ours to write
      for (int e = tid; e < TLT * nz; e += blockDim.x) {
        const int ll = e % TLT, k = e / TLT;
        if (ll == 0 || ll >= lines) continue;
        copy_elem<FMT>(o0, o1, e, t3_0, t3_1, ll + static_cast<long long>(k) * lines);
      }
      __syncthreads();                   // the output tile is rewritten by the next tile
    }
  }
  if (tid == 0) {
    if (!ok)   // the loads of local tiles i .. issued - 1 may still be landing
      for (long long k = i; k < issued; ++k)
        ptx::mbar_wait(ptx::smem_u32(&full[k % S]), static_cast<uint32_t>((k / S) & 1), err,
                       ptx::kErrWaitDrain);
    ptx::bulk_wait_all();
  }
}

// Two adjacent lines per thread (thomas2_kernel).  The same partition method
// as thomas_tma_kernel on the same tiles (32 consecutive lines x all rows,
// streamed by TMA, solved into an output tile stored by TMA), but each thread
// carries two neighbouring lines through its segment, so every recurrence of
// the sweeps runs as two independent dependency chains (the one-line kernel
// spends most cycles waiting on its single chain of reciprocals and shared
// loads), their inputs arrive as one 8-byte shared load and their outputs
// leave as packed pairs.  A line has up to 32 segments of M <= 16 rows
// (segment slot s = 2 * warp + lane / 16, lines 2 (lane % 16) and
// 2 (lane % 16) + 1); a half-warp reads one 128-byte row of the tile, so the
// 8-byte accesses are free of bank conflicts.  The reduced system has 32
// interface rows per line; warp w solves lines 2w and 2w + 1 by parallel
// cyclic reduction over all 32 lanes (lane r = interface row r), the rows
// kept in a shared buffer with a row pitch of 33 floats so that a warp's
// column reads are free of bank conflicts.  The second forward pass keeps its
// values in registers for the back substitution instead of rewriting the
// input tile.
constexpr int kT2Slots = 32;                    // segment slots per line
constexpr int kT2Pitch = kT2Slots + 1;          // row pitch of the reduced-system buffer
constexpr int kT2SmemBudget = 209 * 1024;       // dynamic shared memory (17.1 KB static beside it)

// Elements i and i + 1 (i even) of an output tile in the T3 format.
template <int FMT>
__device__ __forceinline__ void store_pair(void* o0, void* o1, int i, float x0, float x1) {
  if (FMT == kFmtF32) {
    *reinterpret_cast<float2*>(static_cast<float*>(o0) + i) = make_float2(x0, x1);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(o0) + i) = h;
    if (FMT == kFmtSplit) {
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(o1) + i) =
          __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    }
  }
}

// Paired float32 operations (sm_100 and later: __fadd2_rn, __fmul2_rn,
// __ffma2_rn apply two IEEE round-to-nearest operations in one instruction,
// component by component).  A subtraction is a fused multiply-add by -1
// (exact product, one rounding), so it rounds as a - b does.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_dup(float v) { return make_float2(v, v); }

// Row of thomas2_kernel's shared table with each coefficient duplicated for
// the thread's two lines: -beta a_k, beta b_k, beta c_k and the shift factor.
struct RowCoef2 {
  float2 na, b, c, m;
};

// The data of one instance for thomas2_kernel: tensor maps of T2 (in) and
// T3 (out planes), its stage geometry, sizes, tables and flags.  A grouped
// launch reads these from a device table (`first` = the instance's first
// tile in the launch); a single solve passes one as a kernel parameter.
struct ThomasJob {
  CUtensorMap map_in, map_o0, map_o1;
  ThomasGeom geo;
  int nx, ny, nz, ldy, ntiles, first;
  unsigned ldy_magic;   // L / ldy = (L * ldy_magic) >> ldy_shift for 0 <= L < 2^31
  int ldy_shift;
  void *t3_0, *t3_1;
  const float *lamx, *lamy, *az, *bz, *cz;
  float alpha, beta;
  int singular;
  int* err;
  const int* skip;
  // singular problems: the null line (q, p) = (0, 0) in float64 from T2
  // (element k at t2[k * nstride]) with the float64 z rows, the precomputed
  // factorisation of T_z (c', 1 / pivot), the z cell widths and beta
  const float* t2;
  const double *naz, *ncp, *ninvm, *ndz;
  double nbeta;
  long long nstride;
};

// The singular null line of a thomas2_kernel tile, solved in float64 by the
// whole block (one row per thread, Nz <= blockDim.x) into column 0 of the
// output tile: the line is projected to compatible form (dz-weighted mean
// removed), solved with the factorisation of T_z whose last pivot vanishes
// (the last modal unknown set to zero) and shifted to zero dz-weighted mean.
// Both sweeps are first-order linear recurrences, evaluated as block-wide
// scans of affine maps (warp shuffles, then the 16 warp totals in order).
// scr: 64 doubles of shared memory.  Every thread of the block calls it.
template <int FMT>
__device__ void null_line_block(const ThomasJob& J, void* o0, void* o1, double* scr) {
  constexpr int TLT = 32;
  const int k = threadIdx.x, lane = k % 32, warp = k / 32, nw = blockDim.x / 32;
  const int nz = J.nz;
  const bool row = k < nz, elim = k < nz - 1;
  const double f = row ? static_cast<double>(J.t2[static_cast<long long>(k) * J.nstride]) : 0.0;
  const double dzk = row ? J.ndz[k] : 0.0;
  // block sums, the same in every thread
  auto sum2 = [&](double a, double b, double& sa, double& sb) {
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (lane == 0) {
      scr[warp] = a;
      scr[32 + warp] = b;
    }
    __syncthreads();
    sa = 0.0;
    sb = 0.0;
    for (int v = 0; v < nw; ++v) {
      sa += scr[v];
      sb += scr[32 + v];
    }
    __syncthreads();
  };
  // x -> A x + B per row, composed in row order (up) or reverse row order;
  // returns this row's composed map applied to the value entering the line (0)
  auto scan = [&](double A, double B, bool up) -> double {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double Ap = up ? __shfl_up_sync(0xffffffffu, A, d) : __shfl_down_sync(0xffffffffu, A, d);
      const double Bp = up ? __shfl_up_sync(0xffffffffu, B, d) : __shfl_down_sync(0xffffffffu, B, d);
      if (up ? lane >= d : lane + d < 32) {
        B = fma(A, Bp, B);
        A *= Ap;
      }
    }
    if (lane == (up ? 31 : 0)) {         // the map of the whole warp
      scr[warp] = A;
      scr[32 + warp] = B;
    }
    __syncthreads();
    double v = 0.0;                      // the value entering this warp
    if (up) {
      for (int u = 0; u < warp; ++u) v = fma(scr[u], v, scr[32 + u]);
    } else {
      for (int u = nw - 1; u > warp; --u) v = fma(scr[u], v, scr[32 + u]);
    }
    __syncthreads();
    return fma(A, v, B);
  };
  double sf, w;
  sum2(dzk * f, dzk, sf, w);
  const double fshift = sf / w;
  // forward: dp_k = (f_k - fshift - a_k dp_{k-1}) / m_k, dp_{-1} = 0
  const double iv = elim ? J.ninvm[k] : 0.0;
  const double dp = scan(elim ? -J.naz[k] * iv : 1.0, elim ? (f - fshift) * iv : 0.0, true);
  // backward: x_k = dp_k - c'_k x_{k+1}, x_{nz-1} = 0
  const double x = scan(elim ? -J.ncp[k] : 1.0, elim ? dp : 0.0, false);
  double xs, w2;
  sum2(dzk * x, 0.0, xs, w2);
  if (row) Elem<FMT>::store(o0, o1, static_cast<long long>(k) * TLT, static_cast<float>((x - xs / w) / J.nbeta));
}

// lg: the shared-memory layout of the launch (stage count and the largest
// stage, output tile and row table over its instances).
template <int FMT, int M, int MULTI>
__global__ void __launch_bounds__(kThomasThreads, 1)
thomas2_kernel(const __grid_constant__ ThomasJob job0, ThomasGeom lg, int* next_tile, int total_tiles,
               const ThomasJob* __restrict__ jobs, int njobs) {
  if (!MULTI && job0.skip && *job0.skip) return;   // the refinement has stopped
  using O = T3Fmt<FMT>;
  constexpr int TLT = 32;
  static_assert(M >= 2 && M <= 16, "segments of 2 to 16 rows");
  extern __shared__ __align__(128) uint8_t dsm_raw[];
  uint8_t* dsm = dsm_raw + ((1024u - (ptx::smem_u32(dsm_raw) & 1023u)) & 1023u);
  RowCoef2* coef = reinterpret_cast<RowCoef2*>(dsm);
  uint8_t* in_base = dsm + lg.coef_bytes;
  uint8_t* ot = in_base + static_cast<size_t>(lg.stages) * lg.in_bytes;
  // reduced-system buffer: first g_0, u_0, v_0 of segment s in slot s, then
  // the interface row of segment s (A, B, C, D; D overwritten by the interface
  // value y_s) in slot s + 1.  The thread of segment s is the only reader of
  // slot s + 1 before it writes it, so no barrier separates the two uses.
  __shared__ __align__(16) float X[4][(kT2Slots + 1) * kT2Pitch];
  __shared__ __align__(8) uint64_t full[kThomasMaxStages];
  __shared__ int tile_of[kThomasMaxStages];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int s = 2 * warp + lane / 16;    // segment slot
  const int l0 = 2 * (lane % 16);        // first of the thread's two lines in the tile
  const int s0 = s * M;
  const int xo = s * kT2Pitch + l0;      // the thread's entries in X
  const int S = lg.stages;
  long long issued = 0;
  bool exhausted = false;
  int claim = -1;
  int cur = -1;                          // instance whose rows are in `coef`
  int* err0 = MULTI ? nullptr : job0.err;

  // instance of global tile t (its first tile <= t)
  auto job_of = [&](int t) -> const ThomasJob* {
    if constexpr (MULTI) {
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].first <= t) lo = mid;
        else hi = mid - 1;
      }
      return &jobs[lo];
    } else {
      (void)t;
      return &job0;
    }
  };
  // next tile from the counter, passing over the tiles of stopped instances
  auto next = [&]() -> int {
    for (;;) {
      const int t = atomicAdd(next_tile, 1);
      if (!MULTI || t >= total_tiles) return t;
      const ThomasJob& J = *job_of(t);
      if (!(J.skip && *J.skip)) return t;
    }
  };
  auto issue = [&](long long i, int tile) {
    const int st = static_cast<int>(i % S);
    const uint32_t bar = ptx::smem_u32(&full[st]);
    ++issued;
    if (tile >= total_tiles) {
      exhausted = true;
      tile_of[st] = -1;
      ptx::mbar_arrive(bar);
      return;
    }
    const ThomasJob& J = *job_of(tile);
    tile_of[st] = tile;
    ptx::mbar_arrive_expect_tx(bar, static_cast<uint32_t>(J.geo.in_bytes));
    uint8_t* base = in_base + static_cast<size_t>(st) * lg.in_bytes;
    const int lt = tile - J.first;
    for (int b = 0; b < J.geo.nb; ++b)
      ptx::tma_load_2d(ptx::smem_u32(base + b * J.geo.rb * TLT * 4), &J.map_in, bar, lt * TLT, b * J.geo.rb);
  };

  if (tid == 0) {
    for (int i = 0; i < S; ++i) ptx::mbar_init(ptx::smem_u32(&full[i]), 1);
    ptx::fence_mbar_init();
    if (!MULTI) {
      ptx::prefetch_tmap(&job0.map_in);
      ptx::prefetch_tmap(&job0.map_o0);
      if (O::NPL == 2) ptx::prefetch_tmap(&job0.map_o1);
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (long long i = 0; i < S && !exhausted; ++i) issue(i, next());
    if (!exhausted) claim = next();
  }
  __syncthreads();                       // tile_of of the first stages

  // Block barriers per tile: after the forward sweeps (which also agrees
  // whether every thread saw its stage land), after the interface rows, after
  // the reduced systems and after the output tile.  tile_of[st] is written by
  // thread 0 when it issues the stage, at least one tile (S >= 2 stages) and
  // so at least one barrier before it is read here.
  long long i = 0;
  bool ok = true;
  for (;; ++i) {
    const int st = static_cast<int>(i % S);
    const uint32_t bar = ptx::smem_u32(&full[st]);
    const uint32_t par = static_cast<uint32_t>((i / S) & 1);
    const int tile = tile_of[st];
    if (tile < 0) break;
    // every thread waits for the stage itself (bounded); a wait that runs out
    // is agreed on at the first barrier below
    const bool landed = ptx::mbar_wait(bar, par, nullptr, 0);
    const ThomasJob& J = *job_of(tile);
    const int jid = MULTI ? static_cast<int>(&J - jobs) : 0;
    if (jid != cur) {                    // this instance's beta-scaled z rows into the table
      if (cur >= 0) __syncthreads();     // the previous tile is done with them
      for (int k = tid; k < J.geo.sr; k += blockDim.x) {
        float a = 0.0f, b = 1.0f, c = 0.0f, m = 0.0f;   // padding rows: identity
        if (k < J.nz) {
          a = k > 0 ? J.beta * J.az[k] : 0.0f;
          b = J.beta * J.bz[k];
          c = k < J.nz - 1 ? J.beta * J.cz[k] : 0.0f;
          m = 1.0f;
        }
        coef[k] = {p_dup(-a), p_dup(b), p_dup(c), p_dup(m)};
      }
      cur = jid;
      __syncthreads();
    }
    const int lt = tile - J.first;
    const int lines = J.ldy * J.nx;
    const bool active = s < J.geo.nseg;
    void* o0 = ot;
    void* o1 = ot + (O::NPL == 2 ? J.geo.out_bytes / 2 : 0);
    float* in = reinterpret_cast<float*>(in_base + static_cast<size_t>(st) * lg.in_bytes);

    float shift[2];
    {
      // one division per tile: ldy is even and l0 is even, so the thread's
      // second line L + 1 lies in the same row p of modes as its first
      const int L = lt * TLT + l0;
      const int p = static_cast<int>((static_cast<unsigned long long>(L) * J.ldy_magic) >> J.ldy_shift);
      const int q = L - p * J.ldy;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool real = L + j < lines && q + j < J.ny;   // else a padding line: dummy shift
        shift[j] = J.alpha + J.beta * (J.lamx[real ? p : 0] + J.lamy[real ? q + j : 0]);
      }
    }
    // forward elimination of the interior rows (as in thomas_tma_kernel),
    // two lines at a time.  g (zero left boundary) replaces d in the input
    // stage; c' and the spike u (the response to a unit left boundary) stay in
    // registers, so that the final values are x_t = g_t + u_t y_{s-1} - c'_t x_{t+1}.
    // The two lines' operations run as paired instructions (float2 .x, .y).
    float2 ncpv[M - 1], uv[M - 1];       // -c' and u of rows 0 .. M - 2
    float2 cprev = make_float2(0.0f, 0.0f), gprev = cprev, uprev = cprev;
    const float2 sh = make_float2(shift[0], shift[1]);
    if (active) {
      float2 P = make_float2(1.0f, 1.0f), Gs = make_float2(0.0f, 0.0f), Us = Gs;
#pragma unroll
      for (int t = 0; t < M - 1; ++t) {
        const RowCoef2 rc = coef[s0 + t];
        const float2 d = *reinterpret_cast<const float2*>(in + (s0 + t) * TLT + l0);
        const float2 m = p_fma(rc.na, cprev, p_fma(rc.m, sh, rc.b));
        const float2 iv = make_float2(__fdividef(1.0f, m.x), __fdividef(1.0f, m.y));
        const float2 cp = p_mul(rc.c, iv);
        const float2 g = p_mul(p_fma(rc.na, gprev, d), iv);
        const float2 u = p_mul(t == 0 ? rc.na : p_mul(rc.na, uprev), iv);
        ncpv[t] = p_mul(cp, make_float2(-1.0f, -1.0f));
        uv[t] = u;
        Gs = p_fma(P, g, Gs);
        Us = p_fma(P, u, Us);
        P = p_mul(P, ncpv[t]);
        cprev = cp;
        gprev = g;
        uprev = u;
        *reinterpret_cast<float2*>(in + (s0 + t) * TLT + l0) = g;
      }
      X[0][xo] = Gs.x;
      X[0][xo + 1] = Gs.y;
      X[1][xo] = Us.x;
      X[1][xo + 1] = Us.y;
      X[2][xo] = P.x;
      X[2][xo + 1] = P.y;
    } else {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        X[0][xo + j] = 0.0f;
        X[1][xo + j] = 0.0f;
        X[2][xo + j] = 0.0f;
      }
    }
    if (__syncthreads_or(!landed)) {     // a stage did not land in time
      if (tid == 0 && J.err) atomicOr(J.err, ptx::kErrWaitFull);
      ok = false;
      break;
    }
    // interface row of the segment (its last row), coupled to the first row of
    // the next segment through g_0, u_0, v_0 of that segment (slot s + 1),
    // written over those in slot s + 1
    float ra[2] = {0.0f, 0.0f}, rb[2] = {1.0f, 1.0f}, rcc[2] = {0.0f, 0.0f}, rd[2] = {0.0f, 0.0f};
    if (active) {
      const int k = s0 + M - 1;
      const RowCoef2 rc = coef[k];
      const float a = -rc.na.x, b = rc.b.x, c = rc.c.x, mf = rc.m.x;
      const float2 d = *reinterpret_cast<const float2*>(in + k * TLT + l0);
      const float cpr[2] = {cprev.x, cprev.y}, gpr[2] = {gprev.x, gprev.y}, upr[2] = {uprev.x, uprev.y};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        ra[j] = a * upr[j];
        rb[j] = fmaf(-a, cpr[j], fmaf(mf, shift[j], b));
        rd[j] = fmaf(-a, gpr[j], j ? d.y : d.x);
        if (s + 1 < kT2Slots) {
          const int on = xo + kT2Pitch + j;
          rb[j] = fmaf(c, X[1][on], rb[j]);
          rcc[j] = c * X[2][on];
          rd[j] = fmaf(-c, X[0][on], rd[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      X[0][xo + kT2Pitch + j] = ra[j];
      X[1][xo + kT2Pitch + j] = rb[j];
      X[2][xo + kT2Pitch + j] = rcc[j];
      X[3][xo + kT2Pitch + j] = rd[j];
    }
    __syncthreads();
    // reduced systems: warp w takes lines 2w (lanes 0-15) and 2w + 1 (lanes
    // 16-31); lane q of a half holds interface rows 2q and 2q + 1, scaled to a
    // unit diagonal (a x_{r-1} + x_r + c x_{r+1} = d).  One odd-even step
    // eliminates the odd rows from the even ones (the odd row below comes from
    // lane q - 1), parallel cyclic reduction solves the 16 even rows, and each
    // odd row is then recovered from its two even neighbours.  Eliminating both
    // neighbours at distance d gives
    //   a' = -a a_{r-d},  c' = -c c_{r+d},  b' = 1 - a c_{r-d} - c a_{r+d},
    //   d' = d - a d_{r-d} - c d_{r+d},  then the row is scaled by 1 / b'.
    // Row 0 has a = 0 and row 31 has c = 0, and that stays so for every row
    // whose neighbour at distance d lies outside (its a or c is a product
    // with such a zero), so the shuffles that fall off an end of a half (which
    // return the lane's own values) are always multiplied by zero.
    {
      const int q = lane % 16;
      const int col = 2 * warp + lane / 16;
      const int ie = (2 * q + 1) * kT2Pitch + col, io = ie + kT2Pitch;   // rows 2q, 2q + 1
      float ae, ce, de, ao, co, dO;
      {
        const float ibe = __fdividef(1.0f, X[1][ie]), ibo = __fdividef(1.0f, X[1][io]);
        ae = X[0][ie] * ibe;
        ce = X[2][ie] * ibe;
        de = X[3][ie] * ibe;
        ao = X[0][io] * ibo;
        co = X[2][io] * ibo;
        dO = X[3][io] * ibo;
      }
      {
        // the odd row 2q - 1 (lane q - 1) and 2q + 1 (this lane)
        const float am = __shfl_up_sync(0xffffffffu, ao, 1, 16), cm = __shfl_up_sync(0xffffffffu, co, 1, 16);
        const float dm = __shfl_up_sync(0xffffffffu, dO, 1, 16);
        const float b = fmaf(-ae, cm, fmaf(-ce, ao, 1.0f));
        const float d = fmaf(-ae, dm, fmaf(-ce, dO, de));
        const float ib = __fdividef(1.0f, b);
        ae = -ae * am * ib;
        ce = -ce * co * ib;
        de = d * ib;
      }
#pragma unroll
      for (int dlt = 1; dlt < 16; dlt <<= 1) {
        const float Am = __shfl_up_sync(0xffffffffu, ae, dlt, 16), Cm = __shfl_up_sync(0xffffffffu, ce, dlt, 16);
        const float Dm = __shfl_up_sync(0xffffffffu, de, dlt, 16);
        const float Ap = __shfl_down_sync(0xffffffffu, ae, dlt, 16), Cp = __shfl_down_sync(0xffffffffu, ce, dlt, 16);
        const float Dp = __shfl_down_sync(0xffffffffu, de, dlt, 16);
        const float b = fmaf(-ae, Cm, fmaf(-ce, Ap, 1.0f));
        const float d = fmaf(-ae, Dm, fmaf(-ce, Dp, de));
        const float ib = __fdividef(1.0f, b);
        ae = -ae * Am * ib;
        ce = -ce * Cp * ib;
        de = d * ib;
      }
      // de = x_{2q}; the odd row from x_{2q} and x_{2q+2} (lane q + 1)
      const float xn = __shfl_down_sync(0xffffffffu, de, 1, 16);
      X[3][ie] = de;
      X[3][io] = fmaf(-ao, de, fmaf(-co, xn, dO));
    }
    if (tid == 0) ptx::bulk_wait_read<0>();   // the output tile of tile i-1 has been stored
    __syncthreads();
    if (active) {
      // back substitution on the segment with boundary values y_{s-1}, y_s
      float2 x = make_float2(X[3][xo + kT2Pitch], X[3][xo + kT2Pitch + 1]);
      const float2 yl = (s > 0) ? make_float2(X[3][xo], X[3][xo + 1]) : make_float2(0.0f, 0.0f);
      store_pair<FMT>(o0, o1, (s0 + M - 1) * TLT + l0, x.x, x.y);
#pragma unroll
      for (int t = M - 2; t >= 0; --t) {
        const float2 g = *reinterpret_cast<const float2*>(in + (s0 + t) * TLT + l0);
        x = p_fma(ncpv[t], x, p_fma(uv[t], yl, g));
        store_pair<FMT>(o0, o1, (s0 + t) * TLT + l0, x.x, x.y);
      }
    }
    if (J.singular && lt == 0) {         // the null line, in float64, over column 0
      __syncthreads();                   // every back substitution has read X
      null_line_block<FMT>(J, o0, o1, reinterpret_cast<double*>(&X[0][0]));
    }
    ptx::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && !exhausted) {        // the input stage is free: refill it
      issue(i + S, claim);
      if (!exhausted) claim = next();
    }
    if (tid == 0) {
      for (int b = 0; b < J.geo.nb; ++b) {
        const int off = b * J.geo.rb * TLT * O::EB;
        ptx::tma_store_2d(&J.map_o0, ptx::smem_u32(static_cast<uint8_t*>(o0) + off), lt * TLT, b * J.geo.rb);
        if (O::NPL == 2)
          ptx::tma_store_2d(&J.map_o1, ptx::smem_u32(static_cast<uint8_t*>(o1) + off), lt * TLT, b * J.geo.rb);
      }
      ptx::bulk_commit();
    }
  }
  if (tid == 0) {
    if (!ok)   // the loads of local tiles i .. issued - 1 may still be landing
      for (long long k = i; k < issued; ++k) {
        const int t = tile_of[k % S];
        int* e = MULTI ? (t >= 0 && t < total_tiles ? job_of(t)->err : nullptr) : err0;
        ptx::mbar_wait(ptx::smem_u32(&full[k % S]), static_cast<uint32_t>((k / S) & 1), e, ptx::kErrWaitDrain);
      }
    ptx::bulk_wait_all();
  }
}

// Singular null line (q, p) = (0, 0) in float64: the line of T2 is staged in
// shared memory, projected to compatible form (dz-weighted mean removed),
// solved with the plan's precomputed factorisation of T_z (last modal unknown
// set to zero) and shifted to zero dz-weighted mean; the result is written to
// the line of T3.  One warp; it touches no other line, so it runs beside
// thomas_tma_kernel on a second stream.
template <int FMT>
__device__ __forceinline__ void null_line_body(int nz, long long stride, const float* __restrict__ t2, void* t3_0,
                                               void* t3_1, const double* __restrict__ az,
                                               const double* __restrict__ ncp, const double* __restrict__ ninvm,
                                               const double* __restrict__ dz, double beta) {
  extern __shared__ double line[];
  const int lane = threadIdx.x;
  double s = 0.0, w = 0.0;
  for (int k = lane; k < nz; k += 32) {
    const double f = static_cast<double>(t2[static_cast<long long>(k) * stride]);
    line[k] = f;
    s = fma(dz[k], f, s);
    w += dz[k];
  }
  s = warp_sum_d(s);
  w = warp_sum_d(w);
  __syncwarp();
  // The two sweeps are first-order linear recurrences, run as scans: lane L
  // takes rows [k0, k1) of the nz - 1 eliminated rows, composes its rows'
  // affine maps, the warp scans the 32 maps (5 shuffle steps), and each lane
  // reruns its rows from its incoming value.
  const double fshift = s / w;
  const int n1 = nz - 1, chunk = (n1 + 31) / 32;
  const int k0 = min(lane * chunk, n1), k1 = min(k0 + chunk, n1);
  // forward: dp_k = (f_k - fshift - a_k dp_{k-1}) / m_k, dp_{-1} = 0
  double A = 1.0, B = 0.0;
  for (int k = k0; k < k1; ++k) {
    const double al = -az[k] * ninvm[k];
    B = fma(al, B, (line[k] - fshift) * ninvm[k]);
    A *= al;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {   // inclusive scan, lanes in row order
    const double Ap = __shfl_up_sync(0xffffffffu, A, d), Bp = __shfl_up_sync(0xffffffffu, B, d);
    if (lane >= d) {
      B = fma(A, Bp, B);
      A *= Ap;
    }
  }
  double dp = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) dp = 0.0;
  for (int k = k0; k < k1; ++k) {
    dp = fma(-az[k], dp, line[k] - fshift) * ninvm[k];
    line[k] = dp;
  }
  // backward: x_k = dp_k - c'_k x_{k+1}, x_{nz-1} = 0 (the vanishing pivot)
  A = 1.0;
  B = 0.0;
  for (int k = k1 - 1; k >= k0; --k) {
    const double g = -ncp[k];
    B = fma(g, B, line[k]);
    A *= g;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {   // inclusive scan, lanes in reverse row order
    const double Ap = __shfl_down_sync(0xffffffffu, A, d), Bp = __shfl_down_sync(0xffffffffu, B, d);
    if (lane + d < 32) {
      B = fma(A, Bp, B);
      A *= Ap;
    }
  }
  double x = __shfl_down_sync(0xffffffffu, B, 1);
  if (lane == 31) x = 0.0;
  for (int k = k1 - 1; k >= k0; --k) {
    x = fma(-ncp[k], x, line[k]);
    line[k] = x;
  }
  if (lane == 0) line[nz - 1] = 0.0;
  __syncwarp();
  double xs = 0.0;
  for (int k = lane; k < nz; k += 32) xs = fma(dz[k], line[k], xs);
  xs = warp_sum_d(xs);
  const double mean = xs / w;
  for (int k = lane; k < nz; k += 32)
    Elem<FMT>::store(t3_0, t3_1, static_cast<long long>(k) * stride, static_cast<float>((line[k] - mean) / beta));
}

template <int FMT>
__global__ void __launch_bounds__(32)
null_line_kernel(int nz, long long stride, const float* __restrict__ t2, void* t3_0, void* t3_1,
                 const double* __restrict__ az, const double* __restrict__ ncp,
                 const double* __restrict__ ninvm, const double* __restrict__ dz, double beta,
                 const int* skip) {
  if (skip && *skip) return;   // the refinement has stopped
  null_line_body<FMT>(nz, stride, t2, t3_0, t3_1, az, ncp, ninvm, dz, beta);
}

// ------------------------------------------------------------- residual
// beta-scaled float-pair rows of one direction: beta*a, beta*c and beta*w with
// w = -(a + b + c) the diagonal remainder of the float64 rows (zero except at
// Dirichlet walls), so that beta (a phi_- + b phi + c phi_+) =
// beta a (phi_- - phi) + beta c (phi_+ - phi) - beta w phi.
struct BRows {
  const float *ah, *al, *ch, *cl, *wh, *wl;
};

// r = (f - fshift) - alpha phi - beta L phi in float-pair arithmetic, written
// to R (operand format, rows of ldx), and sum r^2 -> sums[0]; fshift (the
// volume-weighted mean of f) only for a singular problem (SING).  Block (32, 4)
// over (i, j); blockIdx.z picks a segment of kseg planes that the thread
// marches through with pointer increments (neighbour offsets are fixed per
// thread; a neighbour past a non-periodic wall is the wrapped index and meets a
// zero coefficient).
template <int FMT, int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__global__ void __launch_bounds__(128)
residual_df_kernel(int nx, int ny, int nz, int ldx, int kseg, const float* __restrict__ fh,
                   const float* __restrict__ fl, const float* __restrict__ ph,
                   const float* __restrict__ pl, void* r0, void* r1, BRows RX, BRows RY, BRows RZ,
                   float alpha_h, float alpha_l, const double* __restrict__ fsums, double inv_vol,
                   double* sums, const int* skip) {
  if (skip && *skip) return;   // the refinement has stopped
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kseg;
  const int k1 = min(nz, k0 + kseg);
  float acc2 = 0.0f;
  if (i < nx && j < ny && k0 < nz) {
    const long long sz = static_cast<long long>(nx) * ny;
    const long long base = i + static_cast<long long>(nx) * j;
    const int dxm = (i == 0) ? nx - 1 : -1, dxp = (i == nx - 1) ? -(nx - 1) : 1;
    const int dym = (j == 0) ? (ny - 1) * nx : -nx, dyp = (j == ny - 1) ? -(ny - 1) * nx : nx;
    const float axh = RX.ah[i], axl = RX.al[i], cxh = RX.ch[i], cxl = RX.cl[i];
    const float ayh = RY.ah[j], ayl = RY.al[j], cyh = RY.ch[j], cyl = RY.cl[j];
    df fshift = {0.0f, 0.0f};
    if (SING) {
      const double c = fsums[2] * inv_vol;
      const float chi = static_cast<float>(c);
      fshift = {chi, static_cast<float>(c - static_cast<double>(chi))};
    }
    const float* hk = ph + base + sz * k0;
    const float* lk = pl + base + sz * k0;
    const float* fhk = fh + base + sz * k0;
    const float* flk = fl + base + sz * k0;
    const long long back = (k0 == 0) ? sz * (nz - 1) : -sz;
    df pm = {hk[back], lk[back]};
    df p0 = {hk[0], lk[0]};
    long long ro = i + static_cast<long long>(ldx) * (j + static_cast<long long>(ny) * k0);
    const long long rstep = static_cast<long long>(ldx) * ny;
    for (int k = k0; k < k1; ++k) {
      const long long fwd = (k == nz - 1) ? -sz * (nz - 1) : sz;
      const df pp = {hk[fwd], lk[fwd]};
      const df xm = {hk[dxm], lk[dxm]}, xp = {hk[dxp], lk[dxp]};
      const df ym = {hk[dym], lk[dym]}, yp = {hk[dyp], lk[dyp]};
      const df fv = {*fhk, *flk};
      // r starts as f (less the compatibility shift of a singular problem)
      // and each operator term is subtracted from it
      df acc = fv;
      if (SING) {
        acc = two_sum(fv.hi, -fshift.hi);
        acc.lo += fv.lo - fshift.lo;
      }
      acc_flux(acc, -axh, -axl, xm, p0);
      acc_flux(acc, -cxh, -cxl, xp, p0);
      acc_flux(acc, -ayh, -ayl, ym, p0);
      acc_flux(acc, -cyh, -cyl, yp, p0);
      acc_flux(acc, -RZ.ah[k], -RZ.al[k], pm, p0);
      acc_flux(acc, -RZ.ch[k], -RZ.cl[k], pp, p0);
      if (WX) acc_mul(acc, RX.wh[i], RX.wl[i], p0);
      if (WY) acc_mul(acc, RY.wh[j], RY.wl[j], p0);
      if (WZ) acc_mul(acc, RZ.wh[k], RZ.wl[k], p0);
      if (HAS_ALPHA) acc_mul(acc, -alpha_h, -alpha_l, p0);
      const float rv = acc.hi + acc.lo;
      Elem<FMT>::store(r0, r1, ro, rv);
      acc2 = fmaf(rv, rv, acc2);
      pm = p0;
      p0 = pp;
      hk += sz;
      lk += sz;
      fhk += sz;
      flk += sz;
      ro += rstep;
    }
  }
  double s2 = warp_sum_d(static_cast<double>(acc2));
  if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == 0) atomicAdd(&sums[0], s2);
}

// exact difference x - y of float pairs (hi parts by TwoSum, lo parts added)
__device__ __forceinline__ df df_diff(df x, df y) {
  df d = two_sum(x.hi, -y.hi);
  d.lo += x.lo - y.lo;
  return d;
}
// acc += coef * d with a float-pair coefficient and an exact pair difference d
__device__ __forceinline__ void acc_term(df& acc, float ch, float cl, df d) {
  const float pr = ch * d.hi;
  float pe = fmaf(ch, d.hi, -pr);
  pe = fmaf(ch, d.lo, pe);
  pe = fmaf(cl, d.hi, pe);
  const df t = two_sum(acc.hi, pr);
  acc.hi = t.hi;
  acc.lo += t.lo + pe;
}

template <int FMT>
struct Elem2;   // two consecutive elements of R in one store
template <>
struct Elem2<kFmtSplit> {
  static __device__ __forceinline__ void store(void* p0, void* p1, long long i, float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(p0) + i) = h;
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(p1) + i) = l;
  }
};
template <>
struct Elem2<kFmtBF16> {
  static __device__ __forceinline__ void store(void* p0, void*, long long i, float a, float b) {
    __nv_bfloat162 h;
    h.x = __float2bfloat16_rn(a);
    h.y = __float2bfloat16_rn(b);
    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(p0) + i) = h;
  }
};
template <>
struct Elem2<kFmtF32> {
  static __device__ __forceinline__ void store(void* p0, void*, long long i, float a, float b) {
    *reinterpret_cast<float2*>(static_cast<float*>(p0) + i) = make_float2(a, b);
  }
};

// Coefficients of the two points (i, i+1) of a thread that do not change
// along z: the x rows of both points, the y row, and the wall diagonals.
struct PairCoefs {
  float axh0, axl0, cxh0, cxl0, axh1, axl1, cxh1, cxl1;
  float ayh, ayl, cyh, cyl;
  float wxh0, wxl0, wxh1, wxl1, wyh, wyl;
};

template <int WX, int WY>
__device__ __forceinline__ PairCoefs pair_coefs(const BRows& RX, const BRows& RY, int i, int j) {
  PairCoefs c;
  c.axh0 = RX.ah[i];
  c.axl0 = RX.al[i];
  c.cxh0 = RX.ch[i];
  c.cxl0 = RX.cl[i];
  c.axh1 = RX.ah[i + 1];
  c.axl1 = RX.al[i + 1];
  c.cxh1 = RX.ch[i + 1];
  c.cxl1 = RX.cl[i + 1];
  c.ayh = RY.ah[j];
  c.ayl = RY.al[j];
  c.cyh = RY.ch[j];
  c.cyl = RY.cl[j];
  c.wxh0 = WX ? RX.wh[i] : 0.0f;
  c.wxl0 = WX ? RX.wl[i] : 0.0f;
  c.wxh1 = WX ? RX.wh[i + 1] : 0.0f;
  c.wxl1 = WX ? RX.wl[i + 1] : 0.0f;
  c.wyh = WY ? RY.wh[j] : 0.0f;
  c.wyl = WY ? RY.wl[j] : 0.0f;
  return c;
}

// z row of one plane: (a hi, a lo, c hi, c lo) and the wall diagonal
struct ZCoef {
  float ah, al, ch, cl, wh, wl;
};

// One plane of the residual of residual_df_kernel at the points a = (i, j, k)
// and b = (i+1, j, k), from their neighbours (float pairs): the face between
// a and b is differenced once, and dza / dzb hold the differences down from
// plane k (carried from plane k - 1) and leave holding those down from plane
// k + 1.  The operations applied to each point, and their order, are those
// of residual_df_kernel, so the results are the same to the bit.
template <int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__device__ __forceinline__ void residual_pair(const PairCoefs& c, const ZCoef& z, float alpha_h, float alpha_l,
                                              df fshift, df p0a, df p0b, df ppa, df ppb, df xm, df xp, df yma,
                                              df ymb, df ypa, df ypb, df fa, df fb, df& dza, df& dzb,
                                              float rv[2]) {
  const df dmid = df_diff(p0b, p0a);                          // across the face between the pair
  const df dupa = df_diff(ppa, p0a), dupb = df_diff(ppb, p0b);
  df acc_a = fa, acc_b = fb;
  if (SING) {
    acc_a = two_sum(fa.hi, -fshift.hi);
    acc_a.lo += fa.lo - fshift.lo;
    acc_b = two_sum(fb.hi, -fshift.hi);
    acc_b.lo += fb.lo - fshift.lo;
  }
  acc_term(acc_a, -c.axh0, -c.axl0, df_diff(xm, p0a));
  acc_term(acc_a, -c.cxh0, -c.cxl0, dmid);
  acc_term(acc_a, -c.ayh, -c.ayl, df_diff(yma, p0a));
  acc_term(acc_a, -c.cyh, -c.cyl, df_diff(ypa, p0a));
  acc_term(acc_a, -z.ah, -z.al, dza);
  acc_term(acc_a, -z.ch, -z.cl, dupa);
  acc_term(acc_b, -c.axh1, -c.axl1, {-dmid.hi, -dmid.lo});
  acc_term(acc_b, -c.cxh1, -c.cxl1, df_diff(xp, p0b));
  acc_term(acc_b, -c.ayh, -c.ayl, df_diff(ymb, p0b));
  acc_term(acc_b, -c.cyh, -c.cyl, df_diff(ypb, p0b));
  acc_term(acc_b, -z.ah, -z.al, dzb);
  acc_term(acc_b, -z.ch, -z.cl, dupb);
  if (WX) {
    acc_mul(acc_a, c.wxh0, c.wxl0, p0a);
    acc_mul(acc_b, c.wxh1, c.wxl1, p0b);
  }
  if (WY) {
    acc_mul(acc_a, c.wyh, c.wyl, p0a);
    acc_mul(acc_b, c.wyh, c.wyl, p0b);
  }
  if (WZ) {
    acc_mul(acc_a, z.wh, z.wl, p0a);
    acc_mul(acc_b, z.wh, z.wl, p0b);
  }
  if (HAS_ALPHA) {
    acc_mul(acc_a, -alpha_h, -alpha_l, p0a);
    acc_mul(acc_b, -alpha_h, -alpha_l, p0b);
  }
  rv[0] = acc_a.hi + acc_a.lo;
  rv[1] = acc_b.hi + acc_b.lo;
  dza = {-dupa.hi, -dupa.lo};                                 // down from plane k + 1
  dzb = {-dupb.hi, -dupb.lo};
}

__device__ __forceinline__ df fshift_of(const double* fsums, double inv_vol) {
  const double c = fsums[2] * inv_vol;
  const float chi = static_cast<float>(c);
  return {chi, static_cast<float>(c - static_cast<double>(chi))};
}

// The residual of residual_df_kernel for even Nx, two neighbouring points
// (i, i+1) per thread (residual_pair), marching through a segment of kseg
// planes with the loads of plane k + 1 issued before the arithmetic of plane
// k.  Used where the plane rows cannot be described by a tensor map.
template <int FMT, int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__global__ void __launch_bounds__(128, 5)
residual_df2_kernel(int nx, int ny, int nz, int ldx, int kseg, const float* __restrict__ fh,
                    const float* __restrict__ fl, const float* __restrict__ ph,
                    const float* __restrict__ pl, void* r0, void* r1, BRows RX, BRows RY, BRows RZ,
                    float alpha_h, float alpha_l, const double* __restrict__ fsums, double inv_vol,
                    double* sums, const int* skip) {
  if (skip && *skip) return;   // the refinement has stopped
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);   // points i and i + 1
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kseg;
  const int k1 = min(nz, k0 + kseg);
  float acc2 = 0.0f;
  if (i < nx && j < ny && k0 < nz) {
    const long long sz = static_cast<long long>(nx) * ny;
    const long long base = i + static_cast<long long>(nx) * j;
    const int dxm = (i == 0) ? nx - 1 : -1;                    // from point i
    const int dxp = (i + 1 == nx - 1) ? -(nx - 2) : 2;         // from point i (to i + 2 or the wrap)
    const int dym = (j == 0) ? (ny - 1) * nx : -nx, dyp = (j == ny - 1) ? -(ny - 1) * nx : nx;
    const PairCoefs c = pair_coefs<WX, WY>(RX, RY, i, j);
    const df fshift = SING ? fshift_of(fsums, inv_vol) : df{0.0f, 0.0f};
    const float* hk = ph + base + sz * k0;
    const float* lk = pl + base + sz * k0;
    const float* fhk = fh + base + sz * k0;
    const float* flk = fl + base + sz * k0;
    auto pair2 = [](const float* h, const float* l, df& a, df& b) {
      const float2 vh = *reinterpret_cast<const float2*>(h);
      const float2 vl = *reinterpret_cast<const float2*>(l);
      a = {vh.x, vl.x};
      b = {vh.y, vl.y};
    };
    const long long back = (k0 == 0) ? sz * (nz - 1) : -sz;
    df p0a, p0b, pma, pmb;
    pair2(hk, lk, p0a, p0b);
    pair2(hk + back, lk + back, pma, pmb);
    df dza = df_diff(pma, p0a), dzb = df_diff(pmb, p0b);        // down from plane k0
    long long ro = i + static_cast<long long>(ldx) * (j + static_cast<long long>(ny) * k0);
    const long long rstep = static_cast<long long>(ldx) * ny;
    struct Loads {
      float2 pph, ppl, ymh, yml, yph, ypl, fh, fl;
      float xmh, xml, xph, xpl;
      ZCoef z;
    };
    auto fetch = [&](int k, const float* h, const float* l, const float* f0, const float* f1, Loads& L) {
      const long long fwd = (k == nz - 1) ? -sz * (nz - 1) : sz;
      L.pph = *reinterpret_cast<const float2*>(h + fwd);
      L.ppl = *reinterpret_cast<const float2*>(l + fwd);
      L.ymh = *reinterpret_cast<const float2*>(h + dym);
      L.yml = *reinterpret_cast<const float2*>(l + dym);
      L.yph = *reinterpret_cast<const float2*>(h + dyp);
      L.ypl = *reinterpret_cast<const float2*>(l + dyp);
      L.fh = *reinterpret_cast<const float2*>(f0);
      L.fl = *reinterpret_cast<const float2*>(f1);
      L.xmh = h[dxm];
      L.xml = l[dxm];
      L.xph = h[dxp];
      L.xpl = l[dxp];
      L.z = {RZ.ah[k], RZ.al[k], RZ.ch[k], RZ.cl[k], WZ ? RZ.wh[k] : 0.0f, WZ ? RZ.wl[k] : 0.0f};
    };
    Loads nxt;
    fetch(k0, hk, lk, fhk, flk, nxt);
    for (int k = k0; k < k1; ++k) {
      const Loads L = nxt;
      if (k + 1 < k1) fetch(k + 1, hk + sz, lk + sz, fhk + sz, flk + sz, nxt);
      const df ppa = {L.pph.x, L.ppl.x}, ppb = {L.pph.y, L.ppl.y};
      float rv[2];
      residual_pair<HAS_ALPHA, WX, WY, WZ, SING>(c, L.z, alpha_h, alpha_l, fshift, p0a, p0b, ppa, ppb,
                                                 {L.xmh, L.xml}, {L.xph, L.xpl}, {L.ymh.x, L.yml.x},
                                                 {L.ymh.y, L.yml.y}, {L.yph.x, L.ypl.x}, {L.yph.y, L.ypl.y},
                                                 {L.fh.x, L.fl.x}, {L.fh.y, L.fl.y}, dza, dzb, rv);
      Elem2<FMT>::store(r0, r1, ro, rv[0], rv[1]);
      acc2 = fmaf(rv[0], rv[0], acc2);
      acc2 = fmaf(rv[1], rv[1], acc2);
      p0a = ppa;
      p0b = ppb;
      hk += sz;
      lk += sz;
      fhk += sz;
      flk += sz;
      ro += rstep;
    }
  }
  double s2 = warp_sum_d(static_cast<double>(acc2));
  if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == 0) atomicAdd(&sums[0], s2);
}

// ---------------------------------------------------------------------------
// Float pairs of two points side by side for the paired instructions (p_add
// and the rest, defined with the Thomas kernels): hi and lo parts as float2
// (.x point a, .y point b).  Every component goes through the operations of
// the scalar helpers above (two_sum, df_diff, acc_term) in the same order, so
// results are the same to the bit; negated operands are passed in
// precomputed.
struct dfx2 {
  float2 hi, lo;
};

// x - y of both points (df_diff): TwoSum of x.hi and -y.hi, whose error
// RN(-y.hi - bb) enters as -RN(y.hi + bb), then the lo parts
__device__ __forceinline__ dfx2 p_diff(const dfx2& x, const dfx2& y) {
  const float2 s = p_sub(x.hi, y.hi);
  const float2 bb = p_sub(s, x.hi);
  const float2 e = p_sub(p_sub(x.hi, p_sub(s, bb)), p_add(y.hi, bb));
  return {s, p_add(e, p_sub(x.lo, y.lo))};
}
// acc += (ch, cl) * d of both points (acc_term; acc_mul with d = x), given
// nch = -ch and ncl = -cl: the product's error chain runs negated
// (RN(pr - ch dh) = -RN(ch dh - pr), and so on) and is subtracted at the end
__device__ __forceinline__ void p_term(dfx2& acc, float2 ch, float2 nch, float2 ncl, const dfx2& d) {
  const float2 pr = p_mul(ch, d.hi);
  float2 ne = p_fma(nch, d.hi, pr);
  ne = p_fma(nch, d.lo, ne);
  ne = p_fma(ncl, d.hi, ne);
  const float2 s = p_add(acc.hi, pr);
  const float2 bb = p_sub(s, acc.hi);
  const float2 e = p_add(p_sub(acc.hi, p_sub(s, bb)), p_sub(pr, bb));
  acc.hi = s;
  acc.lo = p_add(acc.lo, p_sub(e, ne));
}

// Coefficients of two x or y terms of residual_pair_x2 (as applied to
// points a and b): the coefficient (ch), its negation (nch) and the negated
// lo part (ncl).  The x pair is term 1 (-x face of a; of b the face shared
// with a) and term 2 (the face shared with b for a; +x face of b), the y pair
// the -y and +y faces.  They live in shared memory (one x pair per lane, one y
// pair per row of the tile) and are read for every plane, which keeps the
// registers of the consumer threads within three blocks per SM.
struct TermCoefs2 {
  float2 ch0, ch1, nch0, nch1, ncl0, ncl1;
};
// rows d and d + off of one direction's float-pair rows (a at d, c at d + off)
__device__ __forceinline__ TermCoefs2 term_coefs2(const BRows& R, int d0, int d1) {
  // residual_pair's acc_term coefficients are the negated rows
  TermCoefs2 t;
  t.ch0 = make_float2(-R.ah[d0], -R.ah[d1]);
  t.ch1 = make_float2(-R.ch[d0], -R.ch[d1]);
  t.nch0 = make_float2(R.ah[d0], R.ah[d1]);
  t.nch1 = make_float2(R.ch[d0], R.ch[d1]);
  t.ncl0 = make_float2(R.al[d0], R.al[d1]);
  t.ncl1 = make_float2(R.cl[d0], R.cl[d1]);
  return t;
}
__device__ __forceinline__ TermCoefs2 lds_terms(const TermCoefs2* p) {
  TermCoefs2 t;
  const uint32_t a = ptx::smem_u32(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(t.ch0.x), "=f"(t.ch0.y), "=f"(t.ch1.x), "=f"(t.ch1.y) : "r"(a));
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4 + 16];"
               : "=f"(t.nch0.x), "=f"(t.nch0.y), "=f"(t.nch1.x), "=f"(t.nch1.y) : "r"(a));
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4 + 32];"
               : "=f"(t.ncl0.x), "=f"(t.ncl0.y), "=f"(t.ncl1.x), "=f"(t.ncl1.y) : "r"(a));
  return t;
}
// wall diagonals of the pair (Dirichlet walls only)
struct WallCoefs2 {
  float2 wxh, nwxh, nwxl, wyh, nwyh, nwyl;
};
template <int WX, int WY>
__device__ __forceinline__ WallCoefs2 wall_coefs2(const BRows& RX, const BRows& RY, int i, int j) {
  WallCoefs2 c;
  const float wx0 = WX ? RX.wh[i] : 0.0f, wx1 = WX ? RX.wh[i + 1] : 0.0f;
  const float wl0 = WX ? RX.wl[i] : 0.0f, wl1 = WX ? RX.wl[i + 1] : 0.0f;
  c.wxh = make_float2(wx0, wx1);
  c.nwxh = make_float2(-wx0, -wx1);
  c.nwxl = make_float2(-wl0, -wl1);
  const float wy = WY ? RY.wh[j] : 0.0f, wyl = WY ? RY.wl[j] : 0.0f;
  c.wyh = p_dup(wy);
  c.nwyh = p_dup(-wy);
  c.nwyl = p_dup(-wyl);
  return c;
}

// z coefficients of one plane for residual_pair_x2, duplicated for the two
// points: term 5 (the face below, applied to -dz with the row's own sign),
// term 6 (the face above, negated row), the wall diagonal
struct ZCoef2 {
  float2 ch5, nch5, ncl5, ch6, nch6, ncl6, wh, nwh, nwl;
};
__device__ __forceinline__ ZCoef2 zcoef2(float ah, float al, float ch, float cl, float wh, float wl) {
  return {p_dup(ah), p_dup(-ah), p_dup(-al), p_dup(-ch), p_dup(ch), p_dup(cl), p_dup(wh), p_dup(-wh), p_dup(-wl)};
}

// residual_pair with paired instructions: P0 = (phi_a, phi_b), PP the plane
// above, XO = (phi_{i-1}, phi_{i+2}), YM / YP the -y / +y
// neighbours, F = (f_a, f_b), FS the duplicated fshift.  du holds on entry
// phi(k) - phi(k-1) (the negated face difference below) and leaves holding
// phi(k+1) - phi(k).  Term by term the operations are residual_pair's: the
// -dmid of point b is the difference p0a - p0b, the z difference below enters
// with the opposite sign and the row's own sign (the same products).
template <int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__device__ __forceinline__ float2 residual_pair_x2(const TermCoefs2& cx, const TermCoefs2& cy,
                                                   const WallCoefs2& c, const ZCoef2& z, float2 ach,
                                                   float2 anch, float2 ancl, const dfx2& FS,
                                                   const dfx2& P0, const dfx2& PP, const dfx2& XO,
                                                   const dfx2& YM, const dfx2& YP, const dfx2& F, dfx2& du) {
  const dfx2 dup = p_diff(PP, P0);
  dfx2 acc = SING ? p_diff(F, FS) : F;
  // x faces: the -x faces of a and b in one paired difference; the +x face of
  // a is the negated -x face of b (what differencing it again would give, to
  // the bit), so only b's +x face is differenced on its own
  const dfx2 dl = p_diff(dfx2{make_float2(XO.hi.x, P0.hi.x), make_float2(XO.lo.x, P0.lo.x)}, P0);
  p_term(acc, cx.ch0, cx.nch0, cx.ncl0, dl);
  const df db = df_diff(df{XO.hi.y, XO.lo.y}, df{P0.hi.y, P0.lo.y});   // phi_{i+2} - phi_b
  p_term(acc, cx.ch1, cx.nch1, cx.ncl1,
         dfx2{make_float2(-dl.hi.y, db.hi), make_float2(-dl.lo.y, db.lo)});
  p_term(acc, cy.ch0, cy.nch0, cy.ncl0, p_diff(YM, P0));
  p_term(acc, cy.ch1, cy.nch1, cy.ncl1, p_diff(YP, P0));
  p_term(acc, z.ch5, z.nch5, z.ncl5, du);
  p_term(acc, z.ch6, z.nch6, z.ncl6, dup);
  if (WX) p_term(acc, c.wxh, c.nwxh, c.nwxl, P0);
  if (WY) p_term(acc, c.wyh, c.nwyh, c.nwyl, P0);
  if (WZ) p_term(acc, z.wh, z.nwh, z.nwl, P0);
  if (HAS_ALPHA) p_term(acc, ach, anch, ancl, P0);   // (-alpha_h, -alpha_l) * phi
  du = dup;
  return p_add(acc.hi, acc.lo);
}

// ---------------------------------------------------------------------------
// TMA-staged residual.  A block owns a tile of kResTX x kResTY points of the
// (x, y) plane and a segment of up to kResKseg planes; a producer warp
// streams, plane by plane, the phi pair with a halo (x from i0 - 4 to
// i0 + kResTX + 4, rows j0 - 1 to j0 + kResTY) and the f pair of the tile into
// a ring of shared-memory stages.  The tensor maps are 2D over the rows
// (j + Ny k) of the field, so a halo row past a tile's y edge is a row of the
// neighbouring plane, or outside the tensor and zero; either meets a zero
// coefficient unless the direction is periodic, where the edge points load
// the wrapped neighbour directly.  Each consumer warp takes one row of the
// tile, two points per lane, and applies residual_pair, so the results equal
// residual_df2_kernel's.
constexpr int kResTX = 64, kResTY = 8, kResStages = 6, kResKseg = 64;
constexpr int kResPW = kResTX + 8;                         // phi row: 4 halo columns each side
constexpr int kResPBytes = ((kResPW * (kResTY + 2) * 4 + 127) / 128) * 128;
constexpr int kResFBytes = kResTX * kResTY * 4;
constexpr int kResStage = 2 * kResPBytes + 2 * kResFBytes;
constexpr int kResZBytes = kResKseg * static_cast<int>(sizeof(ZCoef2));
constexpr int kResCBytes = (32 + kResTY) * static_cast<int>(sizeof(TermCoefs2));   // x per lane, y per row
constexpr int kResSmem = kResStages * kResStage + 2 * kResStages * 8 + kResZBytes + kResCBytes + 128;
constexpr int kResThreads = 32 * (kResTY + 1);

// The residual of one instance for residual_tma_kernel: tensor maps of the
// phi pair (with halo boxes) and of the f pair, sizes, rows and outputs.  A
// grouped launch reads these from a device table, its block b taking tile
// b - first of instance `job` (tiles x fastest, then y, then z segments).
struct ResJob {
  CUtensorMap tPH, tPL, tFH, tFL;
  int nx, ny, nz, ldx, px, py;
  const float *ph, *pl;
  void *r0, *r1;
  BRows RX, RY, RZ;
  float alpha_h, alpha_l;
  const double* fsums;
  double inv_vol;
  double* sums;
  int* err;
  const int* skip;
  int first, tx, ty, tz;   // first block and tile counts of the instance
};

template <int FMT, int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__device__ __forceinline__ void residual_tma_body(const ResJob& J, int bx, int by, int bz) {
  const CUtensorMap& tPH = J.tPH;
  const CUtensorMap& tPL = J.tPL;
  const CUtensorMap& tFH = J.tFH;
  const CUtensorMap& tFL = J.tFL;
  const int nx = J.nx, ny = J.ny, nz = J.nz, ldx = J.ldx, px = J.px, py = J.py;
  const float* __restrict__ ph = J.ph;
  const float* __restrict__ pl = J.pl;
  void* r0 = J.r0;
  void* r1 = J.r1;
  const BRows RX = J.RX, RY = J.RY, RZ = J.RZ;
  const float alpha_h = J.alpha_h, alpha_l = J.alpha_l;
  double* sums = J.sums;
  int* err = J.err;
  extern __shared__ __align__(128) uint8_t res_smem_raw[];
  uint8_t* smem = res_smem_raw + ((128u - (ptx::smem_u32(res_smem_raw) & 127u)) & 127u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kResStages * kResStage);
  uint64_t* empty = full + kResStages;
  ZCoef2* zc = reinterpret_cast<ZCoef2*>(empty + kResStages);
  TermCoefs2* xyc = reinterpret_cast<TermCoefs2*>(zc + kResKseg);   // [32 lanes | kResTY rows]
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int i0 = bx * kResTX, j0 = by * kResTY;
  const int k0 = bz * kResKseg;
  const int k1 = min(nz, k0 + kResKseg);
  const int nplanes = k1 - k0 + 2;                           // planes k0 - 1 .. k1
  if (threadIdx.x == 0) {
    for (int s = 0; s < kResStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), kResTY);
    }
    ptx::fence_mbar_init();
  }
  for (int t = threadIdx.x; t < k1 - k0; t += kResThreads) {
    const int k = k0 + t;
    zc[t] = zcoef2(RZ.ah[k], RZ.al[k], RZ.ch[k], RZ.cl[k], WZ ? RZ.wh[k] : 0.0f, WZ ? RZ.wl[k] : 0.0f);
  }
  for (int t = threadIdx.x; t < 32 + kResTY; t += kResThreads) {
    if (t < 32) {
      const int ii = i0 + 2 * t < nx ? i0 + 2 * t : 0;
      xyc[t] = term_coefs2(RX, ii, ii + 1);
    } else {
      const int jj = j0 + t - 32 < ny ? j0 + t - 32 : 0;
      xyc[t] = term_coefs2(RY, jj, jj);
    }
  }
  __syncthreads();
  if (warp == kResTY) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      ptx::prefetch_tmap(&tPH);
      ptx::prefetch_tmap(&tPL);
      ptx::prefetch_tmap(&tFH);
      ptx::prefetch_tmap(&tFL);
      int s = 0;
      uint32_t par = 0;
      for (int q = 0; q < nplanes; ++q) {
        if (q >= kResStages && !ptx::mbar_wait(ptx::smem_u32(&empty[s]), par ^ 1u, err, ptx::kErrWaitEmpty)) break;
        const int kk = (k0 - 1 + q + nz) % nz;               // wrapped plane
        const bool with_f = q >= 1 && q < nplanes - 1;
        uint8_t* st = smem + s * kResStage;
        const uint32_t bar = ptx::smem_u32(&full[s]);
        ptx::mbar_arrive_expect_tx(bar, 2 * kResPW * (kResTY + 2) * 4 + (with_f ? 2 * kResFBytes : 0));
        const int yrow = j0 - 1 + ny * kk;
        ptx::tma_load_2d(ptx::smem_u32(st), &tPH, bar, i0 - 4, yrow);
        ptx::tma_load_2d(ptx::smem_u32(st + kResPBytes), &tPL, bar, i0 - 4, yrow);
        if (with_f) {
          ptx::tma_load_2d(ptx::smem_u32(st + 2 * kResPBytes), &tFH, bar, i0, j0 + ny * kk);
          ptx::tma_load_2d(ptx::smem_u32(st + 2 * kResPBytes + kResFBytes), &tFL, bar, i0, j0 + ny * kk);
        }
        if (++s == kResStages) {
          s = 0;
          par ^= 1u;
        }
      }
    }
    return;
  }
  // -------------------------------------------------------------- consumers
  const int i = i0 + 2 * lane, j = j0 + warp;
  const bool active = i < nx && j < ny;
  // periodic directions: the edge points load their wrapped neighbours
  const bool edge = active && ((px && (i == 0 || i + 2 == nx)) || (py && (j == 0 || j == ny - 1)));
  const WallCoefs2 c = wall_coefs2<WX, WY>(RX, RY, active ? i : 0, active ? j : 0);
  const df fshift = SING ? fshift_of(J.fsums, J.inv_vol) : df{0.0f, 0.0f};
  const dfx2 FS = {p_dup(fshift.hi), p_dup(fshift.lo)};
  const float2 ach = p_dup(-alpha_h), anch = p_dup(alpha_h), ancl = p_dup(alpha_l);
  const int pc = (warp + 1) * kResPW + 4 + 2 * lane;          // centre of the pair in a phi stage
  const int fc = warp * kResTX + 2 * lane;
  const long long sz = static_cast<long long>(nx) * ny;
  auto pair_at = [&](const uint8_t* st, int e) -> dfx2 {      // points e, e + 1 (e even)
    return {*reinterpret_cast<const float2*>(reinterpret_cast<const float*>(st) + e),
            *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(st + kResPBytes) + e)};
  };
  auto point_at = [&](const uint8_t* st, int e) -> df {
    return {reinterpret_cast<const float*>(st)[e], reinterpret_cast<const float*>(st + kResPBytes)[e]};
  };
  auto release = [&](int s) {
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&empty[s]));
  };
  float acc2 = 0.0f;
  dfx2 P0 = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}, du = P0;
  bool ok = ptx::mbar_wait(ptx::smem_u32(&full[0]), 0, err, ptx::kErrWaitFull);
  dfx2 PM = P0;
  if (ok) {
    PM = pair_at(smem, pc);
    release(0);
    ok = ptx::mbar_wait(ptx::smem_u32(&full[1]), 0, err, ptx::kErrWaitFull);
  }
  if (ok) P0 = pair_at(smem + kResStage, pc);
  du = p_diff(P0, PM);                                         // phi(k0) - phi(k0 - 1)
  long long ro = i + static_cast<long long>(ldx) * (j + static_cast<long long>(ny) * k0);
  const long long rstep = static_cast<long long>(ldx) * ny;
  int s = 1, sn = 2;                                           // stages of planes k and k + 1
  uint32_t parn = 0;                                           // phase parity of stage sn
#pragma unroll 2
  for (int k = k0; ok && k < k1; ++k) {
    const ZCoef2 z = zc[k - k0];
    if (!ptx::mbar_wait(ptx::smem_u32(&full[sn]), parn, err, ptx::kErrWaitFull)) break;
    const dfx2 PP = pair_at(smem + sn * kResStage, pc);
    const uint8_t* st = smem + s * kResStage;
    df xm = point_at(st, pc - 1), xp = point_at(st, pc + 2);
    dfx2 YM = pair_at(st, pc - kResPW), YP = pair_at(st, pc + kResPW);
    const dfx2 F = {*reinterpret_cast<const float2*>(reinterpret_cast<const float*>(st + 2 * kResPBytes) + fc),
                    *reinterpret_cast<const float2*>(
                        reinterpret_cast<const float*>(st + 2 * kResPBytes + kResFBytes) + fc)};
    if (edge) {
      const long long plane = sz * k;
      if (px && i == 0) {
        const long long o = plane + static_cast<long long>(nx) * j + (nx - 1);
        xm = {ph[o], pl[o]};
      }
      if (px && i + 2 == nx) {
        const long long o = plane + static_cast<long long>(nx) * j;
        xp = {ph[o], pl[o]};
      }
      if (py && j == 0) {
        const long long o = plane + static_cast<long long>(nx) * (ny - 1) + i;
        YM = {*reinterpret_cast<const float2*>(ph + o), *reinterpret_cast<const float2*>(pl + o)};
      }
      if (py && j == ny - 1) {
        const long long o = plane + i;
        YP = {*reinterpret_cast<const float2*>(ph + o), *reinterpret_cast<const float2*>(pl + o)};
      }
    }
    if (active) {
      const dfx2 XO = {make_float2(xm.hi, xp.hi), make_float2(xm.lo, xp.lo)};   // (phi_{i-1}, phi_{i+2})
      const TermCoefs2 cx = lds_terms(xyc + lane), cy = lds_terms(xyc + 32 + warp);
      const float2 rv = residual_pair_x2<HAS_ALPHA, WX, WY, WZ, SING>(cx, cy, c, z, ach, anch, ancl, FS, P0, PP,
                                                                      XO, YM, YP, F, du);
      Elem2<FMT>::store(r0, r1, ro, rv.x, rv.y);
      acc2 = fmaf(rv.x, rv.x, acc2);
      acc2 = fmaf(rv.y, rv.y, acc2);
    }
    release(s);
    P0 = PP;
    ro += rstep;
    s = sn;
    if (++sn == kResStages) {
      sn = 0;
      parn ^= 1u;
    }
  }
  double s2 = warp_sum_d(static_cast<double>(acc2));
  if (lane == 0) atomicAdd(&sums[0], s2);
}

template <int FMT, int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__global__ void __launch_bounds__(kResThreads, (WX || WY || WZ || HAS_ALPHA) ? 2 : 3)
residual_tma_kernel(const __grid_constant__ ResJob J) {
  if (J.skip && *J.skip) return;   // the refinement has stopped
  residual_tma_body<FMT, HAS_ALPHA, WX, WY, WZ, SING>(J, blockIdx.x, blockIdx.y, blockIdx.z);
}

// index of the job whose first unit is the largest one <= u (jobs sorted by first)
template <typename Job>
__device__ __forceinline__ int job_index(const Job* __restrict__ jobs, int njobs, long long u) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].first <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Grouped residual: block b is a tile of the instance whose range holds it.
template <int FMT, int HAS_ALPHA, int WX, int WY, int WZ, int SING>
__global__ void __launch_bounds__(kResThreads, 2)   // the job lookup needs the registers of a third block
residual_tma_group_kernel(const ResJob* __restrict__ jobs, int njobs) {
  const ResJob& J = jobs[job_index(jobs, njobs, blockIdx.x)];
  if (J.skip && *J.skip) return;
  const int t = blockIdx.x - J.first;
  residual_tma_body<FMT, HAS_ALPHA, WX, WY, WZ, SING>(J, t % J.tx, (t / J.tx) % J.ty, t / (J.tx * J.ty));
}

// sum of cell volume times phi (float pair) into *out, for the exact gauge;
// work items are 256-point chunks of x-lines (one division per item)
__global__ void __launch_bounds__(256)
wsum_df_kernel(int nx, int ny, int nz, const float* __restrict__ h, const float* __restrict__ l,
               const float* __restrict__ gx, const float* __restrict__ gy,
               const float* __restrict__ gz, double* out) {
  const int nbi = (nx + 255) / 256;
  const long long items = static_cast<long long>(nbi) * ny * nz;
  df s = {0.0f, 0.0f};
  constexpr int U = 4;
  for (long long t0 = blockIdx.x; t0 < items; t0 += static_cast<long long>(U) * gridDim.x) {
    float hh[U], ll[U];
    long long line[U];
    int ii[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long t = t0 + static_cast<long long>(u) * gridDim.x;
      line[u] = t / nbi;
      ii[u] = static_cast<int>(t % nbi) * 256 + threadIdx.x;
      const bool ok = t < items && ii[u] < nx;
      if (!ok) ii[u] = -1;
      const long long o = ok ? ii[u] + static_cast<long long>(nx) * line[u] : 0;
      hh[u] = ok ? h[o] : 0.0f;
      ll[u] = ok ? l[o] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = ii[u];
      if (i < 0) continue;
      const int j = static_cast<int>(line[u] % ny), k = static_cast<int>(line[u] / ny);
      const df wline = df_mul({gy[j], gy[ny + j]}, {gz[k], gz[nz + k]});
      acc_mul(s, wline.hi, wline.lo, df_mul({gx[i], gx[nx + i]}, {hh[u], ll[u]}));
    }
  }
  s = fast_two_sum(s.hi, s.lo);
  double v = static_cast<double>(s.hi) + s.lo;
  v = warp_sum_d(v);
  if (threadIdx.x % 32 == 0) atomicAdd(out, v);
}

// phi = (hi + lo) - shift, shift = (*wsum) * inv_vol when wsum is given (the
// singular problem's zero volume-weighted-mean gauge, applied exactly); the
// pair is converted with integer operations and one float64 add.
__global__ void __launch_bounds__(256)
df_to_f64_kernel(long long n, const float* __restrict__ h, const float* __restrict__ l,
                 const double* __restrict__ wsum, double inv_vol, double* out) {
  const df shift = df_from_double(wsum ? *wsum * inv_vol : 0.0);
  constexpr int U = 4;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long o0 = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o0 < n; o0 += U * stride) {
    float hh[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long o = o0 + u * stride;
      hh[u] = o < n ? h[o] : 0.0f;
      ll[u] = o < n ? l[o] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long o = o0 + u * stride;
      if (o >= n) break;
      const df x = df_sub({hh[u], ll[u]}, shift);
      out[o] = f2d_int(x.hi) + f2d_int(x.lo);
    }
  }
}

// Vectorised forms of prepare_kernel, wsum_df_kernel and df_to_f64_kernel for
// the common aligned case (Nx a multiple of the vector width): each thread
// moves 2 or 4 consecutive points of an x-line with 16-byte loads and stores,
// and the per-line weights and index divisions are shared by those points.
// Same operations per point as the scalar kernels.
template <int FMT>
__device__ __forceinline__ void prepare2_body(int bx, int G, int nx, int ny, int nz, int ldx,
                                              const double* __restrict__ f, float* __restrict__ fh,
                                              float* __restrict__ fl, void* r0, void* r1,
                                              const float* __restrict__ gx, const float* __restrict__ gy,
                                              const float* __restrict__ gz, double* sums) {
  // a block is blockDim.y rows of threads, one x-line (j, k) each, two
  // points per thread; block bx takes the line groups bx, bx + G, bx + 2G,
  // ... (G blocks), U of them per step, whose (j, k) advance by constant
  // steps without a division
  const int lines = ny * nz;
  constexpr int U = 2;
  const int ty = blockDim.y;
  const int step = U * G * ty;
  const int sj = step % ny, sk = step / ny;
  int jj[U], kk[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int L = (bx + u * G) * ty + threadIdx.y;
    jj[u] = L % ny;
    kk[u] = L / ny;
  }
  float s2 = 0.0f, s1f = 0.0f;
  df sv = {0.0f, 0.0f};
  for (int L0 = bx * ty + threadIdx.y; L0 < lines; L0 += step) {
    for (int i = 2 * threadIdx.x; i < nx; i += 2 * blockDim.x) {
      double2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int L = L0 + u * G * ty;
        v[u] = L < lines ? *reinterpret_cast<const double2*>(f + i + static_cast<long long>(nx) * L)
                         : make_double2(0.0, 0.0);
      }
      const float2 gxh = *reinterpret_cast<const float2*>(gx + i);
      const float2 gxl = *reinterpret_cast<const float2*>(gx + nx + i);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int L = L0 + u * G * ty;
        if (L >= lines) break;
        const long long o = i + static_cast<long long>(nx) * L;
        const df d0 = split_double_int(v[u].x), d1 = split_double_int(v[u].y);
        *reinterpret_cast<float2*>(fh + o) = make_float2(d0.hi, d1.hi);
        *reinterpret_cast<float2*>(fl + o) = make_float2(d0.lo, d1.lo);
        Elem2<FMT>::store(r0, r1, i + static_cast<long long>(ldx) * L, d0.hi + d0.lo, d1.hi + d1.lo);
        s2 = fmaf(d0.hi, d0.hi, s2);
        s2 = fmaf(d1.hi, d1.hi, s2);
        s1f += d0.hi;
        s1f += d1.hi;
        const int j = jj[u], k = kk[u];
        const df wline = df_mul({gy[j], gy[ny + j]}, {gz[k], gz[nz + k]});
        acc_mul(sv, wline.hi, wline.lo, df_mul({gxh.x, gxl.x}, d0));
        acc_mul(sv, wline.hi, wline.lo, df_mul({gxh.y, gxl.y}, d1));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      jj[u] += sj;
      kk[u] += sk;
      if (jj[u] >= ny) {
        jj[u] -= ny;
        ++kk[u];
      }
    }
  }
  df s1 = {s1f, 0.0f};
  sv = fast_two_sum(sv.hi, sv.lo);
  __shared__ float red[3][2][8];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid % 32, w = tid / 32;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 = df_add(s1, {__shfl_xor_sync(0xffffffffu, s1.hi, o), __shfl_xor_sync(0xffffffffu, s1.lo, o)});
    sv = df_add(sv, {__shfl_xor_sync(0xffffffffu, sv.hi, o), __shfl_xor_sync(0xffffffffu, sv.lo, o)});
  }
  if (lane == 0) {
    red[0][0][w] = s2;
    red[1][0][w] = s1.hi;
    red[1][1][w] = s1.lo;
    red[2][0][w] = sv.hi;
    red[2][1][w] = sv.lo;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    const int nw = (blockDim.x * blockDim.y + 31) / 32;   // warps of this block (at most 8)
    for (int q = 0; q < nw; ++q) {
      a += red[0][0][q];
      b += static_cast<double>(red[1][0][q]) + red[1][1][q];
      c += static_cast<double>(red[2][0][q]) + red[2][1][q];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
    atomicAdd(&sums[2], c);
  }
}

template <int FMT>
__global__ void __launch_bounds__(256)
prepare2_kernel(int nx, int ny, int nz, int ldx, const double* __restrict__ f, float* __restrict__ fh,
                float* __restrict__ fl, void* r0, void* r1, const float* __restrict__ gx,
                const float* __restrict__ gy, const float* __restrict__ gz, double* sums) {
  prepare2_body<FMT>(blockIdx.x, gridDim.x, nx, ny, nz, ldx, f, fh, fl, r0, r1, gx, gy, gz, sums);
}

// sum of cell volume times phi, four points of an x-line per thread; lines
// are distributed over blocks as in prepare2_kernel
__device__ __forceinline__ void wsum4_body(int bx, int G, int nx, int ny, int nz, const float* __restrict__ h,
                                           const float* __restrict__ l, const float* __restrict__ gx,
                                           const float* __restrict__ gy, const float* __restrict__ gz,
                                           double* out) {
  const int lines = ny * nz;
  constexpr int U = 2;
  const int ty = blockDim.y;
  const int step = U * G * ty;
  const int sj = step % ny, sk = step / ny;
  int jj[U], kk[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int L = (bx + u * G) * ty + threadIdx.y;
    jj[u] = L % ny;
    kk[u] = L / ny;
  }
  df s = {0.0f, 0.0f};
  for (int L0 = bx * ty + threadIdx.y; L0 < lines; L0 += step) {
    for (int i = 4 * threadIdx.x; i < nx; i += 4 * blockDim.x) {
      float4 hh[U], ll[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int L = L0 + u * G * ty;
        const long long o = i + static_cast<long long>(nx) * (L < lines ? L : 0);
        hh[u] = L < lines ? *reinterpret_cast<const float4*>(h + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        ll[u] = L < lines ? *reinterpret_cast<const float4*>(l + o) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const float4 gh = *reinterpret_cast<const float4*>(gx + i);
      const float4 gl = *reinterpret_cast<const float4*>(gx + nx + i);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (L0 + u * G * ty >= lines) break;
        const int j = jj[u], k = kk[u];
        const df wline = df_mul({gy[j], gy[ny + j]}, {gz[k], gz[nz + k]});
        acc_mul(s, wline.hi, wline.lo, df_mul({gh.x, gl.x}, {hh[u].x, ll[u].x}));
        acc_mul(s, wline.hi, wline.lo, df_mul({gh.y, gl.y}, {hh[u].y, ll[u].y}));
        acc_mul(s, wline.hi, wline.lo, df_mul({gh.z, gl.z}, {hh[u].z, ll[u].z}));
        acc_mul(s, wline.hi, wline.lo, df_mul({gh.w, gl.w}, {hh[u].w, ll[u].w}));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      jj[u] += sj;
      kk[u] += sk;
      if (jj[u] >= ny) {
        jj[u] -= ny;
        ++kk[u];
      }
    }
  }
  s = fast_two_sum(s.hi, s.lo);
  double v = static_cast<double>(s.hi) + s.lo;
  v = warp_sum_d(v);
  if ((threadIdx.x + blockDim.x * threadIdx.y) % 32 == 0) atomicAdd(out, v);
}

__global__ void __launch_bounds__(256, 4)
wsum4_kernel(int nx, int ny, int nz, const float* __restrict__ h, const float* __restrict__ l,
             const float* __restrict__ gx, const float* __restrict__ gy, const float* __restrict__ gz,
             double* out) {
  wsum4_body(blockIdx.x, gridDim.x, nx, ny, nz, h, l, gx, gy, gz, out);
}

// df_to_f64_kernel on groups of four points (n a multiple of 4, out 16-byte aligned)
__device__ __forceinline__ void df_to_f64_v4_body(int bx, int G, long long n4, const float4* __restrict__ h,
                                                  const float4* __restrict__ l, const double* __restrict__ wsum,
                                                  double inv_vol, double2* out) {
  const df shift = df_from_double(wsum ? *wsum * inv_vol : 0.0);
  constexpr int U = 2;
  const long long stride = static_cast<long long>(G) * blockDim.x;
  for (long long g0 = bx * static_cast<long long>(blockDim.x) + threadIdx.x; g0 < n4; g0 += U * stride) {
    float4 hh[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long g = g0 + u * stride;
      hh[u] = g < n4 ? h[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      ll[u] = g < n4 ? l[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long g = g0 + u * stride;
      if (g >= n4) break;
      const df a = df_sub({hh[u].x, ll[u].x}, shift), b = df_sub({hh[u].y, ll[u].y}, shift);
      const df c = df_sub({hh[u].z, ll[u].z}, shift), d = df_sub({hh[u].w, ll[u].w}, shift);
      out[2 * g] = make_double2(f2d_int(a.hi) + f2d_int(a.lo), f2d_int(b.hi) + f2d_int(b.lo));
      out[2 * g + 1] = make_double2(f2d_int(c.hi) + f2d_int(c.lo), f2d_int(d.hi) + f2d_int(d.lo));
    }
  }
}

__global__ void __launch_bounds__(256)
df_to_f64_v4_kernel(long long n4, const float4* __restrict__ h, const float4* __restrict__ l,
                    const double* __restrict__ wsum, double inv_vol, double2* out) {
  df_to_f64_v4_body(blockIdx.x, gridDim.x, n4, h, l, wsum, inv_vol, out);
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

// Block of 256 threads as rows of one x-line each: blockDim.x covers Nx with
// `per` points per thread (a multiple of 32, at most 256), blockDim.y lines.
dim3 line_block(int nx, int per) {
  int tx = ((nx + per - 1) / per + 31) / 32 * 32;
  if (tx > 256) tx = 256;
  return dim3(tx, 256 / tx, 1);
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
  note_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? TPT_ERR_OOM : TPT_ERR_CUDA;
}
#define MX_TRY(expr)               \
  do {                             \
    int st_ = (expr);              \
    if (st_ != TPT_OK) return st_; \
  } while (0)
#define MX_CUDA(expr) MX_TRY(st_of(expr))

int dev_alloc(tpt_plan_s* p, size_t bytes, void** out) { return p->arena.alloc(bytes, out); }

template <typename T>
int upload_vec(tpt_plan_s* p, const std::vector<T>& h, T** d) {
  void* ptr = nullptr;
  MX_TRY(p->arena.upload(h.data(), h.size() * sizeof(T), &ptr));
  *d = static_cast<T*>(ptr);
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
  double* scal;        // 16 doubles: [1] sum r^2, [2] sum vol*phi, [5..7] sums of f,
                       // [14] Thomas tile counter (int), [15] error flag
  double* nl;          // 2 * Nz doubles: c', d' of the null line
  float *fh, *fl, *ph, *pl;
  void* R[2];
  void* A[2];
  void* B[2];
  int* skip;           // scal[8]: nonzero once the refinement has stopped (every kernel of a
                       // correction, and its residual, then returns at entry)
};

struct MixedSizes {
  size_t nf, nr, nab, eb, np;
};

MixedSizes sizes_of(const tpt_plan_s* p) {
  const MixedTables& m = p->mixed;
  const size_t nx = p->n[0], ny = p->n[1], nz = p->n[2];
  MixedSizes s;
  s.nf = nx * ny * nz;
  s.nr = static_cast<size_t>(m.ldx) * ny * nz;
  s.nab = std::max(static_cast<size_t>(m.ldy) * nx, static_cast<size_t>(m.ldx) * ny) * nz;
  s.eb = elem_bytes(m.fmt);
  s.np = nplanes(m.fmt);
  return s;
}

MixedWork carve(const tpt_plan_s* p, void* work) {
  const MixedSizes z = sizes_of(p);
  char* w = static_cast<char*>(work);
  MixedWork mw;
  mw.scal = reinterpret_cast<double*>(w);
  mw.skip = reinterpret_cast<int*>(mw.scal + 8);
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
  // B holds T2 as float32 (4 bytes an element) and later T4 in the operand
  // format: two regions of nab 2-byte elements, plane 1 in the second
  mw.B[0] = w;
  mw.B[1] = (z.np == 2) ? static_cast<void*>(w + align256(z.nab * 2)) : nullptr;
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

// Applies the plan's tile choice for transform stage i (0..3).
tc::GemmOut tuned(tc::GemmOut g, const MixedTables& m, int i) {
  g.bn = m.gemm_bn[i];
  g.max_ctas = m.gemm_ctas[i];
  g.pair = m.gemm_pair[i];
  return g;
}

constexpr int kBig = 1 << 30;

template <int FMT>
cudaError_t launch_prepare(const tpt_plan_s* p, const double* f, const MixedWork& w, cudaStream_t s) {
  const int nbi = (p->n[0] + 255) / 256;
  const long long items = static_cast<long long>(nbi) * p->n[1] * p->n[2];
  note_launch(1);
  if (p->n[0] % 2 == 0 && reinterpret_cast<uintptr_t>(f) % 16 == 0) {   // two points per thread
    const long long lines = static_cast<long long>(p->n[1]) * p->n[2];
    const dim3 blk = line_block(p->n[0], 2);
    prepare2_kernel<FMT><<<grid_for(lines * blk.x, blk.x * blk.y, p->dev), blk, 0, s>>>(
        p->n[0], p->n[1], p->n[2], p->mixed.ldx, f, w.fh, w.fl, w.R[0], w.R[1], p->mixed.dfgeom[0],
        p->mixed.dfgeom[1], p->mixed.dfgeom[2], w.scal + 5);
    return cudaGetLastError();
  }
  prepare_kernel<FMT><<<grid_for(items * 256, 256, p->dev), 256, 0, s>>>(
      p->n[0], p->n[1], p->n[2], p->mixed.ldx, nbi, f, w.fh, w.fl, w.R[0], w.R[1], p->mixed.dfgeom[0],
      p->mixed.dfgeom[1], p->mixed.dfgeom[2], w.scal + 5);
  return cudaGetLastError();
}

// Tile width and segment length for Nz rows: 32-line tiles (16 segment slots)
// up to Nz = 512, 16-line tiles (32 slots) above; M is the candidate whose
// nseg = ceil(Nz / M) slots leave the fewest padding rows (ties: the smaller M).
void thomas_shape(int nz, int* tlt, int* m_out) {
  *tlt = nz <= 512 ? 32 : 16;
  const int slots = kThomasThreads / *tlt;
  static const int cand[] = {4, 8, 12, 16, 24, 32};
  int best = 0, pad = 1 << 30;
  for (int m : cand) {
    const int nseg = (nz + m - 1) / m;
    if (nseg > slots) continue;
    if (nseg * m - nz < pad) {
      pad = nseg * m - nz;
      best = m;
    }
  }
  *m_out = best;
}

// Stage geometry and ring size of thomas_tma_kernel; false when the shared
// memory budget cannot hold two input stages and the output tile.
bool thomas_geom(int nz, int m, int tlt, int out_npl, int out_eb, ThomasGeom* g, int budget = kThomasSmemBudget,
                 int row_bytes = static_cast<int>(sizeof(RowCoef))) {
  g->nseg = (nz + m - 1) / m;
  const int r = g->nseg * m;
  g->nb = (r + 255) / 256;
  g->rb = (r + g->nb - 1) / g->nb;
  g->sr = g->nb * g->rb;
  g->in_bytes = g->sr * tlt * 4;
  g->out_bytes = g->sr * tlt * out_eb * out_npl;
  g->coef_bytes = (g->sr * row_bytes + 1023) & ~1023;
  g->stages = (budget - 1024 - g->coef_bytes - g->out_bytes) / g->in_bytes;
  if (g->stages > kThomasMaxStages) g->stages = kThomasMaxStages;
  return g->stages >= 2;
}

template <int FMT, int M, int TLT, int NT = kThomasThreads>
cudaError_t launch_thomas_m(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  constexpr int kPerSm = kThomasThreads / NT;   // CTAs resident on one SM
  using O = T3Fmt<FMT>;
  const MixedTables& m = p->mixed;
  const long long lines = static_cast<long long>(m.ldy) * p->n[0];
  const int nz = p->n[2];
  const long long ntiles = (lines + TLT - 1) / TLT;
  if (ntiles <= 0) return cudaSuccess;
  if (lines + TLT > 0x7fffffffLL) return cudaErrorInvalidValue;   // int line indices and TMA coordinates
  ThomasGeom geo;
  if (!thomas_geom(nz, M, TLT, O::NPL, O::EB, &geo, kThomasSmemBudget / kPerSm)) return cudaErrorInvalidConfiguration;
  CUtensorMap mi, mo0, mo1;
  if (!tc::make_plain_map(&mi, w.B[0], 4, lines, nz, lines * 4, TLT, geo.rb)) return cudaErrorInvalidValue;
  if (!tc::make_plain_map(&mo0, w.A[0], O::EB, lines, nz, lines * O::EB, TLT, geo.rb)) return cudaErrorInvalidValue;
  if (O::NPL == 2) {
    if (!tc::make_plain_map(&mo1, w.A[1], O::EB, lines, nz, lines * O::EB, TLT, geo.rb))
      return cudaErrorInvalidValue;
  } else {
    mo1 = mo0;
  }
  int* next_tile = reinterpret_cast<int*>(w.scal + 14);
  cudaError_t e = cudaMemsetAsync(next_tile, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t smem = 1024 + static_cast<size_t>(geo.coef_bytes) + static_cast<size_t>(geo.stages) * geo.in_bytes +
                      static_cast<size_t>(geo.out_bytes);
  auto kern = thomas_tma_kernel<FMT, M, TLT, NT>;
  // The cap is the kernel's fixed budget, never the size of this launch:
  // threads that launch the same kernel for different Nz (the server's slots)
  // would otherwise lower each other's cap between setting it and launching.
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kThomasSmemBudget / kPerSm);
  if (e != cudaSuccess) return e;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev);
  const long long grid = ntiles < kPerSm * sms ? ntiles : kPerSm * sms;
  note_launch(1);
  kern<<<static_cast<unsigned>(grid), NT, smem, s>>>(
      mi, mo0, mo1, geo, p->n[0], p->n[1], nz, m.ldy, static_cast<int>(ntiles), next_tile, w.A[0], w.A[1],
      m.lam_f[0], m.lam_f[1], m.zrows_f, m.zrows_f + nz, m.zrows_f + 2 * nz, static_cast<float>(p->alpha),
      static_cast<float>(p->beta), p->singular ? 1 : 0, reinterpret_cast<int*>(w.scal + 15), w.skip);
  return cudaGetLastError();
}

// Segment length of thomas2_kernel for Nz rows: the candidate M <= 16 whose
// ceil(Nz / M) <= 32 segments leave the fewest padding rows (ties: the
// smaller M); 0 when Nz > 512.
int thomas2_m(int nz) {
  static const int cand[] = {4, 8, 12, 16};
  int best = 0, pad = 1 << 30;
  for (int m : cand) {
    const int nseg = (nz + m - 1) / m;
    if (nseg > kT2Slots) continue;
    if (nseg * m - nz < pad) {
      pad = nseg * m - nz;
      best = m;
    }
  }
  return best;
}

// Division by d (1 <= d < 2^31) of any 0 <= n < 2^31 as n * magic >> shift:
// with 2^(s-1) < d <= 2^s, magic = floor(2^(31+s) / d) + 1 < 2^32 exceeds
// 2^(31+s) / d by e / d with 0 < e <= d <= 2^s, so n * e < 2^(31+s) and the
// quotient floor(n * magic / 2^(31+s)) is floor(n / d).
void div_magic(unsigned d, unsigned* magic, int* shift) {
  int s = 0;
  while ((1ull << s) < d) ++s;
  *magic = static_cast<unsigned>((1ull << (31 + s)) / d + 1);
  *shift = 31 + s;
}

// The job record of a plan's Thomas step on workspace w (tile numbers from
// `first`); false when T2 or T3 cannot be described by tensor maps or the
// segments do not fit.
template <int FMT, int M>
bool thomas2_job(const tpt_plan_s* p, const MixedWork& w, int first, ThomasJob* J) {
  using O = T3Fmt<FMT>;
  constexpr int TLT = 32;
  const MixedTables& m = p->mixed;
  const long long lines = static_cast<long long>(m.ldy) * p->n[0];
  const int nz = p->n[2];
  if (lines + TLT > 0x7fffffffLL) return false;   // int line indices and TMA coordinates
  std::memset(J, 0, sizeof(*J));
  if (!thomas_geom(nz, M, TLT, O::NPL, O::EB, &J->geo, kT2SmemBudget, static_cast<int>(sizeof(RowCoef2))) ||
      J->geo.nseg > kT2Slots)
    return false;
  if (!tc::make_plain_map(&J->map_in, w.B[0], 4, lines, nz, lines * 4, TLT, J->geo.rb)) return false;
  if (!tc::make_plain_map(&J->map_o0, w.A[0], O::EB, lines, nz, lines * O::EB, TLT, J->geo.rb)) return false;
  if (O::NPL == 2) {
    if (!tc::make_plain_map(&J->map_o1, w.A[1], O::EB, lines, nz, lines * O::EB, TLT, J->geo.rb)) return false;
  } else {
    J->map_o1 = J->map_o0;
  }
  J->nx = p->n[0];
  J->ny = p->n[1];
  J->nz = nz;
  J->ldy = m.ldy;
  J->ntiles = static_cast<int>((lines + TLT - 1) / TLT);
  J->first = first;
  div_magic(static_cast<unsigned>(m.ldy), &J->ldy_magic, &J->ldy_shift);
  J->t3_0 = w.A[0];
  J->t3_1 = w.A[1];
  J->lamx = m.lam_f[0];
  J->lamy = m.lam_f[1];
  J->az = m.zrows_f;
  J->bz = m.zrows_f + nz;
  J->cz = m.zrows_f + 2 * nz;
  J->alpha = static_cast<float>(p->alpha);
  J->beta = static_cast<float>(p->beta);
  J->singular = p->singular ? 1 : 0;
  J->err = reinterpret_cast<int*>(w.scal + 15);
  J->skip = w.skip;
  J->t2 = static_cast<const float*>(w.B[0]);
  J->naz = p->d_rows[2];
  J->ncp = m.null_cp;
  J->ninvm = m.null_invm;
  J->ndz = p->d_dxf[2];
  J->nbeta = p->beta;
  J->nstride = lines;
  return true;
}

size_t thomas2_smem(const ThomasGeom& g) {
  return 1024 + static_cast<size_t>(g.coef_bytes) + static_cast<size_t>(g.stages) * g.in_bytes +
         static_cast<size_t>(g.out_bytes);
}

template <int FMT, int M>
cudaError_t launch_thomas2_m(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  ThomasJob J;
  if (!thomas2_job<FMT, M>(p, w, 0, &J)) return cudaErrorInvalidValue;
  if (J.ntiles <= 0) return cudaSuccess;
  int* next_tile = reinterpret_cast<int*>(w.scal + 14);
  cudaError_t e = cudaMemsetAsync(next_tile, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t smem = thomas2_smem(J.geo);
  auto kern = thomas2_kernel<FMT, M, 0>;
  // a fixed cap (see launch_thomas_m)
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kT2SmemBudget);
  if (e != cudaSuccess) return e;
  if (smem > static_cast<size_t>(kT2SmemBudget)) return cudaErrorInvalidConfiguration;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->dev);
  const int grid = J.ntiles < sms ? J.ntiles : sms;
  note_launch(1);
  kern<<<static_cast<unsigned>(grid), kThomasThreads, smem, s>>>(J, J.geo, next_tile, J.ntiles, nullptr, 0);
  return cudaGetLastError();
}

// Thomas kernel for a plan: 1 one line per thread (thomas_tma_kernel), 2 two
// lines per thread (thomas2_kernel); `variant` 0 picks the two-line kernel
// where its segments are at least 8 rows long (Nz from 193 to 512), where it
// has work for all but a few of its threads.
int thomas_variant(int nz, int variant) {
  if (variant == 1) return 1;
  const int m2 = thomas2_m(nz);
  if (variant == 2) return m2 > 0 ? 2 : 1;
  return (m2 >= 8 && nz > 192) ? 2 : 1;
}

// Step 2.3: T3 = modal Thomas solve of T2 (float32, in B) into A.  The null
// line of a singular problem: inside thomas2_kernel, else on the second stream.
template <int FMT>
cudaError_t launch_thomas(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  const MixedTables& m = p->mixed;
  const int nz = p->n[2];
  const float* t2 = static_cast<const float*>(w.B[0]);
  const bool two = thomas_variant(nz, m.thomas_kernel) == 2;
  const bool fork = p->singular && !two;
  std::unique_lock<std::recursive_mutex> side_lock(const_cast<tpt_plan_s*>(p)->side_mu, std::defer_lock);
  if (fork) {   // fork: the float64 null line runs beside the partition kernel
    side_lock.lock();
    cudaError_t e = cudaEventRecord(m.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m.side, m.fork, 0);
    if (e != cudaSuccess) return e;
    note_launch(1);
    null_line_kernel<FMT><<<1, 32, static_cast<size_t>(nz) * sizeof(double), m.side>>>(
        nz, static_cast<long long>(m.ldy) * p->n[0], t2, w.A[0], w.A[1], p->d_rows[2], m.null_cp, m.null_invm,
        p->d_dxf[2], p->beta, w.skip);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(m.join, m.side);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaErrorInvalidConfiguration;
  int tlt = 0, mm = 0;
  thomas_shape(nz, &tlt, &mm);
  if (two) {
    switch (thomas2_m(nz)) {
      case 4: e = launch_thomas2_m<FMT, 4>(p, w, s); break;
      case 8: e = launch_thomas2_m<FMT, 8>(p, w, s); break;
      case 12: e = launch_thomas2_m<FMT, 12>(p, w, s); break;
      case 16: e = launch_thomas2_m<FMT, 16>(p, w, s); break;
      default: break;
    }
  } else if (tlt == 32) {
    switch (mm) {
      case 4: e = launch_thomas_m<FMT, 4, 32>(p, w, s); break;
      case 8: e = launch_thomas_m<FMT, 8, 32>(p, w, s); break;
      case 12: e = launch_thomas_m<FMT, 12, 32>(p, w, s); break;
      case 16: e = launch_thomas_m<FMT, 16, 32>(p, w, s); break;
      case 24: e = launch_thomas_m<FMT, 24, 32>(p, w, s); break;
      case 32: e = launch_thomas_m<FMT, 32, 32>(p, w, s); break;
      default: break;
    }
  } else {
    switch (mm) {
      case 24: e = launch_thomas_m<FMT, 24, 16>(p, w, s); break;
      case 32: e = launch_thomas_m<FMT, 32, 16>(p, w, s); break;
      default: break;
    }
  }
  if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(s, m.join, 0);   // join
  return e;
}

BRows rows_of(const float* t, int n) {
  return BRows{t, t + n, t + 2 * n, t + 3 * n, t + 4 * n, t + 5 * n};
}

// The residual job of a plan on workspace w with tensor maps m (phi pair,
// f pair), its blocks numbered from `first`.
ResJob res_job(const tpt_plan_s* p, const MixedWork& w, const CUtensorMap m[4], int first) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  ResJob J;
  std::memset(&J, 0, sizeof(J));
  J.tPH = m[0];
  J.tPL = m[1];
  J.tFH = m[2];
  J.tFL = m[3];
  J.nx = nx;
  J.ny = ny;
  J.nz = nz;
  J.ldx = p->mixed.ldx;
  J.px = p->dir[0].periodic ? 1 : 0;
  J.py = p->dir[1].periodic ? 1 : 0;
  J.ph = w.ph;
  J.pl = w.pl;
  J.r0 = w.R[0];
  J.r1 = w.R[1];
  J.RX = rows_of(p->mixed.dfrows[0], nx);
  J.RY = rows_of(p->mixed.dfrows[1], ny);
  J.RZ = rows_of(p->mixed.dfrows[2], nz);
  J.alpha_h = static_cast<float>(p->alpha);
  J.alpha_l = static_cast<float>(p->alpha - static_cast<double>(J.alpha_h));
  J.fsums = w.scal + 5;
  J.inv_vol = 1.0 / p->vol;
  J.sums = w.scal + 1;
  J.err = reinterpret_cast<int*>(w.scal + 15);
  J.skip = w.skip;
  J.first = first;
  J.tx = (nx + kResTX - 1) / kResTX;
  J.ty = (ny + kResTY - 1) / kResTY;
  J.tz = (nz + kResKseg - 1) / kResKseg;
  return J;
}

bool res_maps(const tpt_plan_s* p, const MixedWork& w, CUtensorMap m[4]) {
  const int nx = p->n[0];
  const long long rows = static_cast<long long>(p->n[1]) * p->n[2];
  return nx % 4 == 0 && tc::make_plain_map(&m[0], w.ph, 4, nx, rows, 4LL * nx, kResPW, kResTY + 2) &&
         tc::make_plain_map(&m[1], w.pl, 4, nx, rows, 4LL * nx, kResPW, kResTY + 2) &&
         tc::make_plain_map(&m[2], w.fh, 4, nx, rows, 4LL * nx, kResTX, kResTY) &&
         tc::make_plain_map(&m[3], w.fl, 4, nx, rows, 4LL * nx, kResTX, kResTY);
}

template <int FMT, int HA, int WX, int WY, int WZ, int SING>
cudaError_t launch_res(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int kseg = 32;
  dim3 block(32, 4), grid((nx + 31) / 32, (ny + 3) / 4, (nz + kseg - 1) / kseg);
  const float ah = static_cast<float>(p->alpha);
  const float al = static_cast<float>(p->alpha - static_cast<double>(ah));
  note_launch(1);
  if (nx % 4 == 0 && p->mixed.res_kernel != 1) {   // TMA-staged tiles (rows of 16-byte multiples)
    CUtensorMap m[4];
    const long long rows = static_cast<long long>(ny) * nz;
    bool maps = tc::make_plain_map(&m[0], w.ph, 4, nx, rows, 4LL * nx, kResPW, kResTY + 2) &&
                tc::make_plain_map(&m[1], w.pl, 4, nx, rows, 4LL * nx, kResPW, kResTY + 2) &&
                tc::make_plain_map(&m[2], w.fh, 4, nx, rows, 4LL * nx, kResTX, kResTY) &&
                tc::make_plain_map(&m[3], w.fl, 4, nx, rows, 4LL * nx, kResTX, kResTY);
    if (maps) {
      auto kern = residual_tma_kernel<FMT, HA, WX, WY, WZ, SING>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem);
      if (e != cudaSuccess) return e;
      const ResJob J = res_job(p, w, m, 0);
      kern<<<dim3(J.tx, J.ty, J.tz), kResThreads, kResSmem, s>>>(J);
      return cudaGetLastError();
    }
  }
  if (nx % 2 == 0) {   // two points per thread
    dim3 grid2((nx / 2 + 31) / 32, (ny + 3) / 4, (nz + kseg - 1) / kseg);
    residual_df2_kernel<FMT, HA, WX, WY, WZ, SING><<<grid2, block, 0, s>>>(
        nx, ny, nz, p->mixed.ldx, kseg, w.fh, w.fl, w.ph, w.pl, w.R[0], w.R[1],
        rows_of(p->mixed.dfrows[0], nx), rows_of(p->mixed.dfrows[1], ny), rows_of(p->mixed.dfrows[2], nz),
        ah, al, w.scal + 5, 1.0 / p->vol, w.scal + 1, w.skip);
    return cudaGetLastError();
  }
  residual_df_kernel<FMT, HA, WX, WY, WZ, SING><<<grid, block, 0, s>>>(
      nx, ny, nz, p->mixed.ldx, kseg, w.fh, w.fl, w.ph, w.pl, w.R[0], w.R[1],
      rows_of(p->mixed.dfrows[0], nx), rows_of(p->mixed.dfrows[1], ny), rows_of(p->mixed.dfrows[2], nz),
      ah, al, w.scal + 5, 1.0 / p->vol, w.scal + 1, w.skip);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_residual(const tpt_plan_s* p, const MixedWork& w, cudaStream_t s) {
  const int* hw = p->mixed.has_w;
  const int code = (p->alpha != 0.0 ? 8 : 0) | (hw[0] ? 4 : 0) | (hw[1] ? 2 : 0) | (hw[2] ? 1 : 0);
  // a singular problem (alpha = 0, every direction periodic or Neumann-Neumann)
  // has no wall with a diagonal remainder, so code is 0 there
  if (p->singular) return launch_res<FMT, 0, 0, 0, 0, 1>(p, w, s);
  switch (code) {
    case 0: return launch_res<FMT, 0, 0, 0, 0, 0>(p, w, s);
    case 8: return launch_res<FMT, 1, 0, 0, 0, 0>(p, w, s);
    default: break;
  }
  // walls with a diagonal remainder (Dirichlet): one general instantiation
  if (p->alpha != 0.0) return launch_res<FMT, 1, 1, 1, 1, 0>(p, w, s);
  return launch_res<FMT, 0, 1, 1, 1, 0>(p, w, s);
}

// Operands and output of transform stage i of one correction (Algorithm 1
// steps 1, 3, 7, 9): 0 x forward, 1 y forward, 2 y inverse, 3 x inverse.
struct StageGemm {
  tc::Operand a, b;
  tc::GemmOut g;
};

StageGemm stage_gemm(const tpt_plan_s* p, const MixedWork& w, int i, bool accumulate) {
  const MixedTables& m = p->mixed;
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int om = out_mode(m.fmt);
  int* err = reinterpret_cast<int*>(w.scal + 15);
  StageGemm t;
  switch (i) {
    case 0:   // A = R rows (j,k), B = Q_x^{-1} rows p -> T1 (j, p, k)
      t.a = operand(w.R, ny * nz, nx, m.ldx);
      t.b = operand(m.q[0][0], nx, nx, m.ldx);
      t.g = gout(ny * nz, nx, nx, ny, static_cast<long long>(m.ldy) * nx, m.ldy, w.A[0], w.A[1], om, 0, 1, err);
      break;
    case 1:   // A = Q_y^{-1} rows q, B = T1 rows (p,k) -> T2 (q, p, k), float32 in B
      t.a = operand(m.q[1][0], ny, ny, m.ldy);
      t.b = operand(w.A, nx * nz, ny, m.ldy);
      t.g = gout(ny, nx * nz, ny, kBig, 0, m.ldy, w.B[0], nullptr, tc::kOutF32, 0, 0, err);
      break;
    case 2:   // A = T3 rows (p,k) in A, B = Q_y rows j -> T4 (p, j, k) in B
      t.a = operand(w.A, nx * nz, ny, m.ldy);
      t.b = operand(m.q[1][1], ny, ny, m.ldy);
      t.g = gout(nx * nz, ny, ny, nx, static_cast<long long>(m.ldx) * ny, m.ldx, w.B[0], w.B[1], om, 0, 1, err);
      break;
    default:  // A = Q_x rows i, B = T4 rows (j,k) -> phi (float pair) (+)= result
      t.a = operand(m.q[0][1], nx, nx, m.ldx);
      t.b = operand(w.B, ny * nz, nx, m.ldx);
      t.g = gout(nx, ny * nz, nx, kBig, 0, nx, w.ph, w.pl, tc::kOutDF, accumulate ? 1 : 0, 0, err);
      break;
  }
  return t;
}

// Direction transformed by stage i (x forward, y forward, y inverse, x inverse).
int stage_dir(int i) { return (i == 0 || i == 3) ? 0 : 1; }

// Stage i as a float32 Fourier-based transform of a uniform direction: the
// same operands and layouts as stage_gemm's, the direction just transformed
// written as the slow index (x forward, y inverse) or in place of the rows.
FftMixedArgs stage_fft(const tpt_plan_s* p, const MixedWork& w, int i, bool accumulate) {
  const MixedTables& m = p->mixed;
  const long long nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int d = stage_dir(i);
  FftMixedArgs a;
  a.kind = m.fft_kind[d];
  a.inverse = i >= 2;
  a.N = p->n[d];
  a.in_fmt = m.fmt;
  for (int k = 0; k < 4; ++k) a.tw[k] = m.fft_tw[d][k];
  a.stop = w.skip;
  const int om = out_mode(m.fmt);
  switch (i) {
    case 0:   // R rows (j,k) -> T1 (j, p, k) in A: j fastest, row stride ldy
      a.nlines = ny * nz;
      a.in0 = w.R[0];
      a.in1 = w.R[1];
      a.ldi = m.ldx;
      a.out0 = w.A[0];
      a.out1 = w.A[1];
      a.out_mode = om;
      a.ldo = m.ldy;
      a.L1 = ny;
      break;
    case 1:   // T1 rows (p,k) -> T2 rows (p,k), float32 in B
      a.nlines = nx * nz;
      a.in0 = w.A[0];
      a.in1 = w.A[1];
      a.ldi = m.ldy;
      a.out0 = w.B[0];
      a.out_mode = tc::kOutF32;
      a.ldo = m.ldy;
      break;
    case 2:   // T3 rows (p,k) in A -> T4 (p, j, k) in B: p fastest, row stride ldx
      a.nlines = nx * nz;
      a.in0 = w.A[0];
      a.in1 = w.A[1];
      a.ldi = m.ldy;
      a.out0 = w.B[0];
      a.out1 = w.B[1];
      a.out_mode = om;
      a.ldo = m.ldx;
      a.L1 = nx;
      break;
    default:  // T4 rows (j,k) in B -> phi (float pair) (+)= result
      a.nlines = ny * nz;
      a.in0 = w.B[0];
      a.in1 = w.B[1];
      a.ldi = m.ldx;
      a.out0 = w.ph;
      a.out1 = w.pl;
      a.out_mode = tc::kOutDF;
      a.ldo = nx;
      a.accumulate = accumulate ? 1 : 0;
      break;
  }
  return a;
}

template <int FMT>
int correction(tpt_plan_s* p, const MixedWork& w, bool accumulate, cudaStream_t s) {
  auto mark = [&](int i) {
    if (p->stage_timing) cudaEventRecord(p->ev[i], s);
  };
  auto xform = [&](int i) {
    if (p->xform[stage_dir(i)] == TPT_XFORM_FFT) return fft_mixed(stage_fft(p, w, i, accumulate), s);
    const StageGemm t = stage_gemm(p, w, i, accumulate);
    tc::GemmOut g = tuned(t.g, p->mixed, i);
    g.skip = w.skip;
    return tc::gemm(kind_of(FMT), nplanes(FMT), t.a, t.b, g, s);
  };
  mark(0);
  MX_CUDA(xform(0));                    // step 2.1: x forward
  mark(1);
  MX_CUDA(xform(1));                    // step 2.2: y forward
  mark(2);
  MX_CUDA(launch_thomas<FMT>(p, w, s)); // step 2.3: modal Thomas along z, in place on T2
  mark(3);
  MX_CUDA(xform(2));                    // step 2.4: y inverse
  mark(4);
  MX_CUDA(xform(3));                    // step 2.5: x inverse
  mark(5);
  return TPT_OK;
}

// Device-side stopping test of the adaptive refinement (Sec. 4.1), run after
// each correction's residual: scal[8] (as int) becomes 1 once ||r|| / ||f||
// <= rtol (norm of f projected to compatible form for a singular problem, as
// proj_norm2 computes it), 2 for a non-finite norm and 3 after a timed-out
// wait, and from then on every kernel of a later correction returns at entry;
// scal[8] + 4 bytes counts the corrections applied; scal[11], scal[12] keep
// the last r^2 and f^2 sums; otherwise r's sum is cleared for the next residual.
__device__ __forceinline__ void converge_body(double* scal, double npts, double vol, int singular, double rtol) {
  int* flags = reinterpret_cast<int*>(scal + 8);
  if (flags[0]) return;
  flags[1] += 1;
  const double r2 = scal[1];
  double fn2 = scal[5];
  if (singular) {
    const double c = scal[7] / vol;
    fn2 = scal[5] - 2.0 * c * scal[6] + npts * c * c;
  }
  scal[11] = r2;
  scal[12] = fn2;
  if (*reinterpret_cast<const int*>(scal + 15)) {
    flags[0] = 3;
    return;
  }
  if (!isfinite(r2) || !isfinite(fn2)) {
    flags[0] = 2;
    return;
  }
  const double rel = fn2 > 0.0 ? sqrt(r2 / fn2) : sqrt(r2);
  if (rel <= rtol) {
    flags[0] = 1;
    return;
  }
  scal[1] = 0.0;
  scal[2] = 0.0;
}

__global__ void converge_kernel(double* scal, double npts, double vol, int singular, double rtol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  converge_body(scal, npts, vol, singular, rtol);
}

// The 16 workspace scalars into a pinned, device-mapped host slot.
__global__ void scal_to_host_kernel(const double* __restrict__ scal, double* host) {
  if (threadIdx.x < 16) host[threadIdx.x] = scal[threadIdx.x];
}

// ------------------------------------------------------- grouped launches
// The per-instance data of the grouped stage kernels of a batch: each of
// those kernels runs once over all instances, a block (or thread) finding its
// instance from the block ranges `first[...]` (ascending).
struct InstJob {
  int nx, ny, nz, ldx;
  const double* f;
  double* phi;
  float *fh, *fl, *ph, *pl;
  void *r0, *r1;
  const float *gx, *gy, *gz;   // cell widths as float pairs
  double* scal;                // the instance's 16 workspace scalars
  int singular;
  double npts, vol, rtol;
  const int* skip;
  int first[3], blocks[3];     // block ranges of the prepare, gauge-sum and output kernels
};

__device__ __forceinline__ int inst_of(const InstJob* __restrict__ jobs, int njobs, int range, int b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].first[range] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// every instance's workspace scalars cleared (one block of 32 per instance)
__global__ void group_clear_kernel(const InstJob* __restrict__ jobs) {
  if (threadIdx.x < 16) jobs[blockIdx.x].scal[threadIdx.x] = 0.0;
}

template <int FMT>
__global__ void __launch_bounds__(256) group_prepare_kernel(const InstJob* __restrict__ jobs, int njobs) {
  const InstJob& J = jobs[inst_of(jobs, njobs, 0, blockIdx.x)];
  prepare2_body<FMT>(blockIdx.x - J.first[0], J.blocks[0], J.nx, J.ny, J.nz, J.ldx, J.f, J.fh, J.fl, J.r0, J.r1,
                     J.gx, J.gy, J.gz, J.scal + 5);
}

// stopping test of every instance (one thread each)
__global__ void group_converge_kernel(const InstJob* __restrict__ jobs, int njobs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= njobs) return;
  const InstJob& J = jobs[i];
  converge_body(J.scal, J.npts, J.vol, J.singular, J.rtol);
}

// gauge sums of the singular instances (scal[2] cleared beforehand)
__global__ void __launch_bounds__(256, 4) group_wsum_kernel(const InstJob* __restrict__ jobs, int njobs) {
  const InstJob& J = jobs[inst_of(jobs, njobs, 1, blockIdx.x)];
  if (!J.singular || J.blocks[1] == 0) return;
  wsum4_body(blockIdx.x - J.first[1], J.blocks[1], J.nx, J.ny, J.nz, J.ph, J.pl, J.gx, J.gy, J.gz, J.scal + 2);
}

__global__ void __launch_bounds__(256) group_output_kernel(const InstJob* __restrict__ jobs, int njobs) {
  const InstJob& J = jobs[inst_of(jobs, njobs, 2, blockIdx.x)];
  const long long n4 = static_cast<long long>(J.npts) / 4;
  df_to_f64_v4_body(blockIdx.x - J.first[2], J.blocks[2], n4, reinterpret_cast<const float4*>(J.ph),
                    reinterpret_cast<const float4*>(J.pl), J.singular ? J.scal + 2 : nullptr, 1.0 / J.vol,
                    reinterpret_cast<double2*>(J.phi));
}

// every instance's gauge sum cleared (one thread each)
__global__ void group_clear2_kernel(const InstJob* __restrict__ jobs, int njobs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < njobs) jobs[i].scal[2] = 0.0;
}

// every instance's 16 scalars into out[16 i .. 16 i + 15] (one block of 32 each)
__global__ void group_gather_kernel(const InstJob* __restrict__ jobs, double* out) {
  if (threadIdx.x < 16) out[16 * blockIdx.x + threadIdx.x] = jobs[blockIdx.x].scal[threadIdx.x];
}

double proj_norm2(const double* h, double npts, double vol, bool singular) {
  if (!singular) return h[5];
  const double c = h[7] / vol;
  return h[5] - 2.0 * c * h[6] + npts * c * c;
}

// Adds the elapsed times between the stage events of one correction (and its
// residual, when recorded) to ms[1..6]; the stream must be synchronised.
void add_stage_times(tpt_plan_s* p, float* ms, bool with_residual) {
  for (int i = 0; i < (with_residual ? 6 : 5); ++i) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]) == cudaSuccess) ms[i + 1] += t;
    else cudaGetLastError();
  }
}

// enqueue_only: fixed 1 + max_refine corrections and a final residual, with
// no host synchronisation (capturable in a CUDA graph); the sums stay in the
// workspace scalars for mixed_info().
// Gauge sum (singular problems) and float64 output of the float-pair phi.
cudaError_t launch_output(const tpt_plan_s* p, const MixedWork& w, double* phi, cudaStream_t s) {
  const long long n = static_cast<long long>(npts(p));
  if (p->singular) {
    cudaError_t e0 = cudaMemsetAsync(w.scal + 2, 0, sizeof(double), s);
    if (e0 != cudaSuccess) return e0;
    note_launch(1);
    if (p->n[0] % 4 == 0)   // four points per thread
      wsum4_kernel<<<grid_for(static_cast<long long>(p->n[1]) * p->n[2] * line_block(p->n[0], 4).x,
                              256, p->dev),
                     line_block(p->n[0], 4), 0, s>>>(p->n[0], p->n[1], p->n[2], w.ph, w.pl, p->mixed.dfgeom[0],
                                                     p->mixed.dfgeom[1], p->mixed.dfgeom[2], w.scal + 2);
    else
      wsum_df_kernel<<<grid_for(n, 256, p->dev), 256, 0, s>>>(p->n[0], p->n[1], p->n[2], w.ph, w.pl,
                                                              p->mixed.dfgeom[0], p->mixed.dfgeom[1],
                                                              p->mixed.dfgeom[2], w.scal + 2);
    e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
  }
  note_launch(1);
  if (n % 4 == 0 && reinterpret_cast<uintptr_t>(phi) % 16 == 0)
    df_to_f64_v4_kernel<<<grid_for(n / 4, 256, p->dev), 256, 0, s>>>(
        n / 4, reinterpret_cast<const float4*>(w.ph), reinterpret_cast<const float4*>(w.pl),
        p->singular ? w.scal + 2 : nullptr, 1.0 / p->vol, reinterpret_cast<double2*>(phi));
  else
    df_to_f64_kernel<<<grid_for(n, 256, p->dev), 256, 0, s>>>(n, w.ph, w.pl, p->singular ? w.scal + 2 : nullptr,
                                                              1.0 / p->vol, phi);
  return cudaGetLastError();
}

// Adaptive refinement without a host round trip per correction: the
// corrections and their residuals are enqueued back to back, each followed by
// converge_kernel, whose flag makes the kernels of corrections past
// convergence return at entry.  As many corrections as the plan's previous
// solve needed are enqueued first, with the output conversion behind them,
// and the stream is synchronised once; should they not have converged, the
// remaining corrections and the output conversion are enqueued again.
template <int FMT>
int enqueue_adaptive(tpt_plan_s* p, const MixedWork& w, const double* f, double* phi, int first, int last,
                     bool with_prepare, double* d_hdst, cudaStream_t s) {
  const double np = static_cast<double>(npts(p));
  if (with_prepare) {
    MX_CUDA(cudaMemsetAsync(w.scal, 0, 16 * sizeof(double), s));
    MX_CUDA(launch_prepare<FMT>(p, f, w, s));
  }
  for (int c = first; c < last; ++c) {
    MX_TRY(correction<FMT>(p, w, c > 0, s));
    MX_CUDA(launch_residual<FMT>(p, w, s));
    note_launch(1);
    converge_kernel<<<1, 32, 0, s>>>(w.scal, np, p->vol, p->singular ? 1 : 0, p->rtol);
    MX_CUDA(cudaGetLastError());
  }
  MX_CUDA(launch_output(p, w, phi, s));
  if (!d_hdst) return TPT_OK;   // the caller gathers the scalars itself
  note_launch(1);
  scal_to_host_kernel<<<1, 32, 0, s>>>(w.scal, d_hdst);   // no copy engine: see pinned_slot_acquire
  return cudaGetLastError() == cudaSuccess ? TPT_OK : TPT_ERR_CUDA;
}

// The first `planned` corrections as a CUDA graph (captured on the plan's own
// stream; its scalars land in the plan's pinned copy).
template <int FMT>
int capture_adaptive(tpt_plan_s* p, const MixedWork& w, const double* f, double* phi, int planned) {
  if (p->solve_exec) {
    cudaGraphExecDestroy(p->solve_exec);
    p->solve_exec = nullptr;
  }
  if (!p->cap_stream) MX_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  // the plan's second stream belongs to the capture until it ends: other
  // threads' solves on this plan wait to use it (see tpt_plan_s::side_mu)
  std::lock_guard<std::recursive_mutex> side_guard(p->side_mu);
  const unsigned long long before = launch_count();
  MX_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
  const int st = enqueue_adaptive<FMT>(p, w, f, phi, 0, planned, true, p->d_hscal, p->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
  const unsigned long long recorded = launch_count() - before;
  forget_launches(recorded);   // recorded, not run
  if (st != TPT_OK || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != TPT_OK ? st : TPT_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&p->solve_exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    p->solve_exec = nullptr;
    cudaGetLastError();
    return TPT_ERR_CUDA;
  }
  p->graph_launches = recorded;
  return TPT_OK;
}

// Corrections an adaptive solve enqueues before its first look at the stop
// flags: what the plan's last solve needed, else an estimate from the
// residual reduction one correction of this operand format typically gives
// (measured on stretched grids: ~3.5e-4 split bf16, ~2e-3 tf32, ~8e-3 bf16).
int planned_corrections(const tpt_plan_s* p) {
  const int corrections = 1 + p->max_refine;
  int planned = corrections;
  const int li = p->last_iters.load();
  if (li > 0) {
    planned = li < corrections ? li : corrections;
  } else {
    const double c = p->mixed.fmt == kFmtSplit ? 3.5e-4 : (p->mixed.fmt == kFmtF32 ? 2e-3 : 8e-3);
    const double est = std::ceil(std::log(p->rtol) / std::log(c));
    if (est >= 1.0 && est < corrections) planned = static_cast<int>(est);
  }
  return planned;
}

template <int FMT>
int solve_adaptive(tpt_plan_s* p, const MixedWork& w, const double* f, double* phi, void* work, cudaStream_t s,
                   tpt_info* info) {
  const int corrections = 1 + p->max_refine;
  const int planned = planned_corrections(p);
  int enq = 0;
  bool own = !p->graph_busy.exchange(true);   // this caller may use and update the plan's graph
  // the scalars come back through a pinned slot: the plan's own, or one of
  // this call's when another caller holds the plan's
  double* d_h = nullptr;
  double* h = nullptr;
  double* mine = nullptr;
  if (own) {
    if (!p->h_scal) p->h_scal = pinned_slot_acquire(&p->d_hscal);
    h = p->h_scal;
    d_h = p->d_hscal;
  }
  if (!h) {
    mine = pinned_slot_acquire(&d_h);
    h = mine;
  }
  if (!h) {
    if (own) p->graph_busy.store(false);
    return TPT_ERR_OOM;
  }
  auto leave = [&](int st) {
    if (own) p->graph_busy.store(false);
    pinned_slot_release(mine);
    return st;
  };
  const void* key[3] = {f, phi, work};
  auto same = [&](const void* const* a, int pl, unsigned gen) {
    return a[0] == key[0] && a[1] == key[1] && a[2] == key[2] && pl == planned && gen == p->generation;
  };
  if (own && p->solve_exec && same(p->gkey, p->gkey_planned, p->gkey_gen)) {
    if (cudaGraphLaunch(p->solve_exec, s) != cudaSuccess) {
      cudaGetLastError();
      return leave(TPT_ERR_CUDA);
    }
    note_launch(p->graph_launches);
    enq = planned;
  } else {
    const int st = enqueue_adaptive<FMT>(p, w, f, phi, 0, planned, true, d_h, s);
    if (st != TPT_OK) return leave(st);
    enq = planned;
    if (own && same(p->gprev, p->gprev_planned, p->gprev_gen)) {
      // the same call twice in a row: keep it as a graph for the next ones
      if (capture_adaptive<FMT>(p, w, f, phi, planned) == TPT_OK) {
        for (int i = 0; i < 3; ++i) p->gkey[i] = key[i];
        p->gkey_planned = planned;
        p->gkey_gen = p->generation;
      }
    }
    if (own) {
      for (int i = 0; i < 3; ++i) p->gprev[i] = key[i];
      p->gprev_planned = planned;
      p->gprev_gen = p->generation;
    }
  }
  int flags[2] = {0, 0};
  double hv[16];
  for (;;) {
    const cudaError_t se = cudaStreamSynchronize(s);
    if (se != cudaSuccess) {
      cudaGetLastError();
      return leave(TPT_ERR_CUDA);
    }
    for (int i = 0; i < 16; ++i) hv[i] = static_cast<volatile double*>(h)[i];
    std::memcpy(flags, &hv[8], sizeof(flags));
    if (flags[0] != 0 || enq >= corrections) break;
    // not converged within the planned corrections: the rest, enqueued directly
    const int st = enqueue_adaptive<FMT>(p, w, f, phi, enq, corrections, false, d_h, s);
    if (st != TPT_OK) return leave(st);
    enq = corrections;
  }
  leave(TPT_OK);
  const int iters = flags[1];
  p->last_iters.store(iters);
  const double rel = hv[12] > 0.0 ? std::sqrt(hv[11] / hv[12]) : std::sqrt(hv[11]);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = iters;
    info->rel_residual = rel;
    info->compat_defect = p->singular ? hv[7] / p->vol : 0.0;
  }
  if (flags[0] == 3) return TPT_ERR_TIMEOUT;
  if (flags[0] == 2) return TPT_ERR_NONFINITE;
  if (flags[0] != 1) return TPT_ERR_NOT_CONVERGED;
  return TPT_OK;
}

template <int FMT>
int solve_fmt(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s, tpt_info* info,
              bool enqueue_only) {
  const MixedWork w = carve(p, work);
  float ms[8] = {0.0f};
  const bool timing = p->stage_timing && info && !enqueue_only;
  if (p->rtol > 0.0 && !enqueue_only && !timing) return solve_adaptive<FMT>(p, w, f, phi, work, s, info);
  if (timing && !p->ev[0])
    for (cudaEvent_t& e : p->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return TPT_ERR_CUDA;
  const int saved_timing = p->stage_timing;
  p->stage_timing = timing ? 1 : 0;
  if (timing) cudaEventRecord(p->ev[8], s);
  MX_CUDA(cudaMemsetAsync(w.scal, 0, 16 * sizeof(double), s));
  MX_CUDA(launch_prepare<FMT>(p, f, w, s));
  if (timing) cudaEventRecord(p->ev[9], s);
  const int corrections = 1 + p->max_refine;
  const bool adaptive = p->rtol > 0.0 && !enqueue_only;
  const double np = static_cast<double>(npts(p));
  double h[16] = {0.0};
  double rel = -1.0;
  int iters = 0, status = TPT_OK;
  bool converged = false;
  for (;;) {
    MX_TRY(correction<FMT>(p, w, iters > 0, s));
    ++iters;
    const bool need_residual = iters < corrections || adaptive || info || enqueue_only;
    if (!need_residual) {
      if (timing) {
        MX_CUDA(cudaEventSynchronize(p->ev[5]));
        add_stage_times(p, ms, false);
      }
      break;
    }
    MX_CUDA(cudaMemsetAsync(w.scal + 1, 0, 2 * sizeof(double), s));
    MX_CUDA(launch_residual<FMT>(p, w, s));
    if (timing) {
      cudaEventRecord(p->ev[6], s);
      MX_CUDA(cudaEventSynchronize(p->ev[6]));
      add_stage_times(p, ms, true);
    }
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
  if (timing) cudaEventRecord(p->ev[10], s);
  MX_CUDA(launch_output(p, w, phi, s));
  if (timing) {
    cudaEventRecord(p->ev[11], s);
    MX_CUDA(cudaEventSynchronize(p->ev[11]));
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, p->ev[8], p->ev[9]) == cudaSuccess) ms[0] = t;
    if (cudaEventElapsedTime(&t, p->ev[10], p->ev[11]) == cudaSuccess) ms[7] = t;
    cudaGetLastError();
  }
  if (adaptive && !converged) status = TPT_ERR_NOT_CONVERGED;
  if (info && !enqueue_only) {
    if (!adaptive) {
      MX_CUDA(cudaMemcpyAsync(h, w.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MX_CUDA(cudaStreamSynchronize(s));
      const double fn2 = proj_norm2(h, np, p->vol, p->singular);
      rel = fn2 > 0.0 ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
    }
    info->iters = iters;
    info->rel_residual = rel;
    info->compat_defect = p->singular ? h[7] / p->vol : 0.0;
    for (int i = 0; i < 8; ++i) info->ms_stage[i] = ms[i];
  }
  p->stage_timing = saved_timing;
  return status;
}

}  // namespace

int mixed_pack_basis(DevArena& a, int fmt, const Eigen1D& e, const std::vector<double>& dxf, int dev,
                     void* q[2][2], float** lam_f) {
  const int n = static_cast<int>(dxf.size());
  const int ld = (n + 7) & ~7;
  const int np = nplanes(fmt);
  const size_t eb = elem_bytes(fmt);
  std::vector<double> fwd(static_cast<size_t>(n) * n), inv(static_cast<size_t>(n) * n);
  for (int mode = 0; mode < n; ++mode)
    for (int i = 0; i < n; ++i) {
      const double s = std::sqrt(dxf[i]);
      const double v = e.qt[static_cast<size_t>(mode) * n + i];
      fwd[static_cast<size_t>(mode) * n + i] = v * s;   // Q^{-1}(mode, i), row-major
      inv[static_cast<size_t>(i) * n + mode] = v / s;   // Q(i, mode), row-major
    }
  for (int role = 0; role < 2; ++role) {
    const std::vector<double>& src = role == 0 ? fwd : inv;
    void* stage = nullptr;
    MX_TRY(a.upload(src.data(), src.size() * sizeof(double), &stage));
    q[role][0] = q[role][1] = nullptr;
    for (int pl = 0; pl < np; ++pl) {
      MX_TRY(a.alloc(eb * static_cast<size_t>(n) * ld, &q[role][pl]));
      MX_CUDA(cudaMemsetAsync(q[role][pl], 0, eb * static_cast<size_t>(n) * ld, a.stream));
    }
    MX_CUDA(pack_operand(fmt, n, n, ld, static_cast<const double*>(stage), q[role][0], q[role][1], dev, a.stream));
  }
  std::vector<float> lf(e.lam.begin(), e.lam.end());
  void* lp = nullptr;
  MX_TRY(a.upload(lf.data(), lf.size() * sizeof(float), &lp));
  *lam_f = static_cast<float*>(lp);
  // the host staging vectors die here
  MX_CUDA(cudaStreamSynchronize(a.stream));
  return TPT_OK;
}

// Tables of a Fourier-transformed direction d of a mixed plan: eigenvalues in
// the transform's mode order and the float32 twiddles (rounded from long
// double), in the plan's arena.
int fft_tables_f32(tpt_plan_s* p, int d) {
  MixedTables& m = p->mixed;
  const int n = p->n[d];
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<float> t[4];
  t[0].assign(n / 2 > 0 ? n / 2 : 1, 1.0f);
  t[1].assign(t[0].size(), 0.0f);
  t[2].resize(n);
  t[3].resize(n);
  for (int k = 0; k < n / 2; ++k) {
    t[0][k] = static_cast<float>(std::cos(2.0L * pi * k / n));
    t[1][k] = static_cast<float>(std::sin(2.0L * pi * k / n));
  }
  for (int k = 0; k < n; ++k) {
    t[2][k] = static_cast<float>(std::cos(pi * k / (2.0L * n)));
    t[3][k] = static_cast<float>(std::sin(pi * k / (2.0L * n)));
  }
  for (int k = 0; k < 4; ++k) {
    float* dptr = nullptr;
    MX_TRY(upload_vec(p, t[k], &dptr));
    m.fft_tw[d][k] = dptr;
  }
  std::vector<float> lf(p->eig[d].lam.begin(), p->eig[d].lam.end());
  MX_TRY(upload_vec(p, lf, &m.lam_f[d]));
  m.fft_kind[d] = p->fft[d].kind;
  MX_CUDA(cudaStreamSynchronize(p->arena.stream));   // the host vectors die here
  return TPT_OK;
}

int mixed_setup(tpt_plan_s* p) {
  MixedTables& m = p->mixed;
  m.fmt = fmt_of(p->precision);
  m.ldx = (p->n[0] + 7) & ~7;
  m.ldy = (p->n[1] + 7) & ~7;
  for (int d = 0; d < 2; ++d) {
    if (p->xform[d] == TPT_XFORM_FFT) {   // no operand matrices: float32 twiddles
      MX_TRY(fft_tables_f32(p, d));
      continue;
    }
    void* q[2][2] = {};
    if (p->basis[d]) MX_TRY(entry_mixed_tables(*p->basis[d], m.fmt, p->dev, q, &m.lam_f[d]));
    else MX_TRY(mixed_pack_basis(p->arena, m.fmt, p->eig[d], p->dir[d].dxf, p->dev, q, &m.lam_f[d]));
    for (int r = 0; r < 2; ++r)
      for (int pl = 0; pl < 2; ++pl) m.q[d][r][pl] = q[r][pl];
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
    const int n = p->dir[d].n;
    void* ptr = nullptr;
    MX_TRY(dev_alloc(p, 6 * sizeof(float) * static_cast<size_t>(n), &ptr));
    m.dfrows[d] = static_cast<float*>(ptr);
  }
  MX_TRY(mixed_set_beta(p));
  {
    // factorisation of T_z with the last (singular) row left out: c'_k, 1/m_k
    const Dir1D& z = p->dir[2];
    std::vector<double> ncp(z.n, 0.0), ninv(z.n, 0.0);
    double cprev = 0.0;
    for (int k = 0; k + 1 < z.n; ++k) {
      const double mk = z.b[k] - z.a[k] * cprev;
      ninv[k] = 1.0 / mk;
      ncp[k] = z.c[k] * ninv[k];
      cprev = ncp[k];
    }
    MX_TRY(upload_vec(p, ncp, &m.null_cp));
    MX_TRY(upload_vec(p, ninv, &m.null_invm));
  }
  for (int d = 0; d < 3; ++d) {
    const int n = p->dir[d].n;
    std::vector<float> t(2 * static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) split_ld(p->dir[d].dxf[i], &t[i], &t[n + i]);
    MX_TRY(upload_vec(p, t, &m.dfgeom[d]));
  }
  MX_CUDA(cudaStreamCreateWithFlags(&m.side, cudaStreamNonBlocking));
  MX_CUDA(cudaEventCreateWithFlags(&m.fork, cudaEventDisableTiming));
  MX_CUDA(cudaEventCreateWithFlags(&m.join, cudaEventDisableTiming));
  MX_CUDA(cudaStreamSynchronize(p->arena.stream));
  return TPT_OK;
}

int mixed_set_beta(tpt_plan_s* p) {
  MixedTables& m = p->mixed;
  const long double beta = p->beta;
  for (int d = 0; d < 3; ++d) {
    const Dir1D& dd = p->dir[d];
    const int n = dd.n;
    std::vector<float> t(6 * static_cast<size_t>(n));
    int hw = 0;
    for (int i = 0; i < n; ++i) {
      const long double a = dd.a[i], b = dd.b[i], c = dd.c[i];
      long double w = -(a + b + c);
      // the remainder of b = -(a + c) rounded is ~1e-16 |b|: dropped; a
      // Dirichlet wall term (2 / dx^2) is kept
      if (std::fabs(static_cast<double>(w)) <= 1e-12 * (std::fabs(dd.a[i]) + std::fabs(dd.c[i]))) w = 0.0L;
      if (w != 0.0L) hw = 1;
      split_ld(beta * a, &t[i], &t[n + i]);
      split_ld(beta * c, &t[2 * n + i], &t[3 * n + i]);
      split_ld(beta * w, &t[4 * n + i], &t[5 * n + i]);
    }
    m.has_w[d] = hw;
    MX_CUDA(cudaMemcpyAsync(m.dfrows[d], t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice,
                            p->arena.stream));
    MX_CUDA(cudaStreamSynchronize(p->arena.stream));   // t dies here; the next solve may run on any stream
  }
  m.rows_beta = p->beta;
  return TPT_OK;
}

size_t mixed_workspace_bytes(const tpt_plan_s* p) {
  const MixedSizes z = sizes_of(p);
  size_t b = 256 + align256(2 * sizeof(double) * p->n[2]);
  b += 4 * align256(z.nf * sizeof(float));
  b += z.np * align256(z.nr * z.eb);
  b += z.np * align256(z.nab * z.eb);   // A
  b += 2 * align256(z.nab * 2);          // B: float32 T2, then T4
  return b;
}

int mixed_solve(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s, tpt_info* info) {
  switch (p->mixed.fmt) {
    case kFmtSplit: return solve_fmt<kFmtSplit>(p, f, phi, work, s, info, false);
    case kFmtBF16: return solve_fmt<kFmtBF16>(p, f, phi, work, s, info, false);
    default: return solve_fmt<kFmtF32>(p, f, phi, work, s, info, false);
  }
}

int mixed_enqueue(tpt_plan_s* p, const double* f, double* phi, void* work, cudaStream_t s) {
  if (p->rtol > 0.0) {   // every correction enqueued; those past convergence return at entry
    const MixedWork w = carve(p, work);
    const int corrections = 1 + p->max_refine;
    switch (p->mixed.fmt) {
      case kFmtSplit: return enqueue_adaptive<kFmtSplit>(p, w, f, phi, 0, corrections, true, nullptr, s);
      case kFmtBF16: return enqueue_adaptive<kFmtBF16>(p, w, f, phi, 0, corrections, true, nullptr, s);
      default: return enqueue_adaptive<kFmtF32>(p, w, f, phi, 0, corrections, true, nullptr, s);
    }
  }
  switch (p->mixed.fmt) {
    case kFmtSplit: return solve_fmt<kFmtSplit>(p, f, phi, work, s, nullptr, true);
    case kFmtBF16: return solve_fmt<kFmtBF16>(p, f, phi, work, s, nullptr, true);
    default: return solve_fmt<kFmtF32>(p, f, phi, work, s, nullptr, true);
  }
}

// ------------------------------------------------------ grouped batch solve
// Every instance of a batch solved by grouped launches: one kernel per stage
// over all instances (per Thomas segment length and per residual variant),
// each taking its units (tiles of a GEMM, line tiles of the Thomas sweep,
// plane tiles of the residual, blocks of the elementwise stages) from the
// whole batch; an instance that has met its rtol stops, its units passed
// over by every later kernel.  Qualifying batches: split-bf16 plans with
// rtol > 0, Nx a multiple of 4, Nz <= 512.
struct GroupSolve {
  int n = 0, dev = 0;
  std::vector<tpt_plan_s*> plans;
  std::vector<size_t> ws_off;          // workspace of instance i at work + ws_off[i]
  size_t ws_bytes = 0;
  // device tables: instances, GEMM jobs of the four stages (x inverse: first
  // correction and later ones), Thomas jobs per segment length, residual jobs
  // per variant, ids of the singular instances, Thomas tile counters
  void* dmem = nullptr;
  size_t dmem_bytes = 0;
  InstJob* d_inst = nullptr;
  tc::GemmJob* d_gemm[5] = {};
  long long gemm_units[5] = {};
  bool gemm_tma[5] = {};
  struct TGroup { int m = 0; int njobs = 0; int tiles = 0; ThomasGeom lg{}; ThomasJob* d = nullptr; };
  std::vector<TGroup> tg;
  struct RGroup { int code = 0; int njobs = 0; int blocks = 0; ResJob* d = nullptr; };
  std::vector<RGroup> rg;
  int* d_counters = nullptr;           // one per Thomas group and correction
  int max_nz = 0;
  int blocks[3] = {0, 0, 0};           // prepare, gauge sum, output
  std::vector<const void*> key;        // buffers the tables were built for
  std::vector<unsigned> gens;
  unsigned long long kernels = 0;      // kernels of the last enqueue
  bool external = false;               // dmem belongs to the caller
};

namespace {

int res_code(const tpt_plan_s* p) {
  if (p->singular) return 1;
  const int* hw = p->mixed.has_w;
  if (!hw[0] && !hw[1] && !hw[2]) return p->alpha != 0.0 ? 2 : 0;
  return p->alpha != 0.0 ? 3 : 4;
}

template <int HA, int WX, int WY, int WZ, int SING>
cudaError_t launch_res_group(const GroupSolve::RGroup& r, cudaStream_t s) {
  auto kern = residual_tma_group_kernel<kFmtSplit, HA, WX, WY, WZ, SING>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem);
  if (e != cudaSuccess) return e;
  note_launch(1);
  kern<<<r.blocks, kResThreads, kResSmem, s>>>(r.d, r.njobs);
  return cudaGetLastError();
}

cudaError_t launch_res_code(const GroupSolve::RGroup& r, cudaStream_t s) {
  switch (r.code) {
    case 0: return launch_res_group<0, 0, 0, 0, 0>(r, s);
    case 1: return launch_res_group<0, 0, 0, 0, 1>(r, s);
    case 2: return launch_res_group<1, 0, 0, 0, 0>(r, s);
    case 3: return launch_res_group<1, 1, 1, 1, 0>(r, s);
    default: return launch_res_group<0, 1, 1, 1, 0>(r, s);
  }
}

template <int M>
cudaError_t launch_thomas_group(const GroupSolve::TGroup& t, int* counter, int dev, cudaStream_t s) {
  auto kern = thomas2_kernel<kFmtSplit, M, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kT2SmemBudget);
  if (e != cudaSuccess) return e;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = t.tiles < sms ? t.tiles : sms;
  ThomasJob none;
  std::memset(&none, 0, sizeof(none));
  note_launch(1);
  kern<<<grid, kThomasThreads, thomas2_smem(t.lg), s>>>(none, t.lg, counter, t.tiles, t.d, t.njobs);
  return cudaGetLastError();
}

cudaError_t launch_thomas_m_group(const GroupSolve::TGroup& t, int* counter, int dev, cudaStream_t s) {
  switch (t.m) {
    case 4: return launch_thomas_group<4>(t, counter, dev, s);
    case 8: return launch_thomas_group<8>(t, counter, dev, s);
    case 12: return launch_thomas_group<12>(t, counter, dev, s);
    case 16: return launch_thomas_group<16>(t, counter, dev, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
bool thomas_job_m(const tpt_plan_s* p, const MixedWork& w, int first, ThomasJob* J) {
  return thomas2_job<kFmtSplit, M>(p, w, first, J);
}

bool thomas_job_any(int m, const tpt_plan_s* p, const MixedWork& w, int first, ThomasJob* J) {
  switch (m) {
    case 4: return thomas_job_m<4>(p, w, first, J);
    case 8: return thomas_job_m<8>(p, w, first, J);
    case 12: return thomas_job_m<12>(p, w, first, J);
    case 16: return thomas_job_m<16>(p, w, first, J);
    default: return false;
  }
}

}  // namespace

bool group_eligible(const tpt_plan_s* p) {
  return p->dev >= 0 && p->precision == TPT_PREC_MIXED_BF16X3 && p->mixed.fmt == kFmtSplit && p->rtol > 0.0 &&
         p->n[0] % 4 == 0 && thomas2_m(p->n[2]) != 0 && p->xform[0] == TPT_XFORM_GEMM &&
         p->xform[1] == TPT_XFORM_GEMM;
}

GroupSolve* group_create(tpt_plan_s* const* plans, int n) {
  if (n <= 0) return nullptr;
  for (int i = 0; i < n; ++i)
    if (!group_eligible(plans[i]) || plans[i]->dev != plans[0]->dev) return nullptr;
  GroupSolve* g = new (std::nothrow) GroupSolve;
  if (!g) return nullptr;
  g->n = n;
  g->dev = plans[0]->dev;
  g->plans.assign(plans, plans + n);
  for (int i = 0; i < n; ++i) {
    g->ws_off.push_back(g->ws_bytes);
    g->ws_bytes += align256(mixed_workspace_bytes(plans[i]));
    g->max_nz = std::max(g->max_nz, plans[i]->n[2]);
  }
  return g;
}

void group_destroy(GroupSolve* g) {
  if (!g) return;
  if (g->dmem && !g->external) cudaFree(g->dmem);
  delete g;
}

size_t group_table_bytes(const GroupSolve* g) {
  // an upper bound of group_prepare's layout: at most 4 Thomas groups (one per
  // segment length) and 5 residual variants, each rounded up to 256 bytes
  const size_t n = g ? static_cast<size_t>(g->n) : 0;
  return align256(sizeof(InstJob) * n) + 5 * align256(sizeof(tc::GemmJob) * n) + sizeof(ThomasJob) * n +
         4 * 256 + sizeof(ResJob) * n + 5 * 256 + align256(sizeof(int) * std::max<size_t>(1, n)) +
         align256(sizeof(int) * 4 * 64);
}

void group_set_memory(GroupSolve* g, void* mem, size_t bytes) {
  if (g->dmem && !g->external) cudaFree(g->dmem);
  g->dmem = mem;
  g->dmem_bytes = bytes;
  g->external = true;
  g->key.clear();
}

size_t group_workspace_bytes(const GroupSolve* g) { return g ? g->ws_bytes : 0; }
unsigned long long group_kernels(const GroupSolve* g) { return g ? g->kernels : 0; }

// Builds the job tables for these buffers and copies them to the device
// (synchronously, so that the launches may be captured afterwards).
int group_prepare(GroupSolve* g, const double* const* f, double* const* phi, void* work, cudaStream_t s) {
  for (int i = 0; i < g->n; ++i)   // 16-byte vector loads of f and stores of phi
    if (reinterpret_cast<uintptr_t>(f[i]) % 16 != 0 || reinterpret_cast<uintptr_t>(phi[i]) % 16 != 0)
      return TPT_ERR_UNSUPPORTED;
  std::vector<const void*> key;
  std::vector<unsigned> gens;
  for (int i = 0; i < g->n; ++i) {
    key.push_back(f[i]);
    key.push_back(phi[i]);
    gens.push_back(g->plans[i]->generation);
  }
  key.push_back(work);
  if (g->dmem && key == g->key && gens == g->gens) return TPT_OK;
  const int n = g->n;
  std::vector<MixedWork> ws(n);
  for (int i = 0; i < n; ++i) ws[i] = carve(g->plans[i], static_cast<char*>(work) + g->ws_off[i]);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->dev);
  // instances and the block ranges of the elementwise stages
  std::vector<InstJob> inst(n);
  int nb[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const tpt_plan_s* p = g->plans[i];
    const MixedWork& w = ws[i];
    InstJob& J = inst[i];
    std::memset(&J, 0, sizeof(J));
    J.nx = p->n[0];
    J.ny = p->n[1];
    J.nz = p->n[2];
    J.ldx = p->mixed.ldx;
    J.f = f[i];
    J.phi = phi[i];
    J.fh = w.fh;
    J.fl = w.fl;
    J.ph = w.ph;
    J.pl = w.pl;
    J.r0 = w.R[0];
    J.r1 = w.R[1];
    J.gx = p->mixed.dfgeom[0];
    J.gy = p->mixed.dfgeom[1];
    J.gz = p->mixed.dfgeom[2];
    J.scal = w.scal;
    J.singular = p->singular ? 1 : 0;
    J.npts = static_cast<double>(npts(p));
    J.vol = p->vol;
    J.rtol = p->rtol;
    J.skip = w.skip;
    const long long lines = static_cast<long long>(p->n[1]) * p->n[2];
    const int per_block = 8;                    // lines of a 32 x 8 block
    const int b0 = static_cast<int>(std::min<long long>((lines + per_block - 1) / per_block, 2LL * sms));
    const int b2 = static_cast<int>(std::min<long long>((npts(p) / 4 + 255) / 256, 2LL * sms));
    J.first[0] = nb[0];
    J.blocks[0] = b0;
    nb[0] += b0;
    J.first[1] = nb[1];
    J.blocks[1] = p->singular ? b0 : 0;
    nb[1] += J.blocks[1];
    J.first[2] = nb[2];
    J.blocks[2] = b2;
    nb[2] += b2;
  }
  for (int r = 0; r < 3; ++r) g->blocks[r] = nb[r];
  // GEMM jobs: x forward, y forward, y inverse, x inverse (first, later)
  std::vector<tc::GemmJob> gj[5];
  for (int st = 0; st < 5; ++st) {
    const int stage = st < 4 ? st : 3;
    long long units = 0;
    bool tma = (stage == 0 || stage == 2 || stage == 1);
    for (int pass = 0; pass < 2; ++pass) {   // with the TMA-store epilogue if every job allows it
      gj[st].assign(n, tc::GemmJob{});
      units = 0;
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) {
        const StageGemm t = stage_gemm(g->plans[i], ws[i], stage, st == 4);
        tc::GemmOut go = t.g;
        go.skip = ws[i].skip;
        go.bn = 256;
        ok = tc::make_job(t.a, t.b, go, tma, &gj[st][i], units);
        units += tc::job_units(go);
      }
      if (ok) break;
      if (!tma) return TPT_ERR_UNSUPPORTED;
      tma = false;
    }
    g->gemm_units[st] = units;
    g->gemm_tma[st] = tma;
  }
  // Thomas jobs grouped by segment length, residual jobs by variant
  std::vector<std::vector<ThomasJob>> tj;
  std::vector<GroupSolve::TGroup> tg;
  std::vector<std::vector<ResJob>> rj;
  std::vector<GroupSolve::RGroup> rg;
  for (int i = 0; i < n; ++i) {
    const tpt_plan_s* p = g->plans[i];
    const int m = thomas2_m(p->n[2]);
    size_t k = 0;
    while (k < tg.size() && tg[k].m != m) ++k;
    if (k == tg.size()) {
      tg.push_back(GroupSolve::TGroup{});
      tg[k].m = m;
      tg[k].lg.stages = 2;
      tj.emplace_back();
    }
    ThomasJob J;
    if (!thomas_job_any(m, p, ws[i], tg[k].tiles, &J)) return TPT_ERR_UNSUPPORTED;
    tg[k].tiles += J.ntiles;
    tg[k].lg.in_bytes = std::max(tg[k].lg.in_bytes, J.geo.in_bytes);
    tg[k].lg.out_bytes = std::max(tg[k].lg.out_bytes, J.geo.out_bytes);
    tg[k].lg.coef_bytes = std::max(tg[k].lg.coef_bytes, J.geo.coef_bytes);
    tj[k].push_back(J);
    const int code = res_code(p);
    size_t r = 0;
    while (r < rg.size() && rg[r].code != code) ++r;
    if (r == rg.size()) {
      rg.push_back(GroupSolve::RGroup{});
      rg[r].code = code;
      rj.emplace_back();
    }
    CUtensorMap m4[4];
    if (!res_maps(p, ws[i], m4)) return TPT_ERR_UNSUPPORTED;
    const ResJob R = res_job(p, ws[i], m4, rg[r].blocks);
    rg[r].blocks += R.tx * R.ty * R.tz;
    rj[r].push_back(R);
  }
  for (auto& t : tg) {   // as many stages as the budget holds beside the output tile and rows
    const long long room = static_cast<long long>(kT2SmemBudget) - 1024 - t.lg.coef_bytes - t.lg.out_bytes;
    t.lg.stages = static_cast<int>(std::min<long long>(kThomasMaxStages, room / std::max(1, t.lg.in_bytes)));
    if (t.lg.stages < 2) return TPT_ERR_UNSUPPORTED;
    t.njobs = 0;
  }
  // one device block for every table
  size_t bytes = align256(sizeof(InstJob) * n);
  for (int st = 0; st < 5; ++st) bytes += align256(sizeof(tc::GemmJob) * n);
  for (auto& v : tj) bytes += align256(sizeof(ThomasJob) * v.size());
  for (auto& v : rj) bytes += align256(sizeof(ResJob) * v.size());
  const int max_corr = 64;
  bytes += align256(sizeof(int) * tg.size() * max_corr);
  if (bytes > g->dmem_bytes) {
    if (g->external) return TPT_ERR_INVALID_ARG;   // group_table_bytes bounds the layout
    MX_CUDA(cudaStreamSynchronize(s));
    if (g->dmem) cudaFree(g->dmem);
    g->dmem = nullptr;
    g->dmem_bytes = 0;
    MX_CUDA(cudaMalloc(&g->dmem, bytes));
    g->dmem_bytes = bytes;
  }
  std::vector<char> host(bytes, 0);
  size_t off = 0;
  auto put = [&](const void* src, size_t sz) {   // src null: a region left zero
    if (sz && src) std::memcpy(host.data() + off, src, sz);
    void* dptr = static_cast<char*>(g->dmem) + off;
    off += align256(sz ? sz : 1);
    return dptr;
  };
  g->d_inst = static_cast<InstJob*>(put(inst.data(), sizeof(InstJob) * n));
  for (int st = 0; st < 5; ++st) g->d_gemm[st] = static_cast<tc::GemmJob*>(put(gj[st].data(), sizeof(tc::GemmJob) * n));
  for (size_t k = 0; k < tg.size(); ++k) {
    tg[k].njobs = static_cast<int>(tj[k].size());
    tg[k].d = static_cast<ThomasJob*>(put(tj[k].data(), sizeof(ThomasJob) * tj[k].size()));
  }
  for (size_t r = 0; r < rg.size(); ++r) {
    rg[r].njobs = static_cast<int>(rj[r].size());
    rg[r].d = static_cast<ResJob*>(put(rj[r].data(), sizeof(ResJob) * rj[r].size()));
  }
  g->d_counters = static_cast<int*>(put(nullptr, sizeof(int) * tg.size() * max_corr));
  // a solve still in flight on s may be reading the previous tables
  MX_CUDA(cudaStreamSynchronize(s));
  MX_CUDA(cudaMemcpyAsync(g->dmem, host.data(), bytes, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaStreamSynchronize(s));
  g->tg = tg;
  g->rg = rg;
  g->key = key;
  g->gens = gens;
  return TPT_OK;
}

// The grouped solve on stream s (tables from group_prepare): every instance's
// scalars cleared, f converted, corrections until each instance's rtol or the
// largest 1 + max_refine of the batch, the gauge and the float64 output, and
// the 16 scalars of instance i gathered into d_scal[16 i ..].
int group_corrections(const GroupSolve* g) {
  int corrections = 1;
  for (tpt_plan_s* p : g->plans) corrections = std::max(corrections, 1 + p->max_refine);
  return corrections;
}

// Corrections c0 .. c1 - 1 of the grouped solve, after the clearing and the
// conversion of f when `prepare`, followed by the gauge and the float64
// output when `output`; the 16 scalars of every instance are gathered into
// d_scal at the end either way.
int group_enqueue_part(GroupSolve* g, double* d_scal, cudaStream_t s, int c0, int c1, bool prepare, bool output) {
  if (c1 > 64) return TPT_ERR_UNSUPPORTED;
  const int n = g->n;
  if (prepare) {
    note_launch(2);
    group_clear_kernel<<<n, 32, 0, s>>>(g->d_inst);
    group_prepare_kernel<kFmtSplit><<<g->blocks[0], dim3(32, 8), 0, s>>>(g->d_inst, n);
    MX_CUDA(cudaGetLastError());
    MX_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(int) * g->tg.size() * 64, s));
  }
  for (int c = c0; c < c1; ++c) {
    for (int st : {0, 1}) MX_CUDA(tc::gemm_grouped(st == 1 ? tc::kOutF32 : tc::kOutSplitBF16, g->gemm_tma[st],
                                                  g->d_gemm[st], n, g->gemm_units[st], s));
    for (size_t k = 0; k < g->tg.size(); ++k)
      MX_CUDA(launch_thomas_m_group(g->tg[k], g->d_counters + 64 * k + c, g->dev, s));
    MX_CUDA(tc::gemm_grouped(tc::kOutSplitBF16, g->gemm_tma[2], g->d_gemm[2], n, g->gemm_units[2], s));
    const int xi = c == 0 ? 3 : 4;
    MX_CUDA(tc::gemm_grouped(tc::kOutDF, false, g->d_gemm[xi], n, g->gemm_units[xi], s));
    for (const auto& r : g->rg) MX_CUDA(launch_res_code(r, s));
    note_launch(1);
    group_converge_kernel<<<(n + 127) / 128, 128, 0, s>>>(g->d_inst, n);
    MX_CUDA(cudaGetLastError());
  }
  if (output) {
    note_launch(3);
    group_clear2_kernel<<<(n + 127) / 128, 128, 0, s>>>(g->d_inst, n);
    if (g->blocks[1] > 0) group_wsum_kernel<<<g->blocks[1], dim3(64, 4), 0, s>>>(g->d_inst, n);
    group_output_kernel<<<g->blocks[2], 256, 0, s>>>(g->d_inst, n);
  }
  note_launch(1);
  group_gather_kernel<<<n, 32, 0, s>>>(g->d_inst, d_scal);
  MX_CUDA(cudaGetLastError());
  return TPT_OK;
}

int group_enqueue(GroupSolve* g, double* d_scal, cudaStream_t s) {
  const unsigned long long before = launch_count();
  const int st = group_enqueue_part(g, d_scal, s, 0, group_corrections(g), true, true);
  g->kernels = launch_count() - before;
  return st;
}

int group_solve_adaptive(GroupSolve* g, double* d_scal, double* h_scal, cudaStream_t s) {
  const int n = g->n;
  const int corrections = std::min(64, group_corrections(g));
  int planned = 1;
  for (tpt_plan_s* p : g->plans) planned = std::max(planned, planned_corrections(p));
  planned = std::min(planned, corrections);
  auto fetch = [&]() -> int {
    MX_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(double) * 16 * n, cudaMemcpyDeviceToHost, s));
    MX_CUDA(cudaStreamSynchronize(s));
    return TPT_OK;
  };
  auto running = [&]() {
    for (int i = 0; i < n; ++i)
      if (reinterpret_cast<const int*>(h_scal + 16 * i + 8)[0] == 0) return true;
    return false;
  };
  MX_TRY(group_enqueue_part(g, d_scal, s, 0, planned, true, false));
  MX_TRY(fetch());
  int c = planned;
  while (c < corrections && running()) {   // the rest, one correction at a time
    MX_TRY(group_enqueue_part(g, d_scal, s, c, c + 1, false, false));
    MX_TRY(fetch());
    ++c;
  }
  MX_TRY(group_enqueue_part(g, d_scal, s, c, c, false, true));
  return fetch();
}

int autotune_gemms(tpt_plan_s* p, void* work, cudaStream_t s) {
  if (p->precision == TPT_PREC_FP64) return TPT_OK;
  MixedTables& m = p->mixed;
  const MixedWork w = carve(p, work);
  MX_CUDA(cudaMemsetAsync(work, 0, mixed_workspace_bytes(p), s));   // finite operands
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int status = TPT_OK;
  for (cudaEvent_t& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) status = TPT_ERR_CUDA;
  const int kind = kind_of(m.fmt), npl = nplanes(m.fmt);
  constexpr int kReps = 3, kRounds = 3;
  for (int i = 0; i < 4 && status == TPT_OK; ++i) {
    if (p->xform[stage_dir(i)] == TPT_XFORM_FFT) continue;   // no GEMM to tune
    const StageGemm t = stage_gemm(p, w, i, false);
    const int top = tc::default_bn(t.g.N);
    // the operand common to neighbouring tiles: the transform matrix, which
    // is B for the x forward and y inverse stages and A for the other two
    const int share = (i == 0 || i == 2) ? 1 : 2;
    int cbn[8], cpair[8], nc = 0;
    for (int cand = 0; cand < 8; ++cand) {
      const int bn = 32 << (cand / 2), pair = (cand % 2) ? share : 0;
      if (bn > top) break;
      if (pair && (m.fmt != kFmtSplit || bn < 128)) continue;
      cbn[nc] = bn;
      cpair[nc++] = pair;
    }
    // rounds over all candidates, keeping each candidate's fastest round, so
    // that a slow moment of the device does not decide for one candidate
    float tbest[8];
    for (int c = 0; c < nc; ++c) tbest[c] = -1.0f;
    for (int round = 0; round < kRounds && status == TPT_OK; ++round) {
      for (int c = 0; c < nc && status == TPT_OK; ++c) {
        tc::GemmOut g = t.g;
        g.bn = cbn[c];
        g.max_ctas = 0;
        g.pair = cpair[c];
        cudaError_t e = cudaSuccess;
        if (round == 0) e = tc::gemm(kind, npl, t.a, t.b, g, s);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        for (int r = 0; r < kReps && e == cudaSuccess; ++r) e = tc::gemm(kind, npl, t.a, t.b, g, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) {
          status = TPT_ERR_CUDA;
          break;
        }
        if (tbest[c] < 0.0f || ms < tbest[c]) tbest[c] = ms;
      }
    }
    // the default (widest tile, one CTA per tile) unless another candidate is
    // faster by more than 1 %
    int best_bn = top, best_pair = 0;
    float best = -1.0f;
    for (int c = 0; c < nc; ++c)
      if (cbn[c] == top && cpair[c] == 0) best = tbest[c];
    for (int c = 0; c < nc; ++c) {
      if (best < 0.0f || tbest[c] < 0.99f * best) {
        best = tbest[c];
        best_bn = cbn[c];
        best_pair = cpair[c];
      }
    }
    m.gemm_bn[i] = best_bn;
    m.gemm_ctas[i] = 0;
    m.gemm_pair[i] = best_pair;
  }
  for (cudaEvent_t& e : ev)
    if (e) cudaEventDestroy(e);
  if (status != TPT_OK) return status;
  int errflag = 0;
  MX_CUDA(cudaMemcpyAsync(&errflag, w.scal + 15, sizeof(int), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  ++p->generation;
  if (errflag) {   // a timed-out candidate aborts the ones after it, which then look fast
    for (int i = 0; i < 4; ++i) m.gemm_bn[i] = m.gemm_pair[i] = 0;
    return TPT_ERR_TIMEOUT;
  }
  return TPT_OK;
}

int mixed_info(const tpt_plan_s* p, const double* h, tpt_info* info) {
  int flags[2] = {0, 0};
  std::memcpy(flags, &h[8], sizeof(flags));
  if (flags[1] > 0) {   // decided on the device (converge_kernel): its count and sums
    const double rel = h[12] > 0.0 ? std::sqrt(h[11] / h[12]) : std::sqrt(h[11]);
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iters = flags[1];
      info->rel_residual = rel;
      info->compat_defect = p->singular ? h[7] / p->vol : 0.0;
    }
    if (flags[0] == 3) return TPT_ERR_TIMEOUT;
    if (flags[0] == 2) return TPT_ERR_NONFINITE;
    return flags[0] == 1 ? TPT_OK : TPT_ERR_NOT_CONVERGED;
  }
  int errflag = 0;
  std::memcpy(&errflag, &h[15], sizeof(int));
  const double np = static_cast<double>(npts(p));
  const double fn2 = proj_norm2(h, np, p->vol, p->singular);
  const double rel = fn2 > 0.0 ? std::sqrt(h[1] / fn2) : std::sqrt(h[1]);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = 1 + p->max_refine;
    info->rel_residual = rel;
    info->compat_defect = p->singular ? h[7] / p->vol : 0.0;
  }
  if (errflag) return TPT_ERR_TIMEOUT;
  if (!std::isfinite(rel)) return TPT_ERR_NONFINITE;
  if (p->rtol > 0.0 && !(rel <= p->rtol)) return TPT_ERR_NOT_CONVERGED;
  return TPT_OK;
}

int mixed_thomas_test(tpt_plan_s* p, const float* t2, void* t3_0, void* t3_1, void* work, cudaStream_t s) {
  if (!p || p->precision == TPT_PREC_FP64 || !t2 || !t3_0 || !work) return TPT_ERR_INVALID_ARG;
  if (p->mixed.fmt == kFmtSplit && !t3_1) return TPT_ERR_INVALID_ARG;
  MixedWork w = carve(p, work);
  MX_CUDA(cudaMemsetAsync(w.scal, 0, 256, s));   // stop flag, tile counter and error flag cleared
  w.B[0] = const_cast<float*>(t2);
  w.A[0] = t3_0;
  w.A[1] = t3_1;
  cudaError_t e;
  switch (p->mixed.fmt) {
    case kFmtSplit: e = launch_thomas<kFmtSplit>(p, w, s); break;
    case kFmtBF16: e = launch_thomas<kFmtBF16>(p, w, s); break;
    default: e = launch_thomas<kFmtF32>(p, w, s); break;
  }
  MX_CUDA(e);
  int errflag = 0;
  MX_CUDA(cudaMemcpyAsync(&errflag, w.scal + 15, sizeof(int), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  return errflag ? TPT_ERR_TIMEOUT : TPT_OK;
}

int tc_gemm_test(int precision, int M, int N, int K, const double* A, const double* B, double* D,
                 void* work, int dev, cudaStream_t s, int tile, int pair) {
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
  tc::GemmOut g = gout(M, N, K, kBig, 0, M, D, nullptr, tc::kOutF64, 0, 0, nullptr);
  g.bn = tile;
  g.pair = pair;
  MX_CUDA(tc::gemm(kind_of(fmt), nplanes(fmt), operand(pa, M, K, ld), operand(pb, N, K, ld), g, s));
  return TPT_OK;
}

int gemm_timeout_test(unsigned polls, void* work, int dev, cudaStream_t s) {
  if (!work || polls == 0) return TPT_ERR_INVALID_ARG;
  // a 256 x 256 x 64 bf16 GEMM whose producer issues no loads: the MMA
  // warp's and the epilogue's bounded waits run out, record their codes in
  // the error flag and return; nothing is read from the (valid) operands
  constexpr int M = 256, N = 256, K = 64;
  char* w = static_cast<char*>(work);
  int* err = reinterpret_cast<int*>(w);
  void* pa[2] = {w + 256, nullptr};
  void* pb[2] = {w + 256 + align256(2 * M * K), nullptr};
  void* out = w + 256 + align256(2 * M * K) + align256(2 * N * K);
  MX_CUDA(cudaMemsetAsync(work, 0, 256, s));
  tc::GemmOut g = gout(M, N, K, kBig, 0, M, out, nullptr, tc::kOutF32, 0, 0, err);
  g.polls = polls;
  g.drop_loads = 1;
  g.tma_out = 0;
  MX_CUDA(tc::gemm(tc::kKindBF16, 1, operand(pa, M, K, K), operand(pb, N, K, K), g, s));
  int h = 0;
  MX_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  (void)dev;
  return h ? TPT_ERR_TIMEOUT : TPT_OK;
}

int tc_gemm_out_test(int precision, int M, int N, int K, const double* A, const double* B, int out_kind,
                     int rm, long long sm, long long sn, void* out0, void* out1, void* work, int dev,
                     cudaStream_t s, int tile, int tma_out, int pair) {
  if (M <= 0 || N <= 0 || K <= 0 || rm <= 0 || !A || !B || !out0 || !work) return TPT_ERR_INVALID_ARG;
  if (precision < TPT_PREC_MIXED_BF16 || precision > TPT_PREC_MIXED_TF32) return TPT_ERR_INVALID_ARG;
  int mode;
  switch (out_kind) {
    case TPT_GEMM_OUT_F32: mode = tc::kOutF32; break;
    case TPT_GEMM_OUT_BF16: mode = tc::kOutBF16; break;
    case TPT_GEMM_OUT_SPLIT_BF16: mode = tc::kOutSplitBF16; break;
    default: return TPT_ERR_INVALID_ARG;
  }
  if (mode == tc::kOutSplitBF16 && !out1) return TPT_ERR_INVALID_ARG;
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
  tc::GemmOut g = gout(M, N, K, rm, sm, sn, out0, out1, mode, 0, 0, nullptr);
  g.bn = tile;
  g.tma_out = tma_out;
  g.pair = pair;
  MX_CUDA(tc::gemm(kind_of(fmt), nplanes(fmt), operand(pa, M, K, ld), operand(pb, N, K, ld), g, s));
  return TPT_OK;
}

}  // namespace tpt
