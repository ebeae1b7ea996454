// Tensor-core transform GEMM for sm_103a (tcgen05 + TMA + TMEM).
//
//   D[m, n] = sum_k A[m, k] * B[n, k]      (both operands K-major)
//
// is the building block of the low-precision eigenbasis transforms (Sec. 2.2.2,
// Eq. forward-xy / inverse-xy; lines stacked as one GEMM).  Operands are bf16
// (one plane, or a hi/lo pair whose three products hi*hi + hi*lo + lo*hi
// approximate the float32 product) or tf32 (float32 planes), accumulated in
// float32 in tensor memory.  The kernel is persistent (one CTA per SM walking
// 128 x BN tiles) with a double-buffered tensor-memory accumulator:
//   warp 0      TMA producer: A and B tiles of 128-byte rows, 128-byte swizzle,
//               into a ring of shared-memory stages (mbarrier full/empty);
//   warp 1      allocates BN tensor-memory columns and issues tcgen05.mma from
//               one thread, committing each stage back to the producer;
//   warps 2..5  epilogue: tcgen05.ld 32 columns at a time, convert, and store
//               with addresses idx(m, n) = (m % rm) + (m / rm) * sm + n * sn, so
//               consecutive lanes (consecutive m) write consecutive addresses.
// Every mbarrier wait is bounded; a timeout sets bits in *err and the CTA
// drains its copies, frees its tensor memory and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "ptx.h"
#include "tc.h"

namespace tpt {
namespace tc {
namespace {

constexpr int BM = 128;
// Threads of a CTA: a producer warp, an MMA warp and the epilogue warps.
// Epilogue warps: eight for the float-pair update (two warps per tensor-memory
// lane quarter, alternate 32-column chunks), so that twice as many
// read-modify-write loads are in flight; four otherwise.
template <int OUT>
__host__ __device__ constexpr int epi_warps() {
  return 8;
}
template <int OUT>
__host__ __device__ constexpr int threads_of() {
  return 32 * (2 + epi_warps<OUT>());
}
constexpr int kSmemBudget = 200 * 1024;

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// (s, e) with s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int KIND, int NPL, int BN>
struct Cfg {
  static constexpr int EB = (KIND == kKindBF16) ? 2 : 4;     // element bytes
  // bytes of a K-row of a stage: 64 (64-byte swizzle) for the split-bf16
  // 256-column tile, so that four stages fit instead of two; 128 otherwise
  static constexpr int SW = (NPL == 2 && BN == 256) ? 64 : 128;
  static constexpr int BK = SW / EB;                          // elements per row
  static constexpr int KI = (KIND == kKindBF16) ? 16 : 8;     // K of one MMA instruction
  static constexpr int A_BYTES = BM * SW;                     // one plane of A per stage
  static constexpr int B_BYTES = BN * SW;
  static constexpr int STAGE = NPL * (A_BYTES + B_BYTES);
  static constexpr int STAGES = (kSmemBudget / STAGE) > 4 ? 4 : (kSmemBudget / STAGE);
  static constexpr int TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;   // two accumulator buffers
  static constexpr int SMEM = STAGES * STAGE + 1024 /* alignment */ + 256 /* barriers */;
  // TMA-store epilogue: per epilogue warp two 32 x 32 chunks of up to 8 bytes
  // an element (split bf16: two 2-byte planes; float32: one 4-byte plane)
  static constexpr int OSTAGE = 4 * 2 * 32 * 32 * 4;
  static constexpr int SMEM_TMAO = STAGES * STAGE + 1024 + OSTAGE + 1024;
  static constexpr int NPROD = (NPL == 2) ? 3 : 1;
};

// Store one 32-column chunk of the accumulator (registers r) for row m.
template <int OUT>
// acc: add into the output (float-pair and float64 modes)
__device__ __forceinline__ void store_chunk(const GemmOut& g, long long mterm, int nb, const uint32_t (&r)[32],
                                            bool acc) {
  if (OUT == kOutDF) {
    // read-modify-write of the float pair: issue every load of the chunk
    // before any dependent arithmetic so the 64 loads overlap
    float* ph = static_cast<float*>(g.out0);
    float* pl = static_cast<float*>(g.out1);
    float oh[32], ol[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      const long long idx = mterm + static_cast<long long>(n < g.N ? n : 0) * g.sn;
      oh[j] = (acc && n < g.N) ? ph[idx] : 0.0f;
      ol[j] = (acc && n < g.N) ? pl[idx] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      if (n >= g.N) break;
      const long long idx = mterm + static_cast<long long>(n) * g.sn;
      float sh, se;
      two_sum(oh[j], __uint_as_float(r[j]), sh, se);
      se += ol[j];
      const float hi = sh + se;
      ph[idx] = hi;
      pl[idx] = se - (hi - sh);
    }
    return;
  }
  if (OUT == kOutF64 && acc) {
    // float64 read-modify-write (the levels of an Ozaki product): every load
    // of the chunk is issued before the first store, so the 32 loads overlap
    double* o = static_cast<double*>(g.out0);
    double old[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      old[j] = n < g.N ? o[mterm + static_cast<long long>(n) * g.sn] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      if (n >= g.N) break;
      o[mterm + static_cast<long long>(n) * g.sn] = old[j] + static_cast<double>(__uint_as_float(r[j]));
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int n = nb + j;
    if (n >= g.N) break;
    const long long idx = mterm + static_cast<long long>(n) * g.sn;
    const float v = __uint_as_float(r[j]);
    if (OUT == kOutSplitBF16) {
      __nv_bfloat16 hi, lo;
      split_bf16(v, hi, lo);
      static_cast<__nv_bfloat16*>(g.out0)[idx] = hi;
      static_cast<__nv_bfloat16*>(g.out1)[idx] = lo;
    } else if (OUT == kOutBF16) {
      static_cast<__nv_bfloat16*>(g.out0)[idx] = __float2bfloat16_rn(v);
    } else if (OUT == kOutF32) {
      static_cast<float*>(g.out0)[idx] = v;
    } else if (OUT == kOutF64) {
      static_cast<double*>(g.out0)[idx] = static_cast<double>(v);
    }
  }
}

template <int BN>
__device__ __forceinline__ void tile_coords(const GemmOut& g, int num_m, int num_n, long long tile,
                                            int& m0, int& n0) {
  int mt, nt;
  if (g.n_fastest) {
    nt = static_cast<int>(tile % num_n);
    mt = static_cast<int>(tile / num_n);
  } else {
    mt = static_cast<int>(tile % num_m);
    nt = static_cast<int>(tile / num_m);
  }
  m0 = mt * BM;
  n0 = nt * BN;
}

// Tile of work unit q for CTA rank r of a pair.  PAIR 0: one CTA per tile
// (q is the tile).  PAIR 1: the two CTAs of a cluster take the m-tiles 2mp and
// 2mp + 1 of one n-tile and share its B tile; PAIR 2: the n-tiles 2np and
// 2np + 1 of one m-tile, sharing its A tile.
template <int BN, int PAIR>
__device__ __forceinline__ void unit_coords(const GemmOut& g, int num_m, int num_n, long long q, int r, int& m0,
                                            int& n0) {
  if (PAIR == 0) {
    tile_coords<BN>(g, num_m, num_n, q, m0, n0);
  } else if (PAIR == 1) {
    const int num_mp = num_m / 2;
    const int nt = static_cast<int>(g.n_fastest ? q % num_n : q / num_mp);
    const int mp = static_cast<int>(g.n_fastest ? q / num_n : q % num_mp);
    m0 = (2 * mp + r) * BM;
    n0 = nt * BN;
  } else {
    const int num_np = num_n / 2;
    const int np = static_cast<int>(g.n_fastest ? q % num_np : q / num_m);
    const int mt = static_cast<int>(g.n_fastest ? q / num_np : q % num_m);
    m0 = mt * BM;
    n0 = (2 * np + r) * BN;
  }
}

// Persistent kernel: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  The tensor-memory accumulator is double-buffered (2 x BN columns): the
// MMA warp fills buffer b for tile t while the epilogue drains buffer b^1 of
// tile t-1.  Barriers: full/empty per smem stage (TMA <-> MMA), acc_full[b]
// (MMA -> epilogue, one commit) and acc_empty[b] (epilogue -> MMA, one arrive
// per epilogue warp).
//
// Grouped launches (MULTI = 1, one CTA per tile): the units are the tiles of
// every job of a device job table, in job order; a unit's job supplies its
// tensor maps, sizes, output and stop flag, and the units of a stopped job
// are passed over by all three roles alike.
template <int KIND, int NPL, int BN, int OUT, int PAIR, int TMAO, int MULTI = 0>
__global__ void __launch_bounds__(threads_of<OUT>(), 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
               const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB1,
               const __grid_constant__ CUtensorMap tO0, const __grid_constant__ CUtensorMap tO1,
               const GemmOut g, const GemmJob* __restrict__ jobs, int njobs, long long total_units) {
  static_assert(!MULTI || PAIR == 0, "grouped launches run one CTA per tile");
  if (!MULTI && g.skip && *g.skip) return;   // uniform over the grid: no barrier or TMEM is touched
  using C = Cfg<KIND, NPL, BN>;
  static_assert(C::STAGES >= 2, "shared-memory ring needs two stages");
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // 1024-byte aligned start, offset on the shared pointer itself so that the
  // epilogue's staging accesses stay shared-memory (not generic) accesses
  uint8_t* smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr int EPI = epi_warps<OUT>();
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  // bars[0..S) full, [S..2S) empty, [2S, 2S+2) acc_full, [2S+2, 2S+4) acc_empty,
  // [2S+4] mma_done (the issuer's last MMAs have completed)
  uint64_t* accf = bars + 2 * C::STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* mdone = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int num_m = (g.M + BM - 1) / BM, num_n = (g.N + BN - 1) / BN;
  const long long num_tiles = static_cast<long long>(num_m) * num_n;
  // work units: tiles, or tile pairs of a two-CTA cluster (the host checks
  // that the paired tile count is even)
  const long long num_units = MULTI ? total_units : (PAIR ? num_tiles / 2 : num_tiles);
  const long long unit0 = PAIR ? blockIdx.x / 2 : blockIdx.x;
  const long long unit_step = PAIR ? gridDim.x / 2 : gridDim.x;
  const int rank = PAIR ? static_cast<int>(ptx::cluster_ctarank()) : 0;
  constexpr uint16_t kPairMask = 0x3;
  const int nk = (g.K + C::BK - 1) / C::BK;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(g.err);
  const uint32_t polls = g.polls ? g.polls : (1u << 22);
  // unit q: its tile origin, K chunks, output description and tensor maps
  // (A0, A1, B0, B1, O0, O1); false when its job has stopped
  auto resolve = [&](long long q, int& m0, int& n0, int& nkq, const GemmOut*& gq,
                     const CUtensorMap*& mq) -> bool {
    if constexpr (MULTI) {
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (jobs[mid].first <= q) lo = mid;
        else hi = mid - 1;
      }
      const GemmJob& jb = jobs[lo];
      gq = &jb.g;
      mq = jb.map;
      if (gq->skip && *gq->skip) return false;
      tile_coords<BN>(*gq, jb.num_m, jb.num_n, q - jb.first, m0, n0);
      nkq = (gq->K + C::BK - 1) / C::BK;
    } else {
      gq = &g;
      mq = nullptr;
      unit_coords<BN, PAIR>(g, num_m, num_n, q, rank, m0, n0);
      nkq = nk;
    }
    return true;
  };
  // products per tile (float64 levels), K chunks of product lv and its B offset
  constexpr bool kLevels = OUT == kOutF64;
  auto npass_of = [&](const GemmOut& gg) -> int { return (kLevels && gg.levels > 0) ? gg.levels : 1; };
  auto nk_of = [&](const GemmOut& gg, int lv, int nkq) -> int {
    return (kLevels && gg.levels > 0) ? ((lv + 1) * gg.level_k) / C::BK : nkq;
  };
  auto bofs_of = [&](const GemmOut& gg, int lv) -> int {
    return (kLevels && gg.levels > 0) ? (gg.levels - 1 - lv) * gg.level_k : 0;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&bars[s]), 1);
      // a stage is free once the MMA of every CTA that reads it has finished
      ptx::mbar_init(ptx::smem_u32(&bars[C::STAGES + s]), PAIR ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_u32(&accf[b]), 1);
      ptx::mbar_init(ptx::smem_u32(&acce[b]), EPI);
    }
    ptx::mbar_init(ptx::smem_u32(mdone), 1);
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (PAIR) ptx::cluster_sync();   // the peer's barriers exist before any remote arrive
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- TMA producer
    if (!MULTI) {
      ptx::prefetch_tmap(&tA0);
      ptx::prefetch_tmap(&tB0);
      if (NPL == 2) {
        ptx::prefetch_tmap(&tA1);
        ptx::prefetch_tmap(&tB1);
      }
    }
    bool ok = true;
    long long it = 0;
    int* last_err = g.err;
    for (long long q = unit0; q < num_units && ok; q += unit_step) {
      int m0, n0, nkq;
      const GemmOut* gq;
      const CUtensorMap* mq;
      if (!resolve(q, m0, n0, nkq, gq, mq)) continue;
      const CUtensorMap* mA0 = MULTI ? &mq[0] : &tA0;
      const CUtensorMap* mA1 = MULTI ? &mq[1] : &tA1;
      const CUtensorMap* mB0 = MULTI ? &mq[2] : &tB0;
      const CUtensorMap* mB1 = MULTI ? &mq[3] : &tB1;
      volatile int* abort_q = MULTI ? reinterpret_cast<volatile int*>(gq->err) : abort_flag;
      last_err = gq->err;
      const int npass = npass_of(*gq);
      for (int lv = 0; lv < npass && ok; ++lv) {
      const int nkp = nk_of(*gq, lv, nkq), kb = bofs_of(*gq, lv);
      for (int kc = 0; kc < nkp; ++kc, ++it) {
        const int s = static_cast<int>(it % C::STAGES);
        const long long round = it / C::STAGES;
        if (round > 0)
          ok = ptx::mbar_wait(ptx::smem_u32(&bars[C::STAGES + s]), static_cast<uint32_t>((round - 1) & 1), gq->err,
                              ptx::kErrWaitEmpty, polls);
        if (!ok || (abort_q && *abort_q)) {
          ok = false;
          break;
        }
        if (g.drop_loads) {      // failure-detection test: no stage ever fills
          ok = false;
          break;
        }
        uint8_t* st = smem + s * C::STAGE;
        const uint32_t full = ptx::smem_u32(&bars[s]);
        ptx::mbar_arrive_expect_tx(full, C::STAGE);
        const int kx = kc * C::BK, kxb = kx + kb;
        if (PAIR == 1) {          // own A; half of the shared B tile, to both CTAs
          const int hb = BN / 2;
          ptx::tma_load_2d(ptx::smem_u32(st), mA0, full, kx, m0);   // n0: the pair's common n-tile
          ptx::tma_load_2d_mc(ptx::smem_u32(st + NPL * C::A_BYTES + rank * hb * C::SW), mB0, full, kxb,
                              n0 + rank * hb, kPairMask);
          if (NPL == 2) {
            ptx::tma_load_2d(ptx::smem_u32(st + C::A_BYTES), mA1, full, kx, m0);
            ptx::tma_load_2d_mc(ptx::smem_u32(st + NPL * C::A_BYTES + C::B_BYTES + rank * hb * C::SW), mB1, full,
                                kxb, n0 + rank * hb, kPairMask);
          }
        } else if (PAIR == 2) {   // half of the shared A tile, to both CTAs; own B
          const int ha = BM / 2;
          ptx::tma_load_2d_mc(ptx::smem_u32(st + rank * ha * C::SW), mA0, full, kx, m0 + rank * ha, kPairMask);
          ptx::tma_load_2d(ptx::smem_u32(st + NPL * C::A_BYTES), mB0, full, kxb, n0);
          if (NPL == 2) {
            ptx::tma_load_2d_mc(ptx::smem_u32(st + C::A_BYTES + rank * ha * C::SW), mA1, full, kx, m0 + rank * ha,
                                kPairMask);
            ptx::tma_load_2d(ptx::smem_u32(st + NPL * C::A_BYTES + C::B_BYTES), mB1, full, kxb, n0);
          }
        } else {
          ptx::tma_load_2d(ptx::smem_u32(st), mA0, full, kx, m0);
          ptx::tma_load_2d(ptx::smem_u32(st + NPL * C::A_BYTES), mB0, full, kxb, n0);
          if (NPL == 2) {
            ptx::tma_load_2d(ptx::smem_u32(st + C::A_BYTES), mA1, full, kx, m0);
            ptx::tma_load_2d(ptx::smem_u32(st + NPL * C::A_BYTES + C::B_BYTES), mB1, full, kxb, n0);
          }
        }
      }
      }
    }
    // drain: every issued stage's copies have landed before the CTA may exit
    // (the same bound as the main waits; a timed-out drain is recorded in
    // g.err, and every caller then treats the output as invalid)
    const long long first = it > C::STAGES ? it - C::STAGES : 0;
    for (long long k = first; k < it; ++k)
      ptx::mbar_wait(ptx::smem_u32(&bars[k % C::STAGES]), static_cast<uint32_t>((k / C::STAGES) & 1), last_err,
                     ptx::kErrWaitDrain, polls);
  } else if (warp == 1 && lane == 0) {
    // -------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = ptx::instr_desc(KIND == kKindBF16 ? 1u : 2u, BM, BN);
    bool ok = true;
    long long it = 0;
    int tcount = 0;
    int* last_err = g.err;
    for (long long q = unit0; q < num_units && ok; q += unit_step) {
      int m0, n0, nkq;
      const GemmOut* gq;
      const CUtensorMap* mq;
      if (!resolve(q, m0, n0, nkq, gq, mq)) continue;
      volatile int* abort_q = MULTI ? reinterpret_cast<volatile int*>(gq->err) : abort_flag;
      last_err = gq->err;
      const int npass = npass_of(*gq);
      for (int lv = 0; lv < npass && ok; ++lv) {
      const int nkp = nk_of(*gq, lv, nkq);
      const int b = tcount & 1, use = tcount >> 1;
      ++tcount;
      if (use > 0)
        ok = ptx::mbar_wait(ptx::smem_u32(&acce[b]), static_cast<uint32_t>((use - 1) & 1), gq->err,
                            ptx::kErrWaitAccum, polls);
      if (!ok || (abort_q && *abort_q)) {
        ok = false;
        break;
      }
      ptx::tc_fence_after();
      const uint32_t d = tmem + static_cast<uint32_t>(b * BN);
      for (int kc = 0; kc < nkp; ++kc, ++it) {
        const int s = static_cast<int>(it % C::STAGES);
        ok = ptx::mbar_wait(ptx::smem_u32(&bars[s]), static_cast<uint32_t>((it / C::STAGES) & 1), gq->err,
                            ptx::kErrWaitFull, polls);
        if (!ok) break;
        ptx::tc_fence_after();
        const uint32_t sa = ptx::smem_u32(smem + s * C::STAGE);
        const uint32_t sb = sa + NPL * C::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < C::BK / C::KI; ++kk) {
          const uint32_t off = kk * C::KI * C::EB;   // bytes along the 128-byte row
#pragma unroll
          for (int p = 0; p < C::NPROD; ++p) {
            // products: (A0,B0), (A0,B1), (A1,B0)
            const uint32_t a = sa + (p == 2 ? C::A_BYTES : 0) + off;
            const uint32_t bb = sb + (p == 1 ? C::B_BYTES : 0) + off;
            const uint32_t acc = (kc > 0 || kk > 0 || p > 0) ? 1u : 0u;
            if (KIND == kKindBF16)
              ptx::mma_bf16(d, ptx::smem_desc_k_sw<C::SW>(a), ptx::smem_desc_k_sw<C::SW>(bb), idesc, acc);
            else
              ptx::mma_tf32(d, ptx::smem_desc_k_sw<C::SW>(a), ptx::smem_desc_k_sw<C::SW>(bb), idesc, acc);
          }
        }
        if (PAIR) ptx::mma_commit_mc(ptx::smem_u32(&bars[C::STAGES + s]), kPairMask);   // frees the stage
        else ptx::mma_commit(ptx::smem_u32(&bars[C::STAGES + s]));                  // in both CTAs
      }
      ptx::mma_commit(ptx::smem_u32(&accf[b]));                 // accumulator b ready
      }
    }
    // every MMA this thread issued has completed before the tensor memory is
    // freed, also when a timed-out wait ended the loop early
    if (it > 0) {
      ptx::mma_commit(ptx::smem_u32(mdone));
      ptx::mbar_wait(ptx::smem_u32(mdone), 0u, last_err, ptx::kErrWaitDrain, polls);
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int quarter = warp % 4;                  // tensor-memory lanes 32*quarter ..
    const int half = (warp - 2) / 4;               // eight warps: chunks of parity `half`
    // TMA-store epilogue: each 32-row x 32-column chunk is written to a
    // shared-memory staging buffer (column-major, rows contiguous, as in the
    // output) and stored by one lane with a 3D bulk tensor store, two chunks
    // in flight per warp
    constexpr int OEB = (OUT == kOutF32) ? 4 : 2;
    constexpr int ONPL = (OUT == kOutSplitBF16) ? 2 : 1;
    constexpr int CHUNK = 32 * 32 * OEB;           // one plane of a chunk
    uint8_t* ostage = smem + C::STAGES * C::STAGE + 1024 + (warp - 2) * (ONPL * CHUNK);
    int chunk_i = 0;
    int tcount = 0;
    bool go = true;
    for (long long q = unit0; q < num_units && go; q += unit_step) {
      int m0, n0, nkq;
      const GemmOut* gq;
      const CUtensorMap* mq;
      if (!resolve(q, m0, n0, nkq, gq, mq)) continue;
      const GemmOut& gu = *gq;
      const CUtensorMap* mO0 = MULTI ? &mq[4] : &tO0;
      const CUtensorMap* mO1 = MULTI ? &mq[5] : &tO1;
      volatile int* abort_q = MULTI ? reinterpret_cast<volatile int*>(gu.err) : abort_flag;
      const int npass = npass_of(gu);
      for (int lv = 0; lv < npass; ++lv) {
      const bool acc_out = gu.accumulate != 0 || lv > 0;   // later levels add to the earlier ones
      const int b = tcount & 1, use = tcount >> 1;
      ++tcount;
      const bool ok = ptx::mbar_wait(ptx::smem_u32(&accf[b]), static_cast<uint32_t>(use & 1), gu.err,
                                     ptx::kErrWaitAccum, polls);
      ptx::tc_fence_after();
      const bool flagged = abort_q && *abort_q;
      // tcgen05.ld is warp-collective: decide for the whole warp
      if (!__all_sync(0xffffffffu, ok && !flagged)) {
        go = false;
        break;
      }
      const int m = m0 + quarter * 32 + lane;
      const bool mvalid = m < gu.M;
      const long long mterm =
          mvalid ? (static_cast<long long>(m % gu.rm) + static_cast<long long>(m / gu.rm) * gu.sm) : 0;
#pragma unroll 1
      for (int c0 = 32 * half; c0 < BN; c0 += 32 * (EPI / 4)) {
        uint32_t r[32];
        ptx::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                    static_cast<uint32_t>(b * BN + c0), r);
        ptx::tmem_ld_wait();
        if (TMAO) {
          if (chunk_i >= 1) {                      // the store of chunk i-1 has left the buffer
            if (lane == 0) ptx::bulk_wait_read<0>();
            __syncwarp();
          }
          uint8_t* sb = ostage;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float v = __uint_as_float(r[j]);
            const int e = j * 32 + lane;
            if (OUT == kOutSplitBF16) {
              __nv_bfloat16 hi, lo;
              split_bf16(v, hi, lo);
              reinterpret_cast<__nv_bfloat16*>(sb)[e] = hi;
              reinterpret_cast<__nv_bfloat16*>(sb + CHUNK)[e] = lo;
            } else if (OUT == kOutBF16) {
              reinterpret_cast<__nv_bfloat16*>(sb)[e] = __float2bfloat16_rn(v);
            } else {
              reinterpret_cast<float*>(sb)[e] = v;
            }
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          const int mc = m0 + quarter * 32;        // first row of the chunk
          if (lane == 0 && mc < gu.M && n0 + c0 < gu.N) {
            // boxes start inside the tensor; the TMA unit clips their far
            // edges.  x stays a multiple of 32 elements: rm is a multiple of
            // 32, or the output is one block of rows (x = m, z = 0)
            const bool flat = gu.rm >= gu.M;
            const int x = flat ? mc : mc % gu.rm, z = flat ? 0 : mc / gu.rm;
            ptx::tma_store_3d(mO0, ptx::smem_u32(sb), x, n0 + c0, z);
            if (ONPL == 2) ptx::tma_store_3d(mO1, ptx::smem_u32(sb + CHUNK), x, n0 + c0, z);
            ptx::bulk_commit();
          }
          ++chunk_i;
        } else if (mvalid) {
          store_chunk<OUT>(gu, mterm, n0 + c0, r, acc_out);
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce[b]));   // buffer b may be refilled
      }
    }
    if (TMAO && lane == 0) ptx::bulk_wait_all();   // staging buffers stay until the stores are done
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (PAIR) ptx::cluster_sync();   // no CTA leaves while its peer may still signal it
  if (warp == 1) ptx::tmem_dealloc(tmem, C::TMEM_COLS);
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// K-major operand plane: rows x K elements, row stride ld elements; box of
// (sw-byte row) x box_rows with the sw-byte swizzle (sw = 64 or 128).
bool make_map(CUtensorMap* map, const void* base, int kind, int rows, int K, int ld, int box_rows, int sw) {
  auto fn = encode_fn();
  if (!fn || !base) return false;
  const int eb = (kind == kKindBF16) ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (static_cast<long long>(ld) * eb) % 16 != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * eb};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(sw / eb), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      (kind == kKindBF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Output tensor of the TMA-store epilogue: element (m, n) at (m % rm) +
// (m / rm) sm + n sn is the 3D tensor {rm, N, M / rm} with strides (sn, sm)
// (a single block of rows when rm >= M), box 32 x 32 x 1.
bool make_out_map(CUtensorMap* map, void* base, int eb, const GemmOut& g) {
  auto fn = encode_fn();
  if (!fn || !base) return false;
  const bool flat = g.rm >= g.M;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(flat ? g.M : g.rm), static_cast<cuuint64_t>(g.N),
                        static_cast<cuuint64_t>(flat ? 1 : g.M / g.rm)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(g.sn) * eb,
                           static_cast<cuuint64_t>(flat ? g.sn * g.N : g.sm) * eb};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || strides[0] % 16 != 0 || strides[1] % 16 != 0) return false;
  std::memset(map, 0, sizeof(*map));
  CUresult r = fn(map, eb == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int KIND, int NPL, int BN, int OUT, int PAIR, int TMAO = 0>
cudaError_t launch(const Operand& A, const Operand& B, const GemmOut& g, cudaStream_t s) {
  using C = Cfg<KIND, NPL, BN>;
  CUtensorMap m[6];
  std::memset(m, 0, sizeof(m));
  if (TMAO) {
    // layouts the tensor map cannot describe (unaligned base or strides) take
    // the direct-store epilogue
    const int eb = (OUT == kOutF32) ? 4 : 2;
    if (!make_out_map(&m[4], g.out0, eb, g)) return launch<KIND, NPL, BN, OUT, PAIR, 0>(A, B, g, s);
    if (OUT == kOutSplitBF16) {
      if (!make_out_map(&m[5], g.out1, eb, g)) return launch<KIND, NPL, BN, OUT, PAIR, 0>(A, B, g, s);
    } else {
      m[5] = m[4];
    }
  }
  // the shared operand of a pair is loaded in halves (one per CTA)
  const int a_rows = PAIR == 2 ? BM / 2 : BM, b_rows = PAIR == 1 ? BN / 2 : BN;
  if (!make_map(&m[0], A.plane[0], KIND, A.rows, A.K, A.ld, a_rows, C::SW)) return cudaErrorInvalidValue;
  if (!make_map(&m[2], B.plane[0], KIND, B.rows, B.K, B.ld, b_rows, C::SW)) return cudaErrorInvalidValue;
  if (NPL == 2) {
    if (!make_map(&m[1], A.plane[1], KIND, A.rows, A.K, A.ld, a_rows, C::SW)) return cudaErrorInvalidValue;
    if (!make_map(&m[3], B.plane[1], KIND, B.rows, B.K, B.ld, b_rows, C::SW)) return cudaErrorInvalidValue;
  } else {
    m[1] = m[0];
    m[3] = m[2];
  }
  auto kern = gemm_tc_kernel<KIND, NPL, BN, OUT, PAIR, TMAO>;
  const int smem_bytes = TMAO ? C::SMEM_TMAO : C::SMEM;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  const long long tiles = static_cast<long long>((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
  if (tiles <= 0) return cudaSuccess;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long cap = (g.max_ctas > 0 && g.max_ctas < sms) ? g.max_ctas : sms;
  if (PAIR == 0) {
    const long long ctas = tiles < cap ? tiles : cap;   // persistent: one CTA per SM
    note_launch(1);
    kern<<<static_cast<unsigned>(ctas), threads_of<OUT>(), smem_bytes, s>>>(m[0], m[1], m[2], m[3], m[4], m[5], g,
                                                                           nullptr, 0, 0LL);
    return cudaGetLastError();
  }
  // clusters of two CTAs, as many as can be resident at once (one CTA per SM)
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads_of<OUT>(), 1, 1);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  long long pairs = (cap / 2 < tiles / 2) ? cap / 2 : tiles / 2;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * pairs), 1, 1);
  int resident = 0;
  if (cudaOccupancyMaxActiveClusters(&resident, kern, &cfg) == cudaSuccess && resident > 0 && resident < pairs)
    pairs = resident;
  cudaGetLastError();
  cfg.gridDim = dim3(static_cast<unsigned>(2 * pairs), 1, 1);
  note_launch(1);
  e = cudaLaunchKernelEx(&cfg, kern, m[0], m[1], m[2], m[3], m[4], m[5], g, static_cast<const GemmJob*>(nullptr), 0,
                         0LL);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Pair mode g.pair when it applies (split bf16 operands, 128- or 256-column
// tiles, an even number of m-tiles (pair 1) or n-tiles (pair 2), an output
// mode instantiated for it, and both operands in the current device's own
// memory, since the pair's shared tile is loaded by a cluster-multicast TMA
// copy), else a single CTA per tile.
template <int KIND, int NPL, int BN, int OUT>
cudaError_t launch_pair(const Operand& A, const Operand& B, const GemmOut& g, cudaStream_t s) {
  const int num_m = (g.M + BM - 1) / BM, num_n = (g.N + BN - 1) / BN;
  if (g.pair != 0) {
    bool local = true;
    for (int pl = 0; pl < NPL; ++pl) local = local && own_device_memory(A.plane[pl]) && own_device_memory(B.plane[pl]);
    if (!local) {
      GemmOut g1 = g;
      g1.pair = 0;
      return launch_pair<KIND, NPL, BN, OUT>(A, B, g1, s);
    }
  }
  constexpr bool can1 = NPL == 2 && BN >= 128 &&
                        (OUT == kOutSplitBF16 || OUT == kOutBF16 || OUT == kOutF32 || OUT == kOutF64);
  constexpr bool can2 = NPL == 2 && BN >= 128 && (OUT == kOutF32 || OUT == kOutDF || OUT == kOutF64);
  // TMA-store epilogue when the output is a plain block of rows or whole
  // 32-row chunks of rm-row blocks
  constexpr bool cant = OUT == kOutSplitBF16 || OUT == kOutBF16 || OUT == kOutF32;
  const bool tma = cant && g.tma_out && (g.rm >= g.M || (g.rm % 32 == 0 && g.M % g.rm == 0));
  if (g.pair == 1 && can1 && num_m % 2 == 0)
    return tma ? launch<KIND, NPL, BN, OUT, can1 ? 1 : 0, cant ? 1 : 0>(A, B, g, s)
               : launch<KIND, NPL, BN, OUT, can1 ? 1 : 0>(A, B, g, s);
  if (g.pair == 2 && can2 && num_n % 2 == 0)
    return tma ? launch<KIND, NPL, BN, OUT, can2 ? 2 : 0, cant ? 1 : 0>(A, B, g, s)
               : launch<KIND, NPL, BN, OUT, can2 ? 2 : 0>(A, B, g, s);
  if (tma) return launch<KIND, NPL, BN, OUT, 0, cant ? 1 : 0>(A, B, g, s);
  return launch<KIND, NPL, BN, OUT, 0>(A, B, g, s);
}

template <int KIND, int NPL, int OUT>
cudaError_t launch_bn(const Operand& A, const Operand& B, const GemmOut& g, cudaStream_t s) {
  switch (g.bn ? g.bn : default_bn(g.N)) {
    case 32: return launch<KIND, NPL, 32, OUT, 0>(A, B, g, s);
    case 64: return launch<KIND, NPL, 64, OUT, 0>(A, B, g, s);
    case 128: return launch_pair<KIND, NPL, 128, OUT>(A, B, g, s);
    case 256: return launch_pair<KIND, NPL, 256, OUT>(A, B, g, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int KIND, int NPL>
cudaError_t launch_out(const Operand& A, const Operand& B, const GemmOut& g, cudaStream_t s) {
  switch (g.mode) {
    case kOutSplitBF16: return launch_bn<KIND, NPL, kOutSplitBF16>(A, B, g, s);
    case kOutBF16: return launch_bn<KIND, NPL, kOutBF16>(A, B, g, s);
    case kOutF32: return launch_bn<KIND, NPL, kOutF32>(A, B, g, s);
    case kOutF64: return launch_bn<KIND, NPL, kOutF64>(A, B, g, s);
    case kOutDF: return launch_bn<KIND, NPL, kOutDF>(A, B, g, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool make_plain_map(CUtensorMap* map, const void* base, int elem_bytes, long long inner, long long outer,
                    long long row_stride_bytes, int box_inner, int box_outer) {
  auto fn = encode_fn();
  if (!fn || !base || (elem_bytes != 2 && elem_bytes != 4)) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || row_stride_bytes % 16 != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_stride_bytes)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_inner), static_cast<cuuint32_t>(box_outer)};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  std::memset(map, 0, sizeof(*map));
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

template <int OUT, int TMAO>
cudaError_t launch_grouped(const GemmJob* d_jobs, int njobs, long long units, cudaStream_t s) {
  using C = Cfg<kKindBF16, 2, 256>;
  auto kern = gemm_tc_kernel<kKindBF16, 2, 256, OUT, 0, TMAO, 1>;
  const int smem_bytes = TMAO ? C::SMEM_TMAO : C::SMEM;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  if (units <= 0 || njobs <= 0) return cudaSuccess;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ctas = units < sms ? units : sms;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  GemmOut g0;
  std::memset(&g0, 0, sizeof(g0));
  note_launch(1);
  kern<<<static_cast<unsigned>(ctas), threads_of<OUT>(), smem_bytes, s>>>(none, none, none, none, none, none, g0,
                                                                         d_jobs, njobs, units);
  return cudaGetLastError();
}

}  // namespace

long long job_units(const GemmOut& g) {
  return static_cast<long long>((g.M + BM - 1) / BM) * ((g.N + 255) / 256);
}

bool make_job(const Operand& A, const Operand& B, const GemmOut& g, bool tma_out, GemmJob* job, long long first) {
  using C = Cfg<kKindBF16, 2, 256>;
  std::memset(job, 0, sizeof(*job));
  if (A.K != B.K || A.rows != g.M || B.rows != g.N || g.M <= 0 || g.N <= 0 || A.K <= 0 || g.rm <= 0) return false;
  if (!make_map(&job->map[0], A.plane[0], kKindBF16, A.rows, A.K, A.ld, BM, C::SW)) return false;
  if (!make_map(&job->map[1], A.plane[1], kKindBF16, A.rows, A.K, A.ld, BM, C::SW)) return false;
  if (!make_map(&job->map[2], B.plane[0], kKindBF16, B.rows, B.K, B.ld, 256, C::SW)) return false;
  if (!make_map(&job->map[3], B.plane[1], kKindBF16, B.rows, B.K, B.ld, 256, C::SW)) return false;
  if (tma_out) {
    const int eb = (g.mode == kOutF32) ? 4 : 2;
    if (!(g.rm >= g.M || (g.rm % 32 == 0 && g.M % g.rm == 0))) return false;
    if (!make_out_map(&job->map[4], g.out0, eb, g)) return false;
    if (g.mode == kOutSplitBF16) {
      if (!make_out_map(&job->map[5], g.out1, eb, g)) return false;
    } else {
      job->map[5] = job->map[4];
    }
  }
  job->g = g;
  job->first = first;
  job->num_m = (g.M + BM - 1) / BM;
  job->num_n = (g.N + 255) / 256;
  return true;
}

cudaError_t gemm_grouped(int mode, bool tma_out, const GemmJob* d_jobs, int njobs, long long units,
                         cudaStream_t s) {
  switch (mode) {
    case kOutSplitBF16:
      return tma_out ? launch_grouped<kOutSplitBF16, 1>(d_jobs, njobs, units, s)
                     : launch_grouped<kOutSplitBF16, 0>(d_jobs, njobs, units, s);
    case kOutF32:
      return tma_out ? launch_grouped<kOutF32, 1>(d_jobs, njobs, units, s)
                     : launch_grouped<kOutF32, 0>(d_jobs, njobs, units, s);
    case kOutDF: return launch_grouped<kOutDF, 0>(d_jobs, njobs, units, s);
    default: return cudaErrorInvalidValue;
  }
}

bool own_device_memory(const void* p) {
  int dev = -1;
  if (!p || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int default_bn(int N) { return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256; }

cudaError_t gemm(int kind, int nplanes, const Operand& A, const Operand& B, const GemmOut& g,
                 cudaStream_t s) {
  if (A.K != B.K || A.rows != g.M || B.rows != g.N || g.M <= 0 || g.N <= 0 || A.K <= 0 || g.rm <= 0)
    return cudaErrorInvalidValue;
  if (kind == kKindBF16 && nplanes == 1) return launch_out<kKindBF16, 1>(A, B, g, s);
  if (kind == kKindBF16 && nplanes == 2) return launch_out<kKindBF16, 2>(A, B, g, s);
  if (kind == kKindTF32 && nplanes == 1) return launch_out<kKindTF32, 1>(A, B, g, s);
  return cudaErrorInvalidValue;
}

}  // namespace tc
}  // namespace tpt
