// Host interface of the tensor-core transform GEMM (gemm_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace tpt {

void note_launch(unsigned long long k);

namespace tc {

enum { kKindBF16 = 0, kKindTF32 = 1 };
enum { kOutSplitBF16 = 0, kOutBF16 = 1, kOutF32 = 2, kOutF64 = 3, kOutDF = 4 };

// K-major operand: `rows` rows of K elements, row stride `ld` elements; one
// plane, or a hi/lo pair of bf16 planes.  Base addresses 16-byte aligned and
// ld * element size a multiple of 16 bytes.
struct Operand {
  const void* plane[2];
  int rows, K, ld;
};

// Output of D = A B^T (M x N): element (m, n) goes to
//   idx = (m % rm) + (m / rm) * sm + n * sn
// of out0 (and out1 for the split-bf16 and float-pair modes).
struct GemmOut {
  int M, N, K;
  int rm;
  long long sm, sn;
  void* out0;
  void* out1;
  int mode;
  int accumulate;   // float-pair and float64 modes: add into the output instead of writing
  int n_fastest;    // tile order: n fastest (A tile reused by consecutive CTAs)
  int* err;         // device flag for timed-out waits (may be null)
  int bn = 0;       // column tile width 32/64/128/256; 0 picks the smallest >= N
  int max_ctas = 0; // cap on the persistent CTAs; 0 = one per SM
  int pair = 0;     // two-CTA clusters sharing an operand tile by TMA multicast:
                    // 1 = pairs of m-tiles share B, 2 = pairs of n-tiles share A
  int tma_out = 1;  // TMA-store epilogue where the output layout allows (split bf16,
                    // bf16 or float32 out, 128/256-column tiles, one CTA per tile)
  const int* skip = nullptr;   // device flag: the kernel returns at entry when it is nonzero
  // Failure-detection tests only: polls of every bounded wait (0 = the
  // default, about 2^22) and a producer that issues no loads, so that the
  // waits run out and the kernel returns with TPT_ERR_TIMEOUT in *err.
  unsigned polls = 0;
  int drop_loads = 0;
  // Float64 output only: `levels` > 0 makes every tile a sequence of that
  // many products accumulated into the output, product l over K = (l + 1) *
  // level_k with A from K offset 0 and B from K offset (levels - 1 - l) *
  // level_k (the levels of an Ozaki product, from operands holding all the
  // slices); level_k a multiple of the 64-element K chunk.
  int levels = 0;
  int level_k = 0;
};

// One GEMM of a grouped launch: its tensor maps (A0, A1, B0, B1, O0, O1; the
// output maps only for the TMA-store epilogue), its output description, its
// first unit in the launch's list of tiles and its tile counts.  Kept in
// device memory.
struct GemmJob {
  CUtensorMap map[6];
  GemmOut g;
  long long first;
  int num_m, num_n;
};

// True when p points into device memory of the current device (not host,
// managed or another GPU's memory).  Operand sharing between the two CTAs of
// a pair (TMA multicast) is used only when every operand plane passes.
bool own_device_memory(const void* p);

// Column tile width used when GemmOut::bn is 0.
int default_bn(int N);

// Unswizzled 2D tensor map over `outer` rows of `inner` elements (2-byte
// bf16 or 4-byte float32), row stride in bytes, box of box_inner x
// box_outer elements.  False when the driver entry point is missing or the
// encoder rejects the layout (base or stride not 16-byte aligned, box too large).
bool make_plain_map(CUtensorMap* map, const void* base, int elem_bytes, long long inner, long long outer,
                    long long row_stride_bytes, int box_inner, int box_outer);

cudaError_t gemm(int kind, int nplanes, const Operand& A, const Operand& B, const GemmOut& g,
                 cudaStream_t s);

// Grouped launches of split-bf16 GEMMs (two planes, three products) with
// 256-column tiles: make_job fills one job on the host (false if an operand
// or the output cannot be described by tensor maps); gemm_grouped launches
// one persistent kernel over the tiles of `njobs` jobs already copied to
// device memory (`d_jobs`), whose units are claimed round-robin.  The output
// mode (g.mode) and tma_out must be the same for every job of a launch.
bool make_job(const Operand& A, const Operand& B, const GemmOut& g, bool tma_out, GemmJob* job,
              long long first);
long long job_units(const GemmOut& g);
cudaError_t gemm_grouped(int mode, bool tma_out, const GemmJob* d_jobs, int njobs, long long units,
                         cudaStream_t s);

}  // namespace tc
}  // namespace tpt
