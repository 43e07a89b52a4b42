// Host-side interface between the C ABI (ctaux_api.cu) and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "ctaux_dev.cuh"

namespace ctaux {

constexpr int kMaxPartials = 4096;  // split-K partial tiles per (chain, spin) and product
constexpr int kMaxMatsFreq = 64;    // Matsubara frequencies of the G(iw) measurement
constexpr int kMaxMatsSites = 1024; // cluster sites of the G(iw) measurement
constexpr int kTieSlices = 64;   // column slices of the near-tie matrix-vector products
// vertices per measurement evaluation chunk: small orders get short chunks
// (more work items for the GPU), large ones longer chunks (fewer partial sums)
constexpr int kMeasChunk = 16;      // the shortest chunk (sizes the partial-sum buffers)
constexpr int kMeasChunkMax = 32;
__host__ __device__ inline int meas_chunk(int n) { return n <= 1024 ? kMeasChunk : kMeasChunkMax; }

// tensor-core flush (mixed form): 128 x 128 output tiles, K chunks of 16 float32;
// the gathered N[S_m][S_n] input of a tile is staged as 128 column segments of
// kTcNsRows source rows
constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 16, kTcStages = 4, kTcThreads = 384;
constexpr int kTcNsRows = 160;

// TMA descriptors of one (chain, spin): split Y (rows a), split X (rows b) and
// both buffers of N, as column segments of kTcNsRows rows, one column (nb1)
// or kTcNsGroup adjacent columns (nbg) per box
constexpr int kTcNsGroup = 8;
struct TcMaps {
  CUtensorMap yh, yl, xh, xl;
  CUtensorMap nb1[2], nbg[2];
  // tensor-core prep: the panels' rows and N, N^T as K-major rows (boxes of
  // 128 rows x kTcBK float32, 64-byte swizzle)
  CUtensorMap cpan, bpan, nb[2], nt[2];
};

enum { PH_RTILDE = 0, PH_GCOL_OLD = 1, PH_GCOL_NEW = 2, PH_FLUSH = 3, PH_MEAS = 4, PH_COUNT = 5 };

// Output tile of each product (rows x columns, per thread TM x TN; 256
// threads).  float64 (FP64-pipe bound, so padding costs time): skinny where
// one dimension is the number of insertions (R~: rows, G_{old,new}: columns)
// or of anchors (measurement product), 32 x 32 otherwise.  float32 (the
// faster pipe makes re-reads of N and per-item overheads matter more): 64 x 64,
// and 128 x 8 for the measurement product.
struct GemmTile {
  int bm, bn, tm, tn;
};
constexpr GemmTile gemm_tile(bool fp64, int phase) {
  return phase == PH_MEAS ? GemmTile{128, 8, 4, 1}
         : !fp64          ? GemmTile{64, 64, 4, 4}
         : phase == PH_RTILDE   ? GemmTile{16, 64, 1, 4}
         : phase == PH_GCOL_OLD ? GemmTile{64, 16, 4, 1}
                                : GemmTile{32, 32, 2, 2};
}

// Compiled tile variants of each product (the autotuner's choices):
// 0 = the default above; 1 and 2 trade re-reads of the operands against
// padding and per-item overhead.  Every variant keeps 256 threads per tile.
constexpr int kTileVariants = 3;
constexpr GemmTile tile_variant(bool fp64, int phase, int v) {
  return v == 0 ? gemm_tile(fp64, phase)
         : phase == PH_MEAS ? (v == 1 ? GemmTile{64, 8, 2, 1} : GemmTile{256, 8, 8, 1})
         : !fp64 ? (v == 1 ? GemmTile{32, 32, 2, 2} : GemmTile{128, 64, 8, 4})
         : phase == PH_RTILDE   ? (v == 1 ? GemmTile{32, 32, 2, 2} : GemmTile{16, 128, 1, 8})
         : phase == PH_GCOL_OLD ? (v == 1 ? GemmTile{32, 32, 2, 2} : GemmTile{128, 16, 8, 1})
                                : (v == 1 ? GemmTile{64, 64, 4, 4} : GemmTile{64, 32, 4, 2});
}

// Tile-variant table of a context (the autotuner's cache): one byte per
// (product, octave of the expansion order, octave of k_max), read by the
// product kernels on the device for each chain's current order.
constexpr int kTileOct = 16, kTileKOct = 9;
constexpr int kTileTable = PH_COUNT * kTileOct * kTileKOct;
static_assert(kTileTable == 720 && kTileVariants == 3, "table size and variants in include/ctaux.h");
__host__ __device__ inline int tile_table_index(int phase, int n, int k) {
  int o = 0, ko = 0;
  while (o + 1 < kTileOct && (2 << o) <= n) ++o;
  while (ko + 1 < kTileKOct && (2 << ko) <= k) ++ko;
  return (phase * kTileOct + o) * kTileKOct + ko;
}

// Fixed launch shapes of one context (derived from capacities at init, so
// that a sweep needs no host-side knowledge of the current orders).
struct LaunchShape {
  int n_chains;
  int gather_slices;
  int kchunk;            // slice width of the inner dimension (while partial tiles fit)
  int persist_ctas;      // grid of the persistent batched kernels
  int tie_grid;          // cooperative grid of the near-tie refinement
  int tie_iters;         // most refinement iterations (0: every near tie takes the fallback)
  int refresh_df64;      // float32 form: refresh elimination in double-float
  int prop_smem;
  int gamma_in_smem;
  int meas_lchunks;      // vertex chunks of the measurement evaluation
  int meas_cb_blocks;
  int meas_acc_blocks;   // one warp per (class, bin) output
  int refresh_grid;
  int use_tc;            // mixed form: flush on the tensor cores
  int tc_ctas;           // persistent grid of the tensor-core flush (one CTA per SM)
  int split_x_blocks;
  int mats;              // Matsubara-frequency measurement on (n_matsubara > 0)
  int tc_wait_limit;     // polls of a tensor-core flush pipeline wait (0: 2^24)
  int prep_tc;           // mixed form: prep products on the tensor cores
  int gamma_lu;          // Gamma kept as L U (CTAUX_GAMMA_LU)
  int max_k;             // largest k_max of the context's chains
  int tile_mask[PH_COUNT];  // tile variants in the context's table, per product (bit v)
};

// CUDA-event timing of the sweep phases and kernel launch counts.  Phases:
// 0 plan + G0 gather, 1 prep products, 2 proposals (Gamma growth), 3 flush
// product, 4 flush support (survivors, Y, end of block), 5 measurement,
// 6 FP64 refresh.  Events are recorded only while profiling is on; launch
// counts are always kept.
struct PhaseTimer {
  static constexpr int kPhases = 8;
  static constexpr int kPool = 1024;
  cudaEvent_t ev[kPool];
  int phase_of[kPool / 2];
  int used = 0;
  int open_slot[kPhases];
  double ms[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long timed[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long kernels[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool created = false;
  bool on = false;
  void begin(int ph, cudaStream_t st) {
    if (!on) return;
    if (used + 2 > kPool) collect();
    open_slot[ph] = used;
    cudaEventRecord(ev[used], st);
    used += 1;
  }
  void end(int ph, cudaStream_t st, int n_kernels) {
    kernels[ph] += n_kernels;
    if (!on) return;
    const int s = open_slot[ph];
    cudaEventRecord(ev[used], st);
    phase_of[s / 2] = ph;
    used += 1;
  }
  // Sums the durations of recorded pairs (synchronises on the last event).
  void collect() {
    if (used == 0) return;
    cudaEventSynchronize(ev[used - 1]);
    for (int s = 0; s + 1 < used; s += 2) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[s], ev[s + 1]) == cudaSuccess) {
        ms[phase_of[s / 2]] += t;
        timed[phase_of[s / 2]] += 1;
      }
    }
    used = 0;
  }
};

// Work run beside a block on a second stream: forked before the block's
// proposals, joined before its end (k_finish_block).
struct BlockFork {
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  void (*fn)(void* arg, cudaStream_t side);
  void* arg;
};

template <typename T>
void launch_block(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st, PhaseTimer* pt,
                  const TcMaps* maps, const BlockFork* fork = nullptr);
template <typename T>
cudaError_t configure_block_kernels(const LaunchShape& ls);
template <typename T>
int launch_gemm(Chain<T>* dchains, const LaunchShape& ls, int phase, cudaStream_t st);
template <typename T>
int refresh_blocks_per_sm(bool df);
size_t refresh_work_doubles(int ld);
template <typename T>
void launch_measure(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st, PhaseTimer* pt);
// The measurement in two parts: the head (counters, G0 panels and the copy of
// the spins) must run before the next block's proposals change the spins; the
// tail reads only what the next block leaves alone until its end.
template <typename T>
int launch_measure_head(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st);
template <typename T>
int launch_measure_tail(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st);
template <typename T>
cudaError_t launch_refresh(Chain<T>* dchains, const LaunchShape& ls, int only_chain,
                           cudaStream_t st, PhaseTimer* pt, int filter = 0);
// scratch: each chain's refresh work area (both spins)
cudaError_t launch_tie_refine(Chain<float>* dchains, const LaunchShape& ls, cudaStream_t st);
template <typename T>
void launch_reset_measure(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st);
template <typename T>
void launch_matsubara(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st);
void launch_g0_matsubara(const double* table, int n_classes, int n_tau, double beta, int n_freq,
                         double2* out, cudaStream_t st);
int tc_smem_bytes();
cudaError_t configure_prep_tc();
void launch_prep_tc(Chain<float>* dchains, const TcMaps* maps, const LaunchShape& ls,
                    cudaStream_t st);
cudaError_t encode_prep_maps(TcMaps* out, float* cpan, float* bpan, int panel_rows,
                             float* n0, float* n1, float* nt0, float* nt1, int ld);
cudaError_t configure_flush_tc();
void launch_flush_tc(Chain<float>* dchains, const TcMaps* maps, const LaunchShape& ls,
                     cudaStream_t st);
void launch_transpose_n(Chain<float>* dchains, const LaunchShape& ls, cudaStream_t st);
cudaError_t encode_tc_maps(TcMaps* out, float* yh, float* yl, float* xh, float* xl, int rows,
                           int kp, float* n0, float* n1, int ld);
void launch_philox_test(uint64_t seed, uint32_t chain, int64_t t0, int count, int purpose,
                        double* out, cudaStream_t st);

}  // namespace ctaux
