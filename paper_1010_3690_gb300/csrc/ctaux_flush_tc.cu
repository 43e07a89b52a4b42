// Woodbury flush of the mixed form on the 5th-generation tensor cores:
//   N'[a][b] = N[S_a][S_b] - sum_r Y[a][r] X[r][b],  X = N[P, S]
// (Eq. Nshermanmorrison with the s=0 rows and columns removed, Sec. IV C),
// as a tcgen05 GEMM with the split 3xTF32 product of Ootomo & Yokota (2022):
// every float32 operand is split into hi = tf32(x) and lo = tf32(x - hi), and
// hi*hi + hi*lo + lo*hi accumulate in one float32 TMEM accumulator.
//
// Operands are K-major split buffers written by the flush preparation kernels
// (Yh/Yl: rows a, Xh/Xl: rows b, KP = k_max rounded up to 32 float32 per row,
// zero beyond k_acc), loaded by TMA into shared memory swizzled over the
// 64-byte row of one 16-wide K chunk (one TMA load per 128 x 16 tile, no
// multicast).
//
// One persistent CTA per SM, warp-specialised, over the (chain, spin,
// 128 x 128 tile) items of all chains:
//   warp 0 (one thread): TMA producer into a ring of kTcStages 32 KB stages;
//   warp 1 (one thread): MMA issuer, 6 tcgen05.mma per 16-wide K step into
//     one of two 128-column TMEM accumulators, each stage released to the
//     producer by tcgen05.commit when its MMAs are done;
//   warp 3: loader of the epilogue input N[S_m][S_n]: the survivor rows
//     S[m0] .. S[m0 + 127] of a tile are contiguous up to the few removed
//     rows, so each of its 128 columns S[n] is a segment of kTcNsRows rows
//     starting at S[m0] rounded down to 16 bytes, loaded by TMA in boxes of
//     kTcNsGroup adjacent columns (a tile whose rows span more falls back to
//     gathered global loads);
//   warps 4-11: epilogue; warp w reads TMEM lane quarter w % 4 (64 of the 128
//     columns), subtracts from the staged N[S_m][S_n] and writes the compacted
//     N', then releases the accumulator and the staged input, so that the
//     epilogue of one tile overlaps the loads and MMAs of the next.
// Every mbarrier wait is bounded: the pipeline roles poll at most `wl` times
// (a launch argument, 2^24 unless the context sets a smaller limit), the
// final drains always 2^24 times.  On timeout the chain's status gets
// DS_TIMEOUT (CTAUX_ETIMEOUT) and every role stops; before the CTA exits, the
// copies issued are waited for, the MMA thread waits for its MMAs, and the
// TMEM is freed.  With `stall` set (a test of this path) the MMA issuer first
// waits on a barrier that nothing completes, so every launch times out.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"
#include "ctaux_tc.cuh"

namespace ctaux {

namespace {

using namespace tc;
constexpr int kStageBytes = 4 * kTileBytes;     // Ah, Al, Bh, Bl
constexpr int kNsSlotBytes = kTcNsRows * 4;     // one staged column segment
constexpr int kNsBytes = kTcBN * kNsSlotBytes;  // the staged input of one tile
static_assert(kTcBK == kBK && kTcBM == 128 && kTcBN == 128, "the shared descriptors' tile");
static_assert(kNsSlotBytes % 128 == 0, "staged column segments must stay 128-byte aligned");
static_assert(kTcBN % kTcNsGroup == 0 && kTcBN / kTcNsGroup <= 32, "one column group per lane");
constexpr uint32_t kTmemCols = 2 * kTcBN;       // two accumulators

}  // namespace

// X = N[P, S] as K-major split rows: Xh/Xl[b * KP + r], zero for r >= k_acc.
// One warp per output row b.
__global__ void __launch_bounds__(256) k_flush_split_x(Chain<float>* chains) {
  const Chain<float>& c = chains[blockIdx.z];
  const Dyn& d = *c.dyn;
  if (d.status || d.flush_noop) return;
  const int spin = blockIdx.y, nn = d.n_new, kacc = d.k_acc, KP = c.kp;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const float* Nb = c.N[d.buf][spin];
  for (int b = warp; b < nn; b += nwarps) {
    const long col = (long)c.S[b] * c.ld;
    for (int r = lane; r < KP; r += 32) {
      float hi = 0.f, lo = 0.f;
      if (r < kacc) split_tf32(Nb[col + c.P[r]], hi, lo);
      c.Xh[spin][(size_t)b * KP + r] = hi;
      c.Xl[spin][(size_t)b * KP + r] = lo;
    }
  }
}

__device__ __forceinline__ int tc_items(const Dyn& d) {
  if (d.status || d.flush_noop) return 0;
  const int tiles = (d.n_new + kTcBM - 1) / kTcBM;
  return 2 * tiles * tiles;
}

struct TcItem {
  int ci, spin, m0, n0, nk, nn;
};

__device__ __forceinline__ TcItem tc_item(Chain<float>* chains, const int* off, int n_chains, int w) {
  TcItem it;
  it.ci = find_chain(off, n_chains, w);
  const Dyn& d = *chains[it.ci].dyn;
  it.nn = d.n_new;
  const int tiles = (it.nn + kTcBM - 1) / kTcBM;
  const int l = w - off[it.ci];
  it.spin = l / (tiles * tiles);
  const int tile = l % (tiles * tiles);
  // consecutive items (processed at the same time by consecutive CTAs) share
  // the column band, i.e. the X operand tile, and walk down the rows
  it.m0 = (tile % tiles) * kTcBM;
  it.n0 = (tile / tiles) * kTcBN;
  it.nk = (d.k_acc + kTcBK - 1) / kTcBK;
  return it;
}

// Staged-input geometry of a tile: source row of its first row rounded down
// to 16 bytes, and whether its rows fit one kTcNsRows segment.
__device__ __forceinline__ bool ns_staged(const int* S, int m0, int nn, int& x0) {
  x0 = __ldg(S + m0) & ~3;
  return __ldg(S + min(m0 + kTcBM - 1, nn - 1)) - x0 < kTcNsRows;
}

// Barrier completion c (0-based) of an mbarrier has parity c & 1.
__global__ void __launch_bounds__(kTcThreads, 1) k_flush_tc(Chain<float>* chains, int n_chains,
                                                            const TcMaps* maps, uint32_t wl,
                                                            int stall) {
  __shared__ int off[kMaxChains + 1];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) off[ci] = tc_items(*chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  if ((int)blockIdx.x >= total) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      ((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  float* ns = reinterpret_cast<float*>(base + kTcStages * kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kTcStages * kStageBytes + kNsBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* accfull = empty + kTcStages;
  uint64_t* accempty = accfull + 2;
  uint64_t* drain = accempty + 2;
  uint64_t* nsfull = drain + 1;
  uint64_t* nsempty = nsfull + 1;
  uint64_t* never = nsempty + 1;  // completed by nothing (the test stall)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* err_s = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint32_t* mma_taken = reinterpret_cast<uint32_t*>(tmem_slot + 2);  // stages the MMA thread waited for
  uint32_t* ns_issued = reinterpret_cast<uint32_t*>(tmem_slot + 3);  // tiles the loader staged

  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(full + s), 1);
      mbar_init(smem_u32(empty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(accfull + b), 1);
      mbar_init(smem_u32(accempty + b), 8);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(drain), 1);
    mbar_init(smem_u32(nsfull), 1);
    mbar_init(smem_u32(nsempty), 8);
    mbar_init(smem_u32(never), 1);
    *err_s = 0;
    *mma_taken = 0;
    *ns_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  uint32_t issued = 0;  // producer: stages issued

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int w = blockIdx.x; w < total && !*err_s; w += gridDim.x) {
      const TcItem t = tc_item(chains, off, n_chains, w);
      if (t.nk == 0) continue;
      const TcMaps& mp = maps[t.ci * 2 + t.spin];
      for (int kc = 0; kc < t.nk; ++kc) {
        const uint32_t stage = issued % kTcStages, use = issued / kTcStages;
        if (use > 0 && !mbar_wait(smem_u32(empty + stage), (use - 1) & 1, wl)) {
          *err_s = 1;
          atomicOr(&chains[t.ci].dyn->status, DS_TIMEOUT);
          break;
        }
        const uint32_t fb = smem_u32(full + stage);
        unsigned char* sb = base + stage * kStageBytes;
        mbar_expect_tx(fb, kStageBytes);
        tma_load_2d(smem_u32(sb + 0 * kTileBytes), &mp.yh, kc * kTcBK, t.m0, fb);
        tma_load_2d(smem_u32(sb + 1 * kTileBytes), &mp.yl, kc * kTcBK, t.m0, fb);
        tma_load_2d(smem_u32(sb + 2 * kTileBytes), &mp.xh, kc * kTcBK, t.n0, fb);
        tma_load_2d(smem_u32(sb + 3 * kTileBytes), &mp.xl, kc * kTcBK, t.n0, fb);
        ++issued;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    uint32_t taken = 0, q = 0;
    if (stall && !mbar_wait(smem_u32(never), 0, wl)) {
      // test of the bounded waits: a barrier that nothing completes
      *err_s = 1;
      atomicOr(&chains[find_chain(off, n_chains, blockIdx.x)].dyn->status, DS_TIMEOUT);
    }
    for (int w = blockIdx.x; w < total && !*err_s; w += gridDim.x) {
      const TcItem t = tc_item(chains, off, n_chains, w);
      if (t.nk == 0) continue;
      const uint32_t b = q & 1, ub = q >> 1;
      bool ok = ub == 0 || mbar_wait(smem_u32(accempty + b), (ub - 1) & 1, wl);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + b * kTcBN;
      for (int kc = 0; kc < t.nk && ok; ++kc) {
        const uint32_t stage = taken % kTcStages, use = taken / kTcStages;
        if (!mbar_wait(smem_u32(full + stage), use & 1, wl)) {
          ok = false;
          break;
        }
        ++taken;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(base + stage * kStageBytes), al = ah + kTileBytes,
                       bh = ah + 2 * kTileBytes, bl = ah + 3 * kTileBytes;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 8; ++kk) {
          const uint32_t offk = kk * 32;  // 8 tf32 = 32 bytes along K
          const uint32_t first = (kc == 0 && kk == 0) ? 0u : 1u;
          mma_tf32(acc, smem_desc(ah + offk), smem_desc(bl + offk), first);  // hi * lo
          mma_tf32(acc, smem_desc(al + offk), smem_desc(bh + offk), 1u);     // lo * hi
          mma_tf32(acc, smem_desc(ah + offk), smem_desc(bh + offk), 1u);     // hi * hi
        }
        mma_commit(smem_u32(empty + stage));  // stage free once these MMAs are done
      }
      if (!ok) {
        *err_s = 1;
        atomicOr(&chains[t.ci].dyn->status, DS_TIMEOUT);
        break;
      }
      mma_commit(smem_u32(accfull + b));
      ++q;
    }
    *mma_taken = taken;
    // every MMA issued so far has completed before the TMEM can be freed
    mma_commit(smem_u32(drain));
    mbar_wait(smem_u32(drain), 0);
  } else if (warp == 3) {
    // ---- loader of the epilogue input, one tile ahead of the epilogue.  The
    // 128 columns go in groups of kTcNsGroup: a group of adjacent source
    // columns (no removed column inside) is one TMA box, any other group one
    // box per column.  Indices are read before the buffer is free.
    uint32_t nq = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      if (__any_sync(0xffffffffu, *err_s != 0)) break;
      const TcItem t = tc_item(chains, off, n_chains, w);
      const Chain<float>& c = chains[t.ci];
      int x0;
      const bool staged = ns_staged(c.S, t.m0, t.nn, x0);
      const int cols = staged ? min(kTcBN, t.nn - t.n0) : 0;
      const int g0 = lane * kTcNsGroup;  // lanes 0-15: one group each
      int s_first = 0;
      bool whole = false;
      if (g0 < cols) {
        s_first = __ldg(c.S + t.n0 + g0);
        whole = g0 + kTcNsGroup <= cols &&
                __ldg(c.S + t.n0 + g0 + kTcNsGroup - 1) - s_first == kTcNsGroup - 1;
      }
      const TcMaps& mp = maps[t.ci * 2 + t.spin];
      const int buf = c.dyn->buf;
      if (nq > 0 && !__all_sync(0xffffffffu, mbar_wait(smem_u32(nsempty), (nq - 1) & 1, wl))) {
        if (lane == 0) {
          *err_s = 1;
          atomicOr(&c.dyn->status, DS_TIMEOUT);
        }
        break;
      }
      if (lane == 0) mbar_expect_tx(smem_u32(nsfull), (uint32_t)(cols * kNsSlotBytes));
      __syncwarp();
      if (g0 < cols) {
        const uint32_t dst = smem_u32(ns) + g0 * kNsSlotBytes;
        if (whole) {
          tma_load_2d(dst, &mp.nbg[buf], x0, s_first, smem_u32(nsfull));
        } else {
          for (int j = g0; j < min(g0 + kTcNsGroup, cols); ++j)
            tma_load_2d(smem_u32(ns) + j * kNsSlotBytes, &mp.nb1[buf], x0, __ldg(c.S + t.n0 + j),
                        smem_u32(nsfull));
        }
      }
      ++nq;
    }
    if (lane == 0) *ns_issued = nq;
  } else if (warp >= 4) {
    // ---- epilogue: warp w, TMEM lanes 32 (w % 4) .. + 31, column half (w - 4) / 4
    const int quarter = warp & 3, colhalf = (warp - 4) >> 2;
    uint32_t q = 0, nq = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      if (__any_sync(0xffffffffu, *err_s != 0)) break;
      const TcItem t = tc_item(chains, off, n_chains, w);
      const Chain<float>& c = chains[t.ci];
      const Dyn& d = *c.dyn;
      const int ld = c.ld, nn = t.nn;
      const float* Nb = c.N[d.buf][t.spin];
      float* out = c.N[1 - d.buf][t.spin];
      const int* S = c.S;
      const int m = t.m0 + quarter * 32 + lane;
      const bool row_ok = m < nn;
      int x0;
      const bool staged = ns_staged(S, t.m0, nn, x0);
      const int srow = row_ok ? __ldg(S + m) : x0;  // rows past the end read a valid slot
      const float* nsrow = ns + (srow - x0);  // staged N[srow][S[n0 + j]] at nsrow[j * kTcNsRows]
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(nsfull), nq & 1, wl))) {
        if (lane == 0) {
          *err_s = 1;
          atomicOr(&c.dyn->status, DS_TIMEOUT);
        }
        break;
      }
      ++nq;
      if (t.nk == 0) {  // no accepted change: the flush is a pure compaction
        if (row_ok)
          for (int j = colhalf * 64; j < colhalf * 64 + 64; ++j) {
            const int n = t.n0 + j;
            if (n < nn)
              out[(long)n * ld + m] = staged ? nsrow[j * kTcNsRows] : Nb[(long)__ldg(S + n) * ld + srow];
          }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(nsempty));
        continue;
      }
      const uint32_t b = q & 1, ub = q >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(accfull + b), ub & 1, wl));
      if (!ok) {
        if (lane == 0) {
          *err_s = 1;
          atomicOr(&c.dyn->status, DS_TIMEOUT);
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[32], cin[32];
#pragma unroll 1
      for (int cc = colhalf * 2; cc < colhalf * 2 + 2; ++cc) {
        if (staged) {
#pragma unroll
          for (int j = 0; j < 32; ++j) cin[j] = nsrow[(cc * 32 + j) * kTcNsRows];
        } else {
          // rows spanning more than one segment: gathered global loads
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = t.n0 + cc * 32 + j;
            cin[j] = (row_ok && n < nn) ? Nb[(long)__ldg(S + n) * ld + srow] : 0.f;
          }
        }
        tmem_ld32(tmem + b * kTcBN + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cc * 32), v);
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = t.n0 + cc * 32 + j;
            if (n < nn) out[(long)n * ld + m] = cin[j] - v[j];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(accempty + b));
        mbar_arrive(smem_u32(nsempty));
      }
      ++q;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies issued but never waited for (only after a timeout): let them land
    for (uint32_t i = *mma_taken; i < issued; ++i)
      mbar_wait(smem_u32(full + i % kTcStages), (i / kTcStages) & 1);
    if (*ns_issued > 0) mbar_wait(smem_u32(nsfull), (*ns_issued - 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// N'^T for the tensor-core prep (its G_{old,new} = N B reads rows of N as
// K-major rows): 64 x 64 tiles of the flushed N' through shared memory (16
// loads in flight per thread), all chains, both spins; nothing to do for a
// block that left N unchanged.
__global__ void __launch_bounds__(256) k_transpose_n(Chain<float>* chains, int n_chains) {
  __shared__ float tile[64][65];
  __shared__ int off[kMaxChains + 1];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
    const Dyn& d = *chains[ci].dyn;
    const int tb = (d.n_new + 63) / 64;
    off[ci] = (d.status || d.flush_noop || !chains[ci].NT[0][0]) ? 0 : 2 * tb * tb;
  }
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int ci = find_chain(off, n_chains, w);
    const Chain<float>& c = chains[ci];
    const Dyn& d = *c.dyn;
    const int nn = d.n_new, tb = (nn + 63) / 64, l = w - off[ci];
    const int spin = l / (tb * tb), t = l % (tb * tb);
    const int i0 = (t % tb) * 64, j0 = (t / tb) * 64, ld = c.ld;
    const float* src = c.N[1 - d.buf][spin];   // the flush wrote the other buffer
    float* dst = c.NT[1 - d.buf][spin];
    __syncthreads();
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = i0 + tx, j = j0 + ty + 4 * u;
      v[u] = (i < nn && j < nn) ? src[(long)j * ld + i] : 0.f;   // N'[i][j]
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) tile[ty + 4 * u][tx] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = i0 + ty + 4 * u, j = j0 + tx;
      if (i < nn && j < nn) dst[(long)i * ld + j] = tile[tx][ty + 4 * u];   // N'^T[j][i] = N'[i][j]
    }
  }
}

int tc_smem_bytes() { return kTcStages * kStageBytes + kNsBytes + 1024 + 256; }

cudaError_t configure_flush_tc() {
  return cudaFuncSetAttribute(k_flush_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc_smem_bytes());
}

void launch_flush_tc(Chain<float>* dchains, const TcMaps* maps, const LaunchShape& ls,
                     cudaStream_t st) {
  k_flush_split_x<<<dim3(ls.split_x_blocks, 2, ls.n_chains), 256, 0, st>>>(dchains);
  const int lim = ls.tc_wait_limit;
  const uint32_t wl = lim > 0 ? (uint32_t)lim : lim < 0 ? (uint32_t)(-(int64_t)lim) : kWaitLimit;
  k_flush_tc<<<ls.tc_ctas, kTcThreads, tc_smem_bytes(), st>>>(dchains, ls.n_chains, maps, wl,
                                                              lim < 0 ? 1 : 0);
}

void launch_transpose_n(Chain<float>* dchains, const LaunchShape& ls, cudaStream_t st) {
  k_transpose_n<<<ls.persist_ctas, 256, 0, st>>>(dchains, ls.n_chains);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return nullptr;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}
}  // namespace

// Host: the prep's TMA descriptors of one (chain, spin): rows of ld float32
// (the panels C and B with panel_rows rows; both buffers of N
// and of N^T with ld rows), boxes of 128 rows x kTcBK float32, 64-byte swizzle.
cudaError_t encode_prep_maps(TcMaps* out, float* cpan, float* bpan, int panel_rows,
                             float* n0, float* n1, float* nt0, float* nt1, int ld) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcBK, 128u};
  float* ptrs[6] = {cpan, bpan, n0, n1, nt0, nt1};
  CUtensorMap* maps[6] = {&out->cpan, &out->bpan, &out->nb[0], &out->nb[1], &out->nt[0], &out->nt[1]};
  for (int i = 0; i < 6; ++i) {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)(i < 2 ? panel_rows : ld)};
    const CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptrs[i], dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// Host: the TMA descriptors of one (chain, spin): K-major float32 operand
// buffers of rows x kp, boxes of 128 rows x kTcBK float32 swizzled over the
// row width; and both buffers of N (ld x ld, column-major), boxes of one or
// kTcNsGroup column segments of kTcNsRows rows, no swizzle.
cudaError_t encode_tc_maps(TcMaps* out, float* yh, float* yl, float* xh, float* xl, int rows,
                           int kp, float* n0, float* n1, int ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcBM};
    float* ptrs[4] = {yh, yl, xh, xl};
    CUtensorMap* maps[4] = {&out->yh, &out->yl, &out->xh, &out->xl};
    for (int i = 0; i < 4; ++i) {
      const CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptrs[i], dims, strides,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    float* ptrs[2] = {n0, n1};
    for (int g = 0; g < 2; ++g) {
      const cuuint32_t box[2] = {(cuuint32_t)kTcNsRows, g ? (cuuint32_t)kTcNsGroup : 1u};
      for (int i = 0; i < 2; ++i) {
        const CUresult r = encode(g ? &out->nbg[i] : &out->nb1[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                  ptrs[i], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
      }
    }
  }
  return cudaSuccess;
}

}  // namespace ctaux
