// Prep products of the mixed form on the 5th-generation tensor cores
// (Sec. IV A: the rows of the extended N for the block's pre-inserted
// vertices, and the columns of G = N_ext G0 for them):
//   product 0: R~[a][j]     = sum_{l<n} C[a][l] N[l][j]            -> N_ext[n + a][j]
//   product 1: G[i][a]      = sum_{l<n} N[i][l] B[l][a]             -> Gcol[a][i], i < n
// (the third prep product, G[n + a][b] += sum_{l<n} C[a][l] G[l][b], is a few
// k x k tiles over the long inner dimension n: the block runs it on the CUDA
// cores, split over K) with C = G0(new, old)(e^{V_old} - 1) and B = G0(old, new) (the gathered
// panels), as 128 x 128 output tiles of a tcgen05 GEMM with the split 3xTF32
// product of Ootomo & Yokota (2022): hi*hi in one float32 TMEM accumulator,
// hi*lo + lo*hi in a second one, added in the epilogue.  The split truncates
// (bit masks, no conversion instructions): the converter warps set the
// kernel's pace.
//
// Both operands are read by TMA as K-major float32 rows (K = the old-vertex
// index l): C and B are the panels' rows, the columns of N (column-major) are
// the K-major rows of product 0's B operand, and product 1's A operand is
// N^T (rows of N), a copy that the flush and the refresh keep beside N.
// Converter warps split every staged float32 tile into tf32 hi (x truncated)
// and lo (x - hi truncated) and zero the elements with l >= n (so rows of
// N_ext being written, and stale panel entries, never enter a product).
//
// One persistent CTA per SM, warp-specialised like the tensor-core flush:
//   warp 0 (one thread): TMA producer into a ring of raw float32 stages;
//   warp 1 (one thread): MMA issuer, 6 tcgen05.mma per 16-wide K chunk into
//     one of two TMEM accumulator pairs (main hi*hi, correction hi*lo + lo*hi);
//   warps 2-7: converters, raw stage -> split stage (warp 2 allocates the
//     TMEM first);
//   warps 8-11: epilogue, TMEM lane quarter w % 4, all 128 columns: adds each
//     segment's partial tile to the float32 tile accumulator in shared memory
//     and writes the tile after the last segment.
// Every mbarrier wait is bounded; on timeout the chain's status gets
// DS_TIMEOUT and every role stops, the copies issued are drained, the MMA
// thread waits for its MMAs and the TMEM is freed.
#include <cuda.h>

#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"
#include "ctaux_tc.cuh"

namespace ctaux {

namespace {

using namespace tc;
constexpr int kRawStages = 3, kSplitStages = 3;
constexpr int kConvWarps = 6;   // warps 2..7 (warp 2 allocates the TMEM first)
// K chunks accumulated in TMEM before the epilogue adds the partial tile to a
// float32 accumulator in shared memory (round to nearest): the tensor cores'
// own additions truncate, so long inner dimensions are summed in segments
constexpr int kSegChunks = 8;
constexpr int kAccBytes = 128 * 128 * 4;          // the output tile, column-major
constexpr int kRawStageBytes = 2 * kTileBytes;    // A, B as float32
constexpr int kSplitStageBytes = 4 * kTileBytes;  // Ah, Al, Bh, Bl
constexpr int kPrepThreads = 384;
// two tiles in flight, each with a main (hi*hi) and a correction (hi*lo +
// lo*hi) accumulator of 128 columns: the small correction terms are not
// accumulated into the large main sum, whose additions truncate (Ootomo &
// Yokota keep them apart for that reason); the epilogue adds the two in
// float32 with round-to-nearest
constexpr uint32_t kPrepTmemCols = 512;

struct PrepItem {
  int ci, spin, prod, m0, n0, M, N, K;
};

// Output sizes of a product of one chain in the current block (M x N, inner K).
__device__ __forceinline__ void prep_dims(const Dyn& d, int prod, int& M, int& N, int& K) {
  const int n = d.n, ki = d.k_ins;
  K = n;
  M = (prod == 1) ? n : ki;
  N = (prod == 0) ? n : ki;
}

__device__ __forceinline__ int prep_items_of(const Dyn& d, int prod) {
  if (d.status) return 0;
  int M, N, K;
  prep_dims(d, prod, M, N, K);
  if (M == 0 || N == 0 || K == 0) return 0;   // no old vertices or no insertions
  return 2 * ((M + 127) / 128) * ((N + 127) / 128);
}

__device__ __forceinline__ int prep_items(const Dyn& d) {
  return prep_items_of(d, 0) + prep_items_of(d, 1);
}

__device__ __forceinline__ PrepItem prep_item(Chain<float>* chains, const int* off, int n_chains,
                                              int w) {
  PrepItem it;
  it.ci = find_chain(off, n_chains, w);
  const Dyn& d = *chains[it.ci].dyn;
  int l = w - off[it.ci];
  const int k0 = prep_items_of(d, 0);
  it.prod = l < k0 ? 0 : 1;
  if (it.prod == 1) l -= k0;
  prep_dims(d, it.prod, it.M, it.N, it.K);
  const int tm = (it.M + 127) / 128, tn = (it.N + 127) / 128;
  it.spin = l / (tm * tn);
  const int tile = l % (tm * tn);
  // consecutive items share the operand that is the same for a whole row
  // (product 0: C) or column (product 1: B) of tiles
  if (it.prod == 1) {
    it.m0 = (tile % tm) * 128;
    it.n0 = (tile / tm) * 128;
  } else {
    it.n0 = (tile % tn) * 128;
    it.m0 = (tile / tn) * 128;
  }
  return it;
}

// Split one staged 16-byte group (4 float32 of one row) into hi and lo and
// zero the K positions at or beyond K.  With the 64-byte swizzle, the group
// at physical 16-byte slot p of row r holds K chunk c = p ^ ((r >> 1) & 3).
__device__ __forceinline__ void split_group(const float4 x, int off_in_tile, int kc, int K,
                                            float4& hi, float4& lo) {
  const int r = off_in_tile >> 6, p = (off_in_tile >> 4) & 3;
  const int k0 = kc * kBK + 4 * (p ^ ((r >> 1) & 3));
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (k0 + e < K) {
      split_tf32_trunc(xs[e], h[e], l[e]);
    } else {
      h[e] = 0.f;
      l[e] = 0.f;
    }
  }
  hi = make_float4(h[0], h[1], h[2], h[3]);
  lo = make_float4(l[0], l[1], l[2], l[3]);
}

}  // namespace

// Products 0 and 1 of every chain.  Barrier completion c of an
// mbarrier has parity c & 1.
__global__ void __launch_bounds__(kPrepThreads, 1) k_prep_tc(Chain<float>* chains, int n_chains,
                                                             const TcMaps* maps, uint32_t wl) {
  __shared__ int off[kMaxChains + 1];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x)
    off[ci] = prep_items(*chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  if ((int)blockIdx.x >= total) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  extern __shared__ __align__(1024) unsigned char prep_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      ((uintptr_t)prep_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* raw = base;                                          // kRawStages x 16 KB
  unsigned char* split = base + kRawStages * kRawStageBytes;         // kSplitStages x 32 KB
  float* acc_s = reinterpret_cast<float*>(split + kSplitStages * kSplitStageBytes);  // 64 KB
  uint64_t* rfull = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(acc_s) + kAccBytes);
  uint64_t* rempty = rfull + kRawStages;
  uint64_t* sfull = rempty + kRawStages;
  uint64_t* sempty = sfull + kSplitStages;
  uint64_t* accfull = sempty + kSplitStages;
  uint64_t* accempty = accfull + 2;
  uint64_t* drain = accempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* err_s = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint32_t* conv_taken = reinterpret_cast<uint32_t*>(tmem_slot + 2);  // raw stages converted

  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kPrepTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(smem_u32(rfull + s), 1);
      mbar_init(smem_u32(rempty + s), kConvWarps);   // one arrival per converter warp
    }
    for (int s = 0; s < kSplitStages; ++s) {
      mbar_init(smem_u32(sfull + s), kConvWarps);    // one arrival per converter warp
      mbar_init(smem_u32(sempty + s), 1);   // tcgen05.commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(accfull + b), 1);
      mbar_init(smem_u32(accempty + b), 4);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(drain), 1);
    *err_s = 0;
    *conv_taken = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  uint32_t issued = 0;  // producer: raw stages issued

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int w = blockIdx.x; w < total && !*err_s; w += gridDim.x) {
      const PrepItem t = prep_item(chains, off, n_chains, w);
      const TcMaps& mp = maps[t.ci * 2 + t.spin];
      const int buf = chains[t.ci].dyn->buf;
      const CUtensorMap* ma = (t.prod == 1) ? &mp.nt[buf] : &mp.cpan;
      const CUtensorMap* mb = (t.prod == 0) ? &mp.nb[buf] : &mp.bpan;
      const int nk = (t.K + kBK - 1) / kBK;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        const uint32_t stage = issued % kRawStages, use = issued / kRawStages;
        if (use > 0 && !mbar_wait(smem_u32(rempty + stage), (use - 1) & 1, wl)) {
          ok = false;
          break;
        }
        const uint32_t fb = smem_u32(rfull + stage);
        unsigned char* sb = raw + stage * kRawStageBytes;
        mbar_expect_tx(fb, kRawStageBytes);
        tma_load_2d(smem_u32(sb), ma, kc * kBK, t.m0, fb);
        tma_load_2d(smem_u32(sb + kTileBytes), mb, kc * kBK, t.n0, fb);
        ++issued;
      }
      if (!ok) {
        *err_s = 1;
        atomicOr(&chains[t.ci].dyn->status, DS_TIMEOUT);
        break;
      }
    }
  } else if (warp >= 8 - kConvWarps && warp < 8) {
    // ---- converters: raw float32 stage -> hi / lo split stage
    const int ct = threadIdx.x - 32 * (8 - kConvWarps);  // 0 .. 32 kConvWarps - 1
    uint32_t taken = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      if (__any_sync(0xffffffffu, *err_s != 0)) break;
      const PrepItem t = prep_item(chains, off, n_chains, w);
      const int nk = (t.K + kBK - 1) / kBK;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc) {
        const uint32_t rs = taken % kRawStages, ru = taken / kRawStages;
        const uint32_t ss = taken % kSplitStages, su = taken / kSplitStages;
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(rfull + rs), ru & 1, wl));
        if (ok && su > 0) ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(sempty + ss), (su - 1) & 1, wl));
        if (!ok) break;
        const unsigned char* rb = raw + rs * kRawStageBytes;
        unsigned char* sb = split + ss * kSplitStageBytes;
        // 2 tiles x 512 groups of 16 bytes, 8 per thread
#pragma unroll
        for (int g = ct; g < 1024; g += 32 * kConvWarps) {   // 2 tiles x 512 groups
          const int tile = g >> 9, o = (g & 511) * 16;
          const float4 x = *reinterpret_cast<const float4*>(rb + tile * kTileBytes + o);
          float4 hi, lo;
          split_group(x, o, kc, t.K, hi, lo);
          // split stage: Ah, Al, Bh, Bl
          *reinterpret_cast<float4*>(sb + (2 * tile) * kTileBytes + o) = hi;
          *reinterpret_cast<float4*>(sb + (2 * tile + 1) * kTileBytes + o) = lo;
        }
        // generic-proxy writes become visible to the tensor cores' async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(sfull + ss));
          mbar_arrive(smem_u32(rempty + rs));
        }
        ++taken;
      }
      if (!ok) {
        if (lane == 0) {
          *err_s = 1;
          atomicOr(&chains[t.ci].dyn->status, DS_TIMEOUT);
        }
        break;
      }
    }
    if (threadIdx.x == 32 * (8 - kConvWarps)) *conv_taken = taken;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: each segment of kSegChunks K chunks into the next free
    // accumulator pair
    uint32_t taken = 0, q = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < total && ok && !*err_s; w += gridDim.x) {
      const PrepItem t = prep_item(chains, off, n_chains, w);
      const int nk = (t.K + kBK - 1) / kBK;
      for (int k0 = 0; k0 < nk && ok; k0 += kSegChunks) {
        const uint32_t b = q & 1, ub = q >> 1;
        ok = ub == 0 || mbar_wait(smem_u32(accempty + b), (ub - 1) & 1, wl);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + b * 256, corr = acc + 128;
        for (int kc = k0; kc < min(nk, k0 + kSegChunks) && ok; ++kc) {
          const uint32_t ss = taken % kSplitStages, su = taken / kSplitStages;
          if (!mbar_wait(smem_u32(sfull + ss), su & 1, wl)) {
            ok = false;
            break;
          }
          ++taken;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = smem_u32(split + ss * kSplitStageBytes), al = ah + kTileBytes,
                         bh = ah + 2 * kTileBytes, bl = ah + 3 * kTileBytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 8; ++kk) {
            const uint32_t offk = kk * 32;  // 8 tf32 = 32 bytes along K
            const uint32_t first = (kc == k0 && kk == 0) ? 0u : 1u;
            mma_tf32(corr, smem_desc(ah + offk), smem_desc(bl + offk), first);  // hi * lo
            mma_tf32(corr, smem_desc(al + offk), smem_desc(bh + offk), 1u);      // lo * hi
            mma_tf32(acc, smem_desc(ah + offk), smem_desc(bh + offk), first);   // hi * hi
          }
          mma_commit(smem_u32(sempty + ss));  // split stage free once these MMAs are done
        }
        if (!ok) {
          *err_s = 1;
          atomicOr(&chains[t.ci].dyn->status, DS_TIMEOUT);
          break;
        }
        mma_commit(smem_u32(accfull + b));
        ++q;
      }
    }
    mma_commit(smem_u32(drain));   // every MMA issued so far completes before the TMEM is freed
    mbar_wait(smem_u32(drain), 0);
  } else if (warp >= 8) {
    // ---- epilogue: TMEM lanes 32 (w % 4) .. + 31 = output rows, all 128 columns
    const int quarter = warp & 3;
    uint32_t q = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      if (__any_sync(0xffffffffu, *err_s != 0)) break;
      const PrepItem t = prep_item(chains, off, n_chains, w);
      const Chain<float>& c = chains[t.ci];
      const Dyn& d = *c.dyn;
      const int ld = c.ld, n = d.n;
      const int rl = quarter * 32 + lane;      // the tile row of this thread
      const int row = t.m0 + rl;
      const int nk = (t.K + kBK - 1) / kBK;
      bool ok = true;
      for (int k0 = 0; k0 < nk; k0 += kSegChunks) {
        const uint32_t b = q & 1, ub = q >> 1;
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(accfull + b), ub & 1, wl))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float v[32], vc[32];
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
          const uint32_t ta = tmem + b * 256 + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cc * 32);
          tmem_ld32(ta, v);
          tmem_ld32(ta + 128, vc);
          float* a = acc_s + (cc * 32) * 128 + rl;   // column-major: [column][row]
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float seg = v[j] + vc[j];
            a[j * 128] = (k0 == 0) ? seg : a[j * 128] + seg;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(accempty + b));
        ++q;
      }
      if (!ok) {
        if (lane == 0) {
          *err_s = 1;
          atomicOr(&c.dyn->status, DS_TIMEOUT);
        }
        break;
      }
      float* Nb = c.N[d.buf][t.spin];
      float* Gc = c.Gcol[t.spin];
      if (row < t.M) {
        for (int j = 0; j < 128; ++j) {
          const int col = t.n0 + j;
          if (col >= t.N) break;
          const float v = acc_s[j * 128 + rl];
          if (t.prod == 0) Nb[(long)col * ld + n + row] = v;
          else Gc[(long)col * ld + row] = v;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // raw copies issued but never converted (only after a timeout): let them land
    for (uint32_t i = *conv_taken; i < issued; ++i)
      mbar_wait(smem_u32(rfull + i % kRawStages), (i / kRawStages) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kPrepTmemCols)
                 : "memory");
}

int prep_tc_smem_bytes() {
  return kRawStages * kRawStageBytes + kSplitStages * kSplitStageBytes + kAccBytes + 1024 + 256;
}

cudaError_t configure_prep_tc() {
  return cudaFuncSetAttribute(k_prep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              prep_tc_smem_bytes());
}

// Products 0 and 1 (independent of each other) on the tensor cores.  Product
// 2 (k_ins x k_ins, reading product 1's columns) has a handful of tiles with a
// long inner dimension, which the tensor-core pipeline runs one K chunk at a
// time on a few SMs; the caller runs it on the CUDA cores (split over K).
void launch_prep_tc(Chain<float>* dchains, const TcMaps* maps, const LaunchShape& ls,
                    cudaStream_t st) {
  const int lim = ls.tc_wait_limit;
  const uint32_t wl = lim > 0 ? (uint32_t)lim : lim < 0 ? (uint32_t)(-(int64_t)lim) : kWaitLimit;
  k_prep_tc<<<ls.tc_ctas, kPrepThreads, prep_tc_smem_bytes(), st>>>(dchains, ls.n_chains, maps, wl);
}

}  // namespace ctaux
