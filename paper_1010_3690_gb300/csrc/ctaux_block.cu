// One submatrix block of CT-AUX on every chain: pre-insertion (Sec. IV A),
// G0 gather, prep products, the k_max proposals with Gamma growth
// (Secs. III D and IV B) and the Woodbury flush with compaction (Sec. IV C).
#include <type_traits>

#include "ctaux_dev.cuh"

#include "ctaux_kernels.h"

namespace ctaux {

// ---------------------------------------------------------------- plan
// One CTA per chain: draw the block's move types, place the insertion
// candidates as s=0 vertices in slots [n, n + k_ins) (Sec. IV A) and record
// the block-start spins.
template <typename T>
__global__ void __launch_bounds__(256) k_plan(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.x];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const int n = d.n, buf = d.buf;
  const int64_t t0 = d.t;
  __shared__ int scan[256];
  const int j = threadIdx.x;
  int is_ins = 0;
  Draws dr;
  if (j < c.k_max) {
    dr = draw(c.seed, c.chain_id, t0 + j);
    is_ins = move_of(dr.u_move, c.p_insert, c.p_remove) == MV_INSERT;
  }
  scan[j] = is_ins;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const int v = (j >= off) ? scan[j - off] : 0;
    __syncthreads();
    scan[j] += v;
    __syncthreads();
  }
  const int k_ins = scan[255];
  const int m = n + k_ins;
  if (m > c.cap_m) {
    if (j == 0) atomicOr(&d.status, DS_CAPACITY);
    return;
  }
  if (j < c.k_max) {
    BlockDraw bd;
    bd.u_acc = dr.u_acc;
    bd.u_idx = dr.u_idx;
    bd.move = (int8_t)move_of(dr.u_move, c.p_insert, c.p_remove);
    bd.s_new = (int8_t)((dr.u_spin < 0.5) ? 1 : -1);
    bd.slot = is_ins ? n + scan[j] - 1 : -1;
    bd.pad = 0;
    c.draws[j] = bd;
  }
  if (is_ins) {
    const int slot = n + scan[j] - 1;
    int site = (int)floor(dr.u_site * (double)c.n_c);
    if (site > c.n_c - 1) site = c.n_c - 1;
    c.tau[buf][slot] = dr.u_tau * c.beta;
    c.site[buf][slot] = site;
    c.s[buf][slot] = 0;
    c.birth[buf][slot] = t0 + j;
  }
  for (int i = j; i < m; i += blockDim.x) c.s0[i] = (i < n) ? c.s[buf][i] : (int8_t)0;
  if (j == 0) {
    d.m = m;
    d.k_ins = k_ins;
  }
}

// -------------------------------------------------------------- gather
// G0 panels of the new vertices (Sec. IV A):
//   C[a][l] = G0(new_a, old_l) (e^{V_l} - 1)   (rows of R~ = C N)
//   B[l][a] = G0(old_l, new_a)                 (G_{:,new} = N_ext [B; G0(new,new)])
//   Gcol[n + a][b] = G0(new_a, new_b)          (accumulated onto by the prep products)
//   N_ext[:, n + a] = e_{n+a}                  (s=0 columns of N_ext are unit vectors)
template <typename T>
__global__ void __launch_bounds__(256) k_gather(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.z];
  const Dyn& d = *c.dyn;
  if (d.status) return;
  const int spin = blockIdx.y;
  const int n = d.n, k_ins = d.k_ins, m = d.m, buf = d.buf, ld = c.ld;
  const double* tau = c.tau[buf];
  const int* site = c.site[buf];
  T* Nb = c.N[buf][spin];
  const long nC = (long)k_ins * n, nB = nC, nG = (long)k_ins * k_ins, nI = (long)m * k_ins;
  const long total = nC + nB + nG + nI;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    if (e < nC) {
      const int a = (int)(e / n), l = (int)(e % n);
      const double ev = c.ev[spin][c.s0[l] + 2];
      c.Cpan[spin][(long)a * ld + l] =
          (T)(g0_eval(c, spin, tau[n + a], site[n + a], tau[l], site[l]) * (ev - 1.0));
    } else if (e < nC + nB) {
      const long f = e - nC;
      const int a = (int)(f / n), l = (int)(f % n);
      c.Bpan[spin][(long)a * ld + l] = (T)g0_eval(c, spin, tau[l], site[l], tau[n + a], site[n + a]);
    } else if (e < nC + nB + nG) {
      const long f = e - nC - nB;
      const int b = (int)(f / k_ins), a = (int)(f % k_ins);
      c.Gcol[spin][(long)b * ld + n + a] =
          (T)g0_eval(c, spin, tau[n + a], site[n + a], tau[n + b], site[n + b]);
    } else {
      const long f = e - nC - nB - nG;
      const int a = (int)(f / m), i = (int)(f % m);
      Nb[(long)(n + a) * ld + i] = (i == n + a) ? (T)1 : (T)0;
    }
  }
}

// ------------------------------------------------------ batched GEMM
// out(i,j) = alpha * sum_k A(i,k) B(k,j) + (cin ? cin(i,j) : 0), every operand
// a strided view with optional row/column index lists (gathers).
template <typename T>
struct View {
  const T* p;
  long rs, cs;
  const int* ri;
  const int* ci;
  __device__ __forceinline__ T at(int i, int j) const {
    const long r = ri ? ri[i] : i;
    const long q = ci ? ci[j] : j;
    return p[r * rs + q * cs];
  }
};

template <typename T>
struct Gemm {
  int M, Nn, Kk;
  double alpha;
  View<T> A, B, Cin;
  bool has_cin;
  T* out;
  long out_rs, out_cs;
};

template <typename T>
__device__ __forceinline__ bool setup_gemm(const Chain<T>& c, const Dyn& d, int spin, int phase,
                                           Gemm<T>& g) {
  const int ld = c.ld, n = d.n, k_ins = d.k_ins;
  T* Nb = c.N[d.buf][spin];
  g.alpha = 1.0;
  g.has_cin = false;
  g.A.ri = g.A.ci = g.B.ri = g.B.ci = g.Cin.ri = g.Cin.ci = nullptr;
  switch (phase) {
    case PH_RTILDE:  // R~ = C N -> N_ext rows [n, m), cols [0, n)
      g.M = k_ins; g.Nn = n; g.Kk = n;
      g.A.p = c.Cpan[spin]; g.A.rs = ld; g.A.cs = 1;
      g.B.p = Nb; g.B.rs = 1; g.B.cs = ld;
      g.out = Nb + n; g.out_rs = 1; g.out_cs = ld;
      break;
    case PH_GCOL_OLD:  // G_{old,new} = N B
      g.M = n; g.Nn = k_ins; g.Kk = n;
      g.A.p = Nb; g.A.rs = 1; g.A.cs = ld;
      g.B.p = c.Bpan[spin]; g.B.rs = 1; g.B.cs = ld;
      g.out = c.Gcol[spin]; g.out_rs = 1; g.out_cs = ld;
      break;
    case PH_GCOL_NEW:  // G_{new,new} = C G_{old,new} + G0(new,new)
      g.M = k_ins; g.Nn = k_ins; g.Kk = n;
      g.A.p = c.Cpan[spin]; g.A.rs = ld; g.A.cs = 1;
      g.B.p = c.Gcol[spin]; g.B.rs = 1; g.B.cs = ld;
      g.Cin.p = c.Gcol[spin] + n; g.Cin.rs = 1; g.Cin.cs = ld; g.has_cin = true;
      g.out = c.Gcol[spin] + n; g.out_rs = 1; g.out_cs = ld;
      break;
    case PH_FLUSH:  // N'[a,b] = N[S_a,S_b] - Y[a,:] N[P,S_b]
      g.M = d.flush_noop ? 0 : d.n_new; g.Nn = d.n_new; g.Kk = d.k_acc;
      g.alpha = -1.0;
      g.A.p = c.Y[spin]; g.A.rs = 1; g.A.cs = ld;
      g.B.p = Nb; g.B.rs = 1; g.B.cs = ld; g.B.ri = c.P; g.B.ci = c.S;
      g.Cin.p = Nb; g.Cin.rs = 1; g.Cin.cs = ld; g.Cin.ri = c.S; g.Cin.ci = c.S; g.has_cin = true;
      g.out = c.N[1 - d.buf][spin]; g.out_rs = 1; g.out_cs = ld;
      break;
    default:  // measurement: v_b = N g_b
      g.M = n; g.Nn = c.n_anchors; g.Kk = n;
      g.A.p = Nb; g.A.rs = 1; g.A.cs = ld;
      g.B.p = c.Mg[spin]; g.B.rs = 1; g.B.cs = ld;
      g.out = c.Mv[spin]; g.out_rs = 1; g.out_cs = ld;
      break;
  }
  return g.M > 0 && g.Nn > 0;
}

constexpr int GBK = 16;

// Tile variant of a product for a chain: the context's table (filled by the
// autotuner) at the chain's current order and k_max; 0 without a table.
template <typename T>
__device__ __forceinline__ int chain_tile_var(const Chain<T>& c, const Dyn& d, int phase) {
  return c.tile_var ? (int)c.tile_var[tile_table_index(phase, d.n, c.k_max)] : 0;
}

// Work items of one product for one chain: 2 spins x output tiles x slices
// of the inner dimension.  Slices are kchunk wide while the partial tiles
// they need fit in kMaxPartials per spin; products with more output tiles
// than that get fewer, wider slices (down to one).  The partition, and with
// it the rounding, depends only on the product's own sizes and the chain's
// tile variant: a chain gives the same bits alone or in a batch.
template <typename T, int PHASE>
__device__ __forceinline__ int gemm_items(const Chain<T>& c, const Dyn& d, int kchunk, int v,
                                          int& tiles_m, int& tiles_n, int& nslices, int& width) {
  const GemmTile tl = tile_variant(sizeof(T) == 8, PHASE, v);
  Gemm<T> g;
  if (d.status || !setup_gemm(c, d, 0, PHASE, g)) return 0;
  tiles_m = (g.M + tl.bm - 1) / tl.bm;
  tiles_n = (g.Nn + tl.bn - 1) / tl.bn;
  nslices = max(1, min((g.Kk + kchunk - 1) / kchunk, kMaxPartials / (tiles_m * tiles_n)));
  width = max(1, (g.Kk + nslices - 1) / nslices);
  return 2 * tiles_m * tiles_n * nslices;
}

// One (chain, spin, tile, slice) item of a product with tile variant V.
// As / Bs: shared staging with row strides SA / SB.
template <typename T, int PHASE, int V, int SA, int SB>
__device__ __forceinline__ void gemm_item(const Chain<T>& c, const Dyn& d, int l, int kchunk, T* As,
                                          T* Bs, int* s_last) {
  constexpr GemmTile tl = tile_variant(sizeof(T) == 8, PHASE, V);
  constexpr int GBM = tl.bm, GBN = tl.bn, TM = tl.tm, TN = tl.tn;
  constexpr int NTX = GBN / TN, NTY = GBM / TM;  // thread grid over the tile
  static_assert(NTX * NTY == 256, "256 threads per output tile");
  static_assert(GBM < SA && GBN < SB, "staging rows hold the tile");
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  int tiles_m, tiles_n, nslices, width;
  gemm_items<T, PHASE>(c, d, kchunk, V, tiles_m, tiles_n, nslices, width);
  const int per_spin = tiles_m * tiles_n * nslices;
  const int spin = l / per_spin, r0 = l % per_spin;
  const int tile = r0 / nslices, ks = r0 % nslices;
  Gemm<T> g;
  setup_gemm(c, d, spin, PHASE, g);
  const int i0 = (tile / tiles_n) * GBM, j0 = (tile % tiles_n) * GBN;
  const int kb = ks * width, ke = min(g.Kk, kb + width);
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = (T)0;
  // the next K step's operands are loaded into registers while the current
  // one is multiplied from shared memory (global latency off the FMA path)
  constexpr int PA = (GBK * GBM + 255) / 256, PB = (GBK * GBN + 255) / 256;
  T ra[PA], rb[PB];
#pragma unroll
  for (int q = 0; q < PA; ++q) {
    const int e = threadIdx.x + 256 * q, ii = e % GBM, kk = e / GBM;
    const int i = i0 + ii, k = kb + kk;
    ra[q] = (e < GBK * GBM && i < g.M && k < ke) ? g.A.at(i, k) : (T)0;
  }
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int e = threadIdx.x + 256 * q, kk = e % GBK, jj = e / GBK;
    const int j = j0 + jj, k = kb + kk;
    rb[q] = (e < GBK * GBN && j < g.Nn && k < ke) ? g.B.at(k, j) : (T)0;
  }
  for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < GBK * GBM) As[(e / GBM) * SA + e % GBM] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < GBK * GBN) Bs[(e % GBK) * SB + e / GBK] = rb[q];
    }
    __syncthreads();
    const int k1 = k0 + GBK;
    if (k1 < ke) {
#pragma unroll
      for (int q = 0; q < PA; ++q) {
        const int e = threadIdx.x + 256 * q, ii = e % GBM, kk = e / GBM;
        const int i = i0 + ii, k = k1 + kk;
        ra[q] = (e < GBK * GBM && i < g.M && k < ke) ? g.A.at(i, k) : (T)0;
      }
#pragma unroll
      for (int q = 0; q < PB; ++q) {
        const int e = threadIdx.x + 256 * q, kk = e % GBK, jj = e / GBK;
        const int j = j0 + jj, k = k1 + kk;
        rb[q] = (e < GBK * GBN && j < g.Nn && k < ke) ? g.B.at(k, j) : (T)0;
      }
    }
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk * SA + ty + NTY * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kk * SB + tx + NTX * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  if (nslices > 1) {
    // the measurement product has partial tiles and tickets of its own: it
    // may run beside a block's products
    T* part = (PHASE == PH_MEAS ? c.kpart_meas[spin] : c.kpart[spin]) + (size_t)tile * nslices * GBM * GBN;
    int* tickets = PHASE == PH_MEAS ? c.ticket_meas[spin] : c.ticket[spin];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b)
        part[(size_t)ks * GBM * GBN + (ty + NTY * a) * GBN + tx + NTX * b] = acc[a][b];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = (atomicAdd(tickets + tile, 1) == nslices - 1);
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        T v = (T)0;
        for (int q = 0; q < nslices; ++q)
          v += __ldcg(part + (size_t)q * GBM * GBN + (ty + NTY * a) * GBN + tx + NTX * b);
        acc[a][b] = v;
      }
    if (threadIdx.x == 0) tickets[tile] = 0;
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int i = i0 + ty + NTY * a;
    if (i >= g.M) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int j = j0 + tx + NTX * b;
      if (j >= g.Nn) continue;
      T v = (T)g.alpha * acc[a][b];
      if (g.has_cin) v += g.Cin.at(i, j);
      g.out[(long)i * g.out_rs + (long)j * g.out_cs] = v;
    }
  }
}

// Persistent batched product: CTAs loop over the (chain, spin, tile, slice)
// items of the chains whose tile variant for this product is V (one launch
// per variant in use).  One output tile and one slice per item (256
// threads).  With more than one slice every slice stores its partial tile,
// and the slice that arrives last at the tile's ticket adds the partials in
// slice order (deterministic, no waiting) and writes the result.
template <typename T, int PHASE, int V>
__global__ void __launch_bounds__(256) k_gemm(Chain<T>* chains, int n_chains, int kchunk) {
  constexpr GemmTile tl = tile_variant(sizeof(T) == 8, PHASE, V);
  constexpr int SA = tl.bm + 1, SB = tl.bn + 1;
  __shared__ int off[kMaxChains + 1];
  __shared__ T As[GBK * SA];
  __shared__ T Bs[GBK * SB];
  __shared__ int s_last;
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
    int a, b, q, wd;
    const Chain<T>& c = chains[ci];
    off[ci] = (chain_tile_var(c, *c.dyn, PHASE) == V)
                  ? gemm_items<T, PHASE>(c, *c.dyn, kchunk, V, a, b, q, wd)
                  : 0;
  }
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int ci = find_chain(off, n_chains, w);
    gemm_item<T, PHASE, V, SA, SB>(chains[ci], *chains[ci].dyn, w - off[ci], kchunk, As, Bs,
                                   &s_last);
  }
}

template <typename T, int PHASE>
void launch_gemm_variants(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st) {
  const dim3 grid(ls.persist_ctas);
  const int n = ls.n_chains, kc = ls.kchunk, mask = ls.tile_mask[PHASE];
  if (mask & 1) k_gemm<T, PHASE, 0><<<grid, 256, 0, st>>>(dchains, n, kc);
  if (mask & 2) k_gemm<T, PHASE, 1><<<grid, 256, 0, st>>>(dchains, n, kc);
  if (mask & 4) k_gemm<T, PHASE, 2><<<grid, 256, 0, st>>>(dchains, n, kc);
}

// One product for every chain: one launch per tile variant the context's
// table holds for it (only variant 0 without a tuned table).
template <typename T>
int launch_gemm(Chain<T>* dchains, const LaunchShape& ls, int phase, cudaStream_t st) {
  switch (phase) {
    case PH_RTILDE: launch_gemm_variants<T, PH_RTILDE>(dchains, ls, st); break;
    case PH_GCOL_OLD: launch_gemm_variants<T, PH_GCOL_OLD>(dchains, ls, st); break;
    case PH_GCOL_NEW: launch_gemm_variants<T, PH_GCOL_NEW>(dchains, ls, st); break;
    case PH_FLUSH: launch_gemm_variants<T, PH_FLUSH>(dchains, ls, st); break;
    default: launch_gemm_variants<T, PH_MEAS>(dchains, ls, st); break;
  }
  return __builtin_popcount(ls.tile_mask[phase]);
}

// ------------------------------------------------------------ proposals
// Interacting Green's function of the block start, G0int(i, j) = G^0_{ij}
// (Sec. III C: "G^0 is the interacting Green's function at step k=0"):
// old columns from N by G = (N e^V - 1)/(e^V - 1) (Eq. NfromG), new (s=0)
// columns from the prep product G_{:,new} = N_ext G0_{:,new}.  Evaluated in
// the arithmetic type A of the form (float64, or float32 in the mixed form).
template <typename A, typename T>
__device__ __forceinline__ A g_int(const Chain<T>& c, const T* Nb, const T* Gc, int n_old, int spin,
                                   int i, int j) {
  if (j < n_old) {
    const int k = c.s0[j] + 2;
    return ((A)Nb[(long)j * c.ld + i] * (A)c.ev[spin][k] - (i == j ? (A)1 : (A)0)) *
           (A)c.inv_em1[spin][k];
  }
  return (A)Gc[(long)(j - n_old) * c.ld + i];
}

// Select the idx-th set bit of a bitmask (one warp).
__device__ __forceinline__ int select_bit(const uint32_t* mask, int n_words, int idx, int lane) {
  int base = 0;
  for (int w0 = 0; w0 < n_words; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t word = (w < n_words) ? mask[w] : 0u;
    const int cnt = __popc(word);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (idx < base + total) {
      const int excl = incl - cnt;
      const bool mine = (idx >= base + excl) && (idx < base + incl);
      const unsigned who = __ballot_sync(0xffffffffu, mine);
      const int src = __ffs(who) - 1;
      int res = -1;
      if (lane == src) res = w * 32 + (__fns(word, 0, idx - base - excl + 1));
      return __shfl_sync(0xffffffffu, res, src);
    }
    base += total;
  }
  return -1;
}

template <typename A>
__device__ __forceinline__ A warp_sum_t(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Relative guard band of the mixed form's tie detection when the FP64
// re-evaluation is off (counted only).  The decision is u < |R| (u < 1, so
// |R| >= 1 always accepts): a float32 |R| with relative error below g can
// change it only when |u - |R|| < g max(u, |R|), which never holds once
// |R| >= 1 / (1 - g).
constexpr double kTieGuard = 1e-4;

// ---- Gamma kept as L U (Sec. III D, the factorisation variant) ----
// L (unit lower, strictly-lower part stored) and U (upper, diagonal included)
// share one j x j array with row stride LG; iu[i] = 1 / U_ii.  Every function
// below is called by both spin halves of the CTA with the same j and start
// index, so the CTA-wide barriers inside match.

// In place: y <- L^{-1} y (Eq. lineq1) and x <- U^{-T} x (Eq. lineq2) over
// rows [r_start, j), entries below r_start being zero.  Blocks of 32 rows: a
// diagonal block is solved by one warp with shuffles (warp 0 of the half for
// y, warp 1 for x), then the 128 threads of the half subtract its
// contribution from the rows below.
template <typename T, typename A>
__device__ __forceinline__ void lu_solve_pair(const T* G, int LG, const A* iu, A* y, A* x, int r_start,
                                              int j, int ht, int hw, int lane) {
  for (int r0 = r_start & ~31; r0 < j; r0 += 32) {
    const int r1 = min(j, r0 + 32), nb = r1 - r0, r = r0 + lane;
    if (hw < 2) {
      // the diagonal block first, in registers (one memory latency instead of
      // one per step): warp 0 lane i holds L[r0 + i][r0 + t], warp 1 lane i
      // holds U[r0 + t][r0 + i], for t < i
      A m[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const bool in = t < lane && r < r1;
        m[t] = in ? (A)(hw == 0 ? G[(size_t)r * LG + r0 + t] : G[(size_t)(r0 + t) * LG + r]) : (A)0;
      }
      if (hw == 0) {
        A v = (r < r1) ? y[r] : (A)0;
#pragma unroll
        for (int t = 0; t < 31; ++t) {
          const A yt = __shfl_sync(0xffffffffu, v, t);
          if (t < lane) v -= m[t] * yt;
        }
        if (r < r1) y[r] = v;
      } else {
        const A iur = (r < r1) ? iu[r] : (A)0;
        A v = (r < r1) ? x[r] : (A)0;
#pragma unroll
        for (int t = 0; t < 31; ++t) {
          const A xt = __shfl_sync(0xffffffffu, v, t) * __shfl_sync(0xffffffffu, iur, t);
          if (t < lane) v -= m[t] * xt;
        }
        if (r < r1) x[r] = v * iur;
      }
    }
    __syncthreads();
    if (r1 < j) {
      // rows below the block: y_r -= L[r, blk] y_blk (threads [0, j - r1)),
      // x_r -= U[blk, r]^T x_blk (the next j - r1 threads: U's rows are read
      // along r, coalesced); several loads in flight per thread
      const int below = j - r1;
      for (int e = ht; e < 2 * below; e += 128) {
        const bool isx = e >= below;
        const int rr = r1 + (isx ? e - below : e);
        A a0 = (A)0, a1 = (A)0;
        if (isx) {
          const T* Uc = G + (size_t)r0 * LG + rr;
#pragma unroll 8
          for (int t = 0; t < nb; t += 2) {
            a0 += (A)Uc[(size_t)t * LG] * x[r0 + t];
            if (t + 1 < nb) a1 += (A)Uc[(size_t)(t + 1) * LG] * x[r0 + t + 1];
          }
          x[rr] -= a0 + a1;
        } else {
          const T* Lr = G + (size_t)rr * LG + r0;
#pragma unroll 8
          for (int t = 0; t < nb; t += 2) {
            a0 += (A)Lr[t] * y[r0 + t];
            if (t + 1 < nb) a1 += (A)Lr[t + 1] * y[r0 + t + 1];
          }
          y[rr] -= a0 + a1;
        }
      }
      __syncthreads();
    }
  }
}

// Bennett's update of L U to the factors of L U + xb yb^T, touching pivots
// [i0, j) (xb and yb are zero below i0; both are overwritten).  Step i: U_ii
// += xb_i yb_i, c = yb_i / U_ii; for r > i: xb_r -= xb_i L_ri, L_ri += c xb_r;
// U_ir += xb_i yb_r, yb_r -= c U_ir.
template <typename T, typename A>
__device__ __forceinline__ void lu_rank_one(T* G, int LG, A* iu, A* xb, A* yb, int i0, int j, int ht,
                                            A* coef) {
  for (int i = i0; i < j; ++i) {
    if (ht == 0) {
      const T uii = (T)((A)G[(size_t)i * LG + i] + xb[i] * yb[i]);
      G[(size_t)i * LG + i] = uii;
      const A inv = (A)1 / (A)uii;
      iu[i] = inv;
      *coef = yb[i] * inv;
    }
    __syncthreads();
    const A xi = xb[i], cf = *coef;
    for (int r = i + 1 + ht; r < j; r += 128) {
      const A lri = (A)G[(size_t)r * LG + i];
      const A xr = xb[r] - xi * lri;
      xb[r] = xr;
      G[(size_t)r * LG + i] = (T)(lri + cf * xr);
      const A uir = (A)G[(size_t)i * LG + r] + xi * yb[r];
      G[(size_t)i * LG + r] = (T)uir;
      yb[r] -= cf * uir;
    }
    __syncthreads();
  }
}

// One CTA per chain, threads [0,128) spin up, [128,256) spin down.  Runs the
// k_max proposals of the block in order; Gamma^{-1} (row-major, row stride
// k_max + 1) is grown by partitioning (Sec. III D): beta = d - w^T Gamma^{-1} s,
// ratio_sigma = -lambda beta (Eq. ratS), the bordered inverse on acceptance.
// A slot touched twice in a block changes only the diagonal of Gamma
// (Eq. Gamma): Sherman-Morrison on Gamma^{-1}, or removal of the slot from P
// when it returns to its block-start spin (then ratio = -(Gamma^{-1})_qq / lambda).
// Arithmetic in T (float64, or float32 in the mixed form, which counts near
// ties of the accept decision).  LU: Gamma = L U instead (Eqs. lineq1-detrat):
// beta = d - x^T y with y = L^{-1} s, x = U^{-T} w; an accepted first touch
// appends x^T to L and (y, beta) to U; (Gamma^{-1})_qq of a re-touched slot is
// x^T y for s = w = e_q; accepted re-touches re-factorise by Bennett's update
// (diagonal change: xb = delta e_q, yb = e_q; return to the block-start spin:
// row and column q deleted, which leaves the outer product of q's old L column
// and U row).
template <typename T, bool GS, bool LU>
__device__ __forceinline__ void proposals_body(Chain<T>* chains) {
  constexpr bool gamma_in_smem = GS;  // Gamma^{-1} in shared memory: known at compile time, so
                                      // its accesses are shared-memory instructions
  using A = T;
  const Chain<T>& c = chains[blockIdx.x];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const int tid = threadIdx.x, half = tid >> 7, ht = tid & 127, hw = ht >> 5, lane = tid & 31;
  const int spin = half;
  const int KM = c.k_max, LG = c.k_max + 1, ld = c.ld;
  const int n_old = d.n, m = d.m, buf = d.buf;
  const int64_t t0 = d.t;
  const T* Nb = c.N[buf][spin];
  const T* Gc = c.Gcol[spin];
  int8_t* s_cur = c.s[buf];
  const int64_t* birth = c.birth[buf];

  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: [Gamma^{-1} 2 x KM x LG (optional)] [vec 2 x 4 x KM] [lam 2 x KM double]
  //         [P KM int] [pmap cap_m short] [alive mask] [1/lambda 2 x KM double]
  //         [block-start spins cap_m]
  unsigned char* sp = smem_raw;
  T* Gs = nullptr;
  if (gamma_in_smem) {
    Gs = reinterpret_cast<T*>(sp);
    sp += (sizeof(T) * 2 * KM * LG + 15) & ~size_t(15);
  }
  A* vec = reinterpret_cast<A*>(sp);
  sp += (sizeof(A) * 8 * KM + 15) & ~size_t(15);
  double* lam_s = reinterpret_cast<double*>(sp);
  sp += sizeof(double) * 2 * KM;
  int* P_s = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * KM;
  short* pmap = reinterpret_cast<short*>(sp);
  sp += sizeof(short) * ((c.cap_m + 7) & ~7);
  uint32_t* alive = reinterpret_cast<uint32_t*>(sp);
  const int n_words = (m + 31) / 32;
  sp += sizeof(uint32_t) * ((c.cap_m + 31) / 32);
  sp = reinterpret_cast<unsigned char*>(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  double* ilam_s = reinterpret_cast<double*>(sp);   // 1/lambda of the slots in P, per spin
  sp += sizeof(double) * 2 * KM;
  A* iu_s = reinterpret_cast<A*>(sp);               // LU form: 1 / U_ii, per spin
  sp += sizeof(double) * 2 * KM;
  int8_t* s0_s = reinterpret_cast<int8_t*>(sp);     // block-start spins

  T* G;
  if constexpr (GS) G = Gs + (size_t)spin * KM * LG;
  else G = LU ? c.Glu[spin] : c.Ginv[spin];
  A* iu = iu_s + spin * KM;
  A* sv = vec + spin * 4 * KM;   // s (column of G^0 over P)
  A* wv = sv + KM;               // w (row of G^0 over P)
  A* yv = wv + KM;               // Gamma^{-1} s
  A* zv = yv + KM;               // w^T Gamma^{-1}
  double* lam = lam_s + spin * KM;

  double* ilam = ilam_s + spin * KM;

  __shared__ A red[2][4];
  __shared__ A gpp_s[2];
  __shared__ double ratio_s[2];
  __shared__ A raw_s[2];        // per spin: beta (first touch), delta or Gamma^{-1}_qq (re-touch)
  __shared__ A gqq_s[2];
  __shared__ A scal_s[2];       // per spin: 1/beta, Sherman-Morrison coefficient or Schur pivot
  __shared__ A coef_s[2];       // LU form: Bennett coefficient of the current pivot
  __shared__ double lamn_s[2];  // per spin: lambda of the proposed change
  __shared__ double ev_s[2][5], iem1_s[2][5];
  __shared__ A glam_s[2][5];
  __shared__ int dec_s;         // 0 reject, 1 accept, 2 near tie (stop)
  __shared__ int fin_s;         // the decision's finite flag, forced flag
  __shared__ double R_s;
  __shared__ double f_s;        // move factor K/(n+1), n/K or 1
  __shared__ int sel_p;
  __shared__ int jP;
  __shared__ int n_cur, sign_s;
  __shared__ long long cnt_prop[3], cnt_acc[3], numeric, ties;
  __shared__ long long flops2;  // algorithmic flops / 2 (integer: no float64 work)
  __shared__ BlockDraw bd_s[kMaxK];

  for (int i = tid; i < m; i += 256) {
    pmap[i] = -1;
    s0_s[i] = c.s0[i];
  }
  for (int w = tid; w < n_words; w += 256) {
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
      const int i = w * 32 + b;
      if (i < m && s_cur[i] != 0) bits |= (1u << b);
    }
    alive[w] = bits;
  }
  if (tid < 10) {
    const int sp_ = tid / 5, k_ = tid % 5;
    ev_s[sp_][k_] = c.ev[sp_][k_];
    iem1_s[sp_][k_] = c.inv_em1[sp_][k_];
    glam_s[sp_][k_] = c.glam[sp_][k_];
  }
  if (tid == 0) {
    jP = 0;
    n_cur = n_old;
    sign_s = d.sign;
    for (int q = 0; q < 3; ++q) cnt_prop[q] = cnt_acc[q] = 0;
    numeric = 0;
    ties = 0;
    flops2 = 0;
  }
  for (int e = tid; e < KM; e += 256) bd_s[e] = c.draws[e];
  // read once: the decision of a near tie taken in FP64 after the previous block
  const int64_t forced_t = (sizeof(T) == 4) ? d.forced_t : -1;
  const double tie_guard = (sizeof(T) == 4 && c.tie_guard > 0.0) ? d.guard_eff : 0.0;
  const int trace_cap = c.trace_cap;
  const int64_t trace_base = d.trace_written;
  __syncthreads();
  int consumed = KM;

  // The chain of a proposal is latency-bound: every step between two barriers
  // is kept short.  Scalar float64 work (the move factor, divisions, the
  // Metropolis decision) runs on one thread per spin half or per CTA and is
  // shared through shared memory (GB300 executes float64 at 1/64 of the
  // float32 rate: a warp-wide float64 instruction holds the pipe ~16 cycles);
  // the divisions needed only on acceptance and the trace record are done
  // beside the decision, by other threads; warps without rows or columns skip
  // the float64 reductions; the tables and block-start spins are in shared
  // memory.
  for (int jj = 0; jj < KM; ++jj) {
    const int64_t t = t0 + jj;
    const BlockDraw dr = bd_s[jj];
    const int move = dr.move;
    const int nc = n_cur;
    int p = -1, s_new = 0;
    if (move == MV_INSERT) {
      p = dr.slot;
      s_new = dr.s_new;
    } else if (nc > 0) {
      if (tid < 32) {
        int idx = (int)floor(dr.u_idx * (double)nc);
        if (idx > nc - 1) idx = nc - 1;
        const int ps = select_bit(alive, n_words, idx, lane);
        if (lane == 0) sel_p = ps;
      }
      __syncthreads();
      p = sel_p;
      if (p < 0 || p >= m) {
        if (tid == 0) atomicOr(&d.status, DS_INDEX);
        break;
      }
      s_new = (move == MV_REMOVE) ? 0 : -(int)s_cur[p];
    }
    // move factor, off the critical path (warp 6 has no gather or matrix-vector
    // rows while j <= 64); read by thread 0 after two barriers
    if (tid == 192)
      f_s = (move == MV_INSERT) ? c.K / (double)(nc + 1) : (move == MV_REMOVE ? (double)nc / c.K : 1.0);
    if (p < 0) {  // removal or flip with no vertex: automatic rejection
      if (tid == 0) {
        cnt_prop[move]++;
        if (trace_cap > 0) {
          TraceRec& r = c.trace[(trace_base + jj) % trace_cap];
          r.t = t; r.move = move; r.n = nc; r.birth = -1; r.s_new = 0; r.accept = 0;
          r.ratio[0] = r.ratio[1] = 0.0; r.R = 0.0; r.u = dr.u_acc;
        }
      }
      continue;
    }
    const int q = pmap[p];
    const int j = jP;
    const int s_start = s0_s[p];
    const int dk = s_new - s_start + 2;   // index of lambda_new in the tables
    const bool to_start = (s_new == s_start);  // lambda_new = 0
    if (q < 0) {
      // first touch: gather s = G^0_{P,p}, w = G^0_{p,P}, G^0_pp
      // (G = (N e^V - 1)/(e^V - 1) for old columns, Eq. NfromG; prep columns for new ones)
      for (int r = ht; r < j; r += 128) {
        const int pr = P_s[r];
        const int kp = s0_s[p] + 2, kr = s0_s[pr] + 2;
        sv[r] = (p < n_old)
                    ? ((A)Nb[(long)p * ld + pr] * (A)ev_s[spin][kp] - (A)0) * (A)iem1_s[spin][kp]
                    : (A)Gc[(long)(p - n_old) * ld + pr];
        wv[r] = (pr < n_old)
                    ? ((A)Nb[(long)pr * ld + p] * (A)ev_s[spin][kr] - (A)0) * (A)iem1_s[spin][kr]
                    : (A)Gc[(long)(pr - n_old) * ld + p];
      }
      if (ht == 127) gpp_s[half] = g_int<A>(c, Nb, Gc, n_old, spin, p, p);
      __syncthreads();
      if constexpr (LU) {
        // s -> y = L^{-1} s, w -> x = U^{-T} w, partial sums of x . y
        lu_solve_pair<T, A>(G, LG, iu, sv, wv, 0, j, ht, hw, lane);
        A part = (A)0;
        for (int r = ht; r < j; r += 128) part += sv[r] * wv[r];
        part = warp_sum_t(part);
        if (lane == 0) red[half][hw] = part;
      } else
      // y = Gamma^{-1} s and the partial sums of w . y (z = w^T Gamma^{-1} only
      // on acceptance).  float64: four threads per row, combined by shuffles;
      // float32: one thread per row, two accumulators.
      {
        A part = (A)0;
        if constexpr (sizeof(A) == 8) {
          const int quad = ht & 3;
          for (int r0 = 0; r0 < j; r0 += 32) {
            if (r0 + (ht >> 2) - (lane >> 2) >= j) break;  // warp without rows (uniform)
            const int r = r0 + (ht >> 2);
            A acc = (A)0;
            if (r < j) {
              const T* Gr = G + (size_t)r * LG;
              for (int cc = quad; cc < j; cc += 4) acc += (A)Gr[cc] * sv[cc];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (r < j && quad == 0) {
              yv[r] = acc;
              part += wv[r] * acc;
            }
          }
        } else if constexpr (GS) {
          for (int r = ht; r < j; r += 128) {
            A a0 = (A)0, a1 = (A)0;
            const T* Gr = G + (size_t)r * LG;
            int cc = 0;
            for (; cc + 1 < j; cc += 2) {
              a0 += (A)Gr[cc] * sv[cc];
              a1 += (A)Gr[cc + 1] * sv[cc + 1];
            }
            if (cc < j) a0 += (A)Gr[cc] * sv[cc];
            const A y = a0 + a1;
            yv[r] = y;
            part += wv[r] * y;
          }
        } else {
          // Gamma^{-1} in global memory: four accumulators, several loads in flight
          for (int r = ht; r < j; r += 128) {
            A a0 = (A)0, a1 = (A)0, a2 = (A)0, a3 = (A)0;
            const T* Gr = G + (size_t)r * LG;
            int cc = 0;
            for (; cc + 3 < j; cc += 4) {
              a0 += (A)Gr[cc] * sv[cc];
              a1 += (A)Gr[cc + 1] * sv[cc + 1];
              a2 += (A)Gr[cc + 2] * sv[cc + 2];
              a3 += (A)Gr[cc + 3] * sv[cc + 3];
            }
            for (; cc < j; ++cc) a0 += (A)Gr[cc] * sv[cc];
            const A y = (a0 + a1) + (a2 + a3);
            yv[r] = y;
            part += wv[r] * y;
          }
        }
        // warps that hold rows reduce their part; the others contribute 0
        const bool has_rows = (sizeof(A) == 8) ? (hw * 8 < j) : (hw * 32 < j);
        if (has_rows) part = warp_sum_t(part);
        if (lane == 0) red[half][hw] = has_rows ? part : (A)0;
      }
      __syncthreads();
      if (ht == 0) {
        const double lam_new = ev_s[spin][dk] - 1.0;
        const A lam_a = (A)lam_new;
        const A dd = gpp_s[half] - glam_s[spin][dk];  // (1 + lambda) / lambda
        const A beta = dd - ((red[half][0] + red[half][1]) + (red[half][2] + red[half][3]));
        ratio_s[half] = (double)(-lam_a * beta);
        raw_s[half] = beta;
        lamn_s[half] = lam_new;
      }
    } else {
      if constexpr (LU) {
        // (Gamma^{-1})_qq = x^T y with y = L^{-1} e_q, x = U^{-T} e_q
        for (int r = ht; r < j; r += 128) sv[r] = wv[r] = (r == q) ? (A)1 : (A)0;
        __syncthreads();
        lu_solve_pair<T, A>(G, LG, iu, sv, wv, q, j, ht, hw, lane);
        A part = (A)0;
        for (int r = q + ht; r < j; r += 128) part += sv[r] * wv[r];
        part = warp_sum_t(part);
        if (lane == 0) red[half][hw] = part;
        __syncthreads();
      }
      if (ht == 0) {
      const double lam_new = ev_s[spin][dk] - 1.0;
      const A lam_a = (A)lam_new;
      const A ilo = (A)ilam[q];  // 1 / lambda of the slot's first change
      const A gqq = LU ? (red[half][0] + red[half][1]) + (red[half][2] + red[half][3])
                       : (A)G[(size_t)q * LG + q];
      A r;
      if (!to_start) {
        const A delta = ilo - (A)iem1_s[spin][dk];  // 1/lambda_old - 1/lambda_new
        r = (lam_a * ilo) * ((A)1 + delta * gqq);
        raw_s[half] = delta;
      } else {
        r = -gqq * ilo;
      }
      gqq_s[half] = gqq;
      ratio_s[half] = (double)r;
      lamn_s[half] = lam_new;
      }
    }
    __syncthreads();
    if (tid == 0) {
      double R;
      bool accept, finite, near;
      // float32 form: the product and the comparisons in float32 (the ratios
      // are float32 already; a decision that the rounding of the product or of
      // u could change lies inside the guard band, which is decided in FP64),
      // unless the float32 product overflows
      const float Rf = (sizeof(T) == 4) ? (float)f_s * (float)ratio_s[0] * (float)ratio_s[1] : 0.f;
      if (sizeof(T) == 4 && isfinite(Rf)) {
        const float uf = (float)dr.u_acc, aR = fabsf(Rf);
        R = (double)Rf;
        finite = true;
        accept = uf < fminf(1.f, aR);
        near = fabsf(uf - aR) < (float)(tie_guard > 0.0 ? tie_guard : kTieGuard) * fmaxf(uf, aR);
      } else {
        R = f_s * ratio_s[0] * ratio_s[1];
        accept = dr.u_acc < fmin(1.0, fabs(R));
        finite = isfinite(R);
        near = (sizeof(T) == 4) && finite &&
               fabs(dr.u_acc - fabs(R)) < (tie_guard > 0.0 ? tie_guard : kTieGuard) * fmax(dr.u_acc, fabs(R));
      }
      if (!finite) accept = false;
      const bool forced = (sizeof(T) == 4) && forced_t == t;
      int dec;
      if (forced) {
        // decided in FP64 after the previous block stopped here (k_tie_refine)
        accept = d.forced_accept != 0;
        R = d.forced_R;
        finite = true;
        dec = accept ? 1 : 0;
      } else if (sizeof(T) == 4 && tie_guard > 0.0 && finite && near) {
        // near tie in the float32 form: the block ends before this proposal,
        // which is decided in FP64 after the flush
        d.tie_pending = 1;
        d.tie_jj = jj;
        d.tie_R32 = R;
        ties++;
        dec = 2;
      } else {
        dec = accept ? 1 : 0;
        if (sizeof(T) == 4 && tie_guard == 0.0 && finite && near)
          ties++;  // detection only (FP64 re-evaluation off)
      }
      if (dec != 2) {
        if (!finite) numeric++;
        if (accept && R < 0.0) sign_s = -sign_s;
        if (forced) d.forced_t = -1;
      }
      R_s = R;
      fin_s = forced ? 1 : 0;
      dec_s = dec;
    } else if ((tid == 32 || tid == 160) && q < 0) {
      // 1 / beta of this spin, needed only on acceptance, beside the decision
      scal_s[half] = (A)1 / raw_s[half];
    } else if ((tid == 32 || tid == 160) && !to_start) {
      const A delta = raw_s[half];
      scal_s[half] = delta / ((A)1 + delta * gqq_s[half]);  // Sherman-Morrison coefficient
    } else if (tid == 32 || tid == 160) {
      scal_s[half] = (A)1 / gqq_s[half];  // Schur complement pivot
    }
    __syncthreads();
    const int dec = dec_s;
    if (dec == 2) {
      consumed = jj;
      break;
    }
    if (tid == 64) {
      // counters and the trace record, off the critical path
      const bool accept = dec == 1;
      cnt_prop[move]++;
      if (accept) cnt_acc[move]++;
      // algorithmic flops, both spins: y GEMV and the dot (first touch); on
      // acceptance the z GEMV and the bordered update, or the rank-one update
      const long long jl = j;
      long long fl;
      if constexpr (LU) {
        // two triangular solves and the dot (over rows >= q for a re-touch);
        // Bennett's update on an accepted re-touch, the append costs nothing
        const long long jq = (q < 0) ? jl : jl - q;
        fl = 2 * jq * jq + 2 * jq;
        if (accept && q >= 0) fl += 3 * jq * jq;
      } else {
        fl = (q < 0) ? (2 * jl * jl + 2 * jl) : 4;
        if (accept) fl += (q < 0) ? 2 * jl * jl + 3 * (jl + 1) * (jl + 1) : 3 * jl * jl;
      }
      flops2 += fl;
      if (trace_cap > 0) {
        const bool forced = fin_s != 0;
        TraceRec& rr = c.trace[(trace_base + jj) % trace_cap];
        rr.t = t; rr.move = move; rr.n = nc;
        rr.birth = birth[p]; rr.s_new = s_new; rr.accept = (accept ? 1 : 0) | (forced ? 2 : 0);
        rr.ratio[0] = forced ? d.forced_ratio[0] : ratio_s[0];
        rr.ratio[1] = forced ? d.forced_ratio[1] : ratio_s[1];
        rr.R = R_s; rr.u = dr.u_acc;
      }
    }
    if (dec == 1 && LU) {
      if (q < 0) {
        // bordering: L gains the row x^T, U the column (y, beta)
        for (int l = ht; l < j; l += 128) {
          G[(size_t)j * LG + l] = (T)wv[l];
          G[(size_t)l * LG + j] = (T)sv[l];
        }
        if (ht == 0) {
          G[(size_t)j * LG + j] = (T)raw_s[half];
          iu[j] = scal_s[half];
          lam[j] = lamn_s[half];
          ilam[j] = iem1_s[spin][dk];
        }
      } else if (!to_start) {
        // Gamma_qq += delta: Bennett with xb = delta e_q, yb = e_q
        const A delta = raw_s[half];
        for (int r = ht; r < j; r += 128) {
          sv[r] = (r == q) ? delta : (A)0;
          wv[r] = (r == q) ? (A)1 : (A)0;
        }
        __syncthreads();
        lu_rank_one<T, A>(G, LG, iu, sv, wv, q, j, ht, &coef_s[half]);
        if (ht == 0) {
          lam[q] = lamn_s[half];
          ilam[q] = iem1_s[spin][dk];
        }
      } else {
        // delete row and column q; what remains is L'U' + (L[>q, q]) (U[q, >q])^T
        for (int r = q + 1 + ht; r < j; r += 128) {
          sv[r - 1] = (A)G[(size_t)r * LG + q];
          wv[r - 1] = (A)G[(size_t)q * LG + r];
        }
        __syncthreads();
        for (int r = ht; r < j; r += 128)
          for (int cc = q; cc < j - 1; ++cc) G[(size_t)r * LG + cc] = G[(size_t)r * LG + cc + 1];
        __syncthreads();
        for (int cc = ht; cc < j - 1; cc += 128)
          for (int r = q; r < j - 1; ++r) G[(size_t)r * LG + cc] = G[(size_t)(r + 1) * LG + cc];
        if (ht == 0)
          for (int l = q; l < j - 1; ++l) {
            lam[l] = lam[l + 1];
            ilam[l] = ilam[l + 1];
          }
        __syncthreads();
        lu_rank_one<T, A>(G, LG, iu, sv, wv, q, j - 1, ht, &coef_s[half]);
      }
      __syncthreads();
      if (tid == 0) {
        if (q < 0) {
          P_s[j] = p;
          pmap[p] = (short)j;
          jP = j + 1;
        } else if (to_start) {
          // later entries of P move down one place (the factors' order)
          for (int l = q; l < j - 1; ++l) {
            P_s[l] = P_s[l + 1];
            pmap[P_s[l]] = (short)l;
          }
          pmap[p] = -1;
          jP = j - 1;
        }
        s_cur[p] = (int8_t)s_new;
        if (s_new == 0) alive[p >> 5] &= ~(1u << (p & 31));
        else alive[p >> 5] |= (1u << (p & 31));
        if (move == MV_INSERT) n_cur = nc + 1;
        else if (move == MV_REMOVE) n_cur = nc - 1;
      }
    } else if (dec == 1) {
      const A sc = scal_s[half];
      if (q < 0) {
        // z = w^T Gamma^{-1} (scaled by 1/beta), then the bordered inverse
        // (Sec. III D): [[G + y z / beta, -y / beta], [-z / beta, 1 / beta]]
        if constexpr (sizeof(A) == 8) {
          const int quad = ht & 3;
          for (int c0 = 0; c0 < j; c0 += 32) {
            if (c0 + (ht >> 2) - (lane >> 2) >= j) break;  // warp without columns (uniform)
            const int cc = c0 + (ht >> 2);
            A acc = (A)0;
            if (cc < j)
              for (int r = quad; r < j; r += 4) acc += wv[r] * (A)G[(size_t)r * LG + cc];
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (cc < j && quad == 0) zv[cc] = acc * sc;
          }
        } else {
          for (int cc = ht; cc < j; cc += 128) {
            A a0 = (A)0, a1 = (A)0, a2 = (A)0, a3 = (A)0;
            int r = 0;
            for (; r + 3 < j; r += 4) {
              a0 += wv[r] * (A)G[(size_t)r * LG + cc];
              a1 += wv[r + 1] * (A)G[(size_t)(r + 1) * LG + cc];
              a2 += wv[r + 2] * (A)G[(size_t)(r + 2) * LG + cc];
              a3 += wv[r + 3] * (A)G[(size_t)(r + 3) * LG + cc];
            }
            for (; r < j; ++r) a0 += wv[r] * (A)G[(size_t)r * LG + cc];
            zv[cc] = ((a0 + a1) + (a2 + a3)) * sc;
          }
        }
        __syncthreads();
        const int j1 = j + 1;
        if constexpr (GS) {
          // (j+1) x (j+1) update: rows from ht / 16, columns from ht % 16 (no division)
          for (int r = ht >> 4; r < j1; r += 8) {
            const A yr = (r < j) ? yv[r] : (A)0;
            for (int cc = ht & 15; cc < j1; cc += 16) {
              A v;
              if (r < j && cc < j) v = (A)G[(size_t)r * LG + cc] + yr * zv[cc];
              else if (r < j) v = -yr * sc;
              else if (cc < j) v = -zv[cc];
              else v = sc;
              G[(size_t)r * LG + cc] = (T)v;
            }
          }
        } else {
          // global memory: items of (column, chunk of 8 rows), consecutive
          // items on consecutive columns (a warp reads a row segment
          // coalesced), spread evenly over the threads
          const int nrc = (j1 + 7) >> 3;
          for (int e = ht; e < j1 * nrc; e += 128) {
            const int cc = e % j1, rb = (e / j1) * 8, re = min(j1, rb + 8);
            const bool old_col = cc < j;
            const A zc = old_col ? zv[cc] : (A)0;
            A g8[8];   // the chunk's old values, loaded before any store
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int r = rb + u;
              g8[u] = (r < re && r < j && old_col) ? (A)G[(size_t)r * LG + cc] : (A)0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int r = rb + u;
              if (r >= re) break;
              A v;
              if (r < j) v = old_col ? g8[u] + yv[r] * zc : -yv[r] * sc;
              else v = old_col ? -zc : sc;
              G[(size_t)r * LG + cc] = (T)v;
            }
          }
        }
        if (ht == 0) {
          lam[j] = lamn_s[half];
          ilam[j] = iem1_s[spin][dk];
        }
      } else if (!to_start) {
        // diagonal change delta of Gamma_qq: Sherman-Morrison on Gamma^{-1}
        for (int r = ht; r < j; r += 128) {
          sv[r] = (A)G[(size_t)r * LG + q];
          wv[r] = (A)G[(size_t)q * LG + r];
        }
        __syncthreads();
        for (int r = ht >> 4; r < j; r += 8)
          for (int cc = ht & 15; cc < j; cc += 16)
            G[(size_t)r * LG + cc] = (T)((A)G[(size_t)r * LG + cc] - sc * sv[r] * wv[cc]);
        if (ht == 0) {
          lam[q] = lamn_s[half];
          ilam[q] = iem1_s[spin][dk];
        }
      } else {
        // back to the block-start spin: Schur complement removes q from P,
        // then the last entry of P moves into position q
        for (int r = ht; r < j; r += 128) {
          sv[r] = (A)G[(size_t)r * LG + q];
          wv[r] = (A)G[(size_t)q * LG + r];
        }
        __syncthreads();
        for (int r = ht >> 4; r < j; r += 8)
          for (int cc = ht & 15; cc < j; cc += 16)
            G[(size_t)r * LG + cc] = (T)((A)G[(size_t)r * LG + cc] - sv[r] * wv[cc] * sc);
        __syncthreads();
        const int last = j - 1;
        if (q != last) {
          for (int e = ht; e < last; e += 128) {
            if (e == q) continue;
            G[(size_t)q * LG + e] = G[(size_t)last * LG + e];
            G[(size_t)e * LG + q] = G[(size_t)e * LG + last];
          }
          if (ht == 0) {
            G[(size_t)q * LG + q] = G[(size_t)last * LG + last];
            lam[q] = lam[last];
            ilam[q] = ilam[last];
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (q < 0) {
          P_s[j] = p;
          pmap[p] = (short)j;
          jP = j + 1;
        } else if (to_start) {
          const int last = j - 1;
          if (q != last) {
            P_s[q] = P_s[last];
            pmap[P_s[q]] = (short)q;
          }
          pmap[p] = -1;
          jP = last;
        }
        s_cur[p] = (int8_t)s_new;
        if (s_new == 0) alive[p >> 5] &= ~(1u << (p & 31));
        else alive[p >> 5] |= (1u << (p & 31));
        if (move == MV_INSERT) n_cur = nc + 1;
        else if (move == MV_REMOVE) n_cur = nc - 1;
      }
    }
    __syncthreads();
  }
  // write back Gamma^{-1}, lambda, P
  const int jf = jP;
  if (gamma_in_smem) {
    T* dst = LU ? c.Glu[spin] : c.Ginv[spin];
    for (int e = ht; e < jf * jf; e += 128) {
      const int r = e / jf, cc = e % jf;
      dst[(size_t)r * LG + cc] = G[(size_t)r * LG + cc];
    }
  }
  for (int r = ht; r < jf; r += 128) c.lam[spin][r] = lam[r];
  for (int r = tid; r < jf; r += 256) c.P[r] = P_s[r];
  if (tid == 0) {
    d.k_acc = jf;
    d.sign = sign_s;
    for (int q = 0; q < 3; ++q) {
      d.proposals[q] += cnt_prop[q];
      d.accepted[q] += cnt_acc[q];
    }
    d.numeric_rejects += numeric;
    d.near_ties += ties;
    d.work_gamma += 2.0 * (double)flops2;
    if (c.trace_cap > 0) d.trace_written += consumed;
  }
}

// -------------------------------------------------------------- flush
// Survivor list S (slots with s != 0 after the block, in slot order) and the
// compacted configuration in the other buffer (Sec. IV C: s=0 rows and
// columns are deleted).

// Gamma^{-1} in global memory (large k_max, large batches): registers held
// to what lets several CTAs share an SM.
template <typename T, bool LU>
__global__ void __launch_bounds__(256) k_proposals(Chain<T>* chains) {
  proposals_body<T, false, LU>(chains);
}

// Gamma^{-1} in shared memory, whose size already limits the CTAs per SM:
// registers unrationed (4-6 % faster per block than at 64 registers).
template <typename T, bool LU>
__global__ void __launch_bounds__(256, 1) k_proposals_smem(Chain<T>* chains) {
  proposals_body<T, true, LU>(chains);
}

// LU form: Gamma^{-1} = U^{-1} L^{-1} from the block's factors, for the flush
// (which uses Gamma^{-1} in either form).  One thread per column c: a = L^{-1}
// e_c by forward substitution (a_r = 0 above c), then b = U^{-1} a by backward
// substitution, in shared memory [row][lane]; 32 columns per CTA, grid
// (column blocks, spin, chain).  2 j^3 / 3 multiply-adds per spin, against the
// flush's n j^2.
template <typename T>
__global__ void __launch_bounds__(32) k_lu_inverse(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.z];
  const Dyn& d = *c.dyn;
  const int j = d.k_acc, c0 = blockIdx.x * 32;
  if (d.status || c0 >= j) return;
  extern __shared__ __align__(16) unsigned char lu_raw[];
  T* a = reinterpret_cast<T*>(lu_raw);
  const int spin = blockIdx.y, lane = threadIdx.x, col = c0 + lane, LG = c.k_max + 1;
  const T* F = c.Glu[spin];
  for (int r = 0; r < c0; ++r) a[r * 32 + lane] = (T)0;
  for (int r = c0; r < j; ++r) {
    const T* Lr = F + (size_t)r * LG;
    T acc = (r == col) ? (T)1 : (T)0;
    for (int l = c0; l < r; ++l) acc -= Lr[l] * a[l * 32 + lane];
    a[r * 32 + lane] = acc;
  }
  T* Gi = c.Ginv[spin];
  for (int r = j - 1; r >= 0; --r) {
    const T* Ur = F + (size_t)r * LG;
    T acc = a[r * 32 + lane];
    for (int l = r + 1; l < j; ++l) acc -= Ur[l] * a[l * 32 + lane];
    acc = acc / Ur[r];
    a[r * 32 + lane] = acc;
    if (col < j) Gi[(size_t)r * LG + col] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_survivors(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.x];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const int m = d.m, buf = d.buf, ob = 1 - buf;
  __shared__ int warp_tot[32];
  __shared__ int base_s;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i0 = 0; i0 < m; i0 += 1024) {
    const int i = i0 + threadIdx.x;
    const int keep = (i < m) && c.s[buf][i] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_tot[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x < 32) {
      int v = warp_tot[threadIdx.x];
      int incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (threadIdx.x >= o) incl += u;
      }
      warp_tot[threadIdx.x] = incl - v;
    }
    __syncthreads();
    if (keep) {
      const int a = base_s + warp_tot[w] + __popc(bal & ((1u << lane) - 1u));
      c.S[a] = i;
      c.tau[ob][a] = c.tau[buf][i];
      c.site[ob][a] = c.site[buf][i];
      c.s[ob][a] = c.s[buf][i];
      c.birth[ob][a] = c.birth[buf][i];
    }
    __syncthreads();
    if (threadIdx.x == 1023) base_s += warp_tot[31] + __popc(bal);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d.n_new = base_s;
    // nothing accepted and the survivors are the slots [0, n_new) in order:
    // N'_SS is the leading block of N_ext, which holds N unchanged in place
    d.flush_noop = (d.k_acc == 0 && (base_s == 0 || c.S[base_s - 1] == base_s - 1)) ? 1 : 0;
  }
}

// Y = (G^0 - 1)_{S,P} Gamma^{-1}, so that N'_{SS} = N_{SS} - Y N_{P,S}
// (Eq. Nshermanmorrison with D^{-1} folded: rows p in P of
// D^{-1}(N - G Gamma^{-1} N_P) equal those of N - (G - 1) Gamma^{-1} N_P).
// A CTA takes 16 surviving rows: it stages (G^0 - 1)_{rows,P} in shared
// memory, then multiplies by Gamma^{-1} read from global memory.
// With SPLIT (mixed form, tensor-core flush) Y is written instead as K-major
// tf32 hi/lo rows Yh/Yl[a * kp + r], zero for k_acc <= r < kp.
constexpr int kYRows = 16;

__device__ __forceinline__ void split_tf32_y(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

template <typename T, bool SPLIT>
__device__ __forceinline__ int flush_y_items(const Dyn& d) {
  if (d.status || d.flush_noop || (!SPLIT && d.k_acc == 0)) return 0;
  return 2 * ((d.n_new + kYRows - 1) / kYRows);
}

template <typename T, bool SPLIT>
__global__ void __launch_bounds__(256) k_flush_y(Chain<T>* chains, int n_chains) {
  using A = T;
  __shared__ int off[kMaxChains + 1];
  __shared__ A gh[kYRows * kMaxK];
  __shared__ int Ps[kMaxK];
  __shared__ int Si[kYRows];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x)
    off[ci] = flush_y_items<T, SPLIT>(*chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int ci = find_chain(off, n_chains, w);
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    const int l = w - off[ci];
    const int groups = (d.n_new + kYRows - 1) / kYRows;
    const int spin = l / groups;
    const int kacc = d.k_acc, nn = d.n_new, KM = c.k_max;
    const int a0 = (l % groups) * kYRows;
    __syncthreads();
    for (int e = threadIdx.x; e < kacc; e += blockDim.x) Ps[e] = c.P[e];
    for (int e = threadIdx.x; e < kYRows; e += blockDim.x) Si[e] = (a0 + e < nn) ? c.S[a0 + e] : -1;
    __syncthreads();
    const T* Nb = c.N[d.buf][spin];
    const T* Gc = c.Gcol[spin];
    const int n_old = d.n;
    for (int e = threadIdx.x; e < kYRows * kacc; e += blockDim.x) {
      const int aa = e % kYRows, q = e / kYRows;
      const int i = Si[aa];
      A v = (A)0;
      if (i >= 0) {
        const int pq = Ps[q];
        v = g_int<A>(c, Nb, Gc, n_old, spin, i, pq) - (i == pq ? (A)1 : (A)0);
      }
      gh[q * kYRows + aa] = v;
    }
    __syncthreads();
    const T* Gi = c.Ginv[spin];
    const int LGi = KM + 1;
    if constexpr (!SPLIT) {
      // float64: one (row, column) per thread (the FP64 pipe bounds it)
      for (int e = threadIdx.x; e < kYRows * kacc; e += blockDim.x) {
        const int aa = e % kYRows, r = e / kYRows;
        if (Si[aa] < 0) continue;
        A acc = (A)0;
        for (int q = 0; q < kacc; ++q) acc += gh[q * kYRows + aa] * (A)Gi[(size_t)q * LGi + r];
        c.Y[spin][(size_t)r * c.ld + a0 + aa] = (T)acc;
      }
      continue;
    }
    // float32: a thread per column r of Y; the 16 rows' sums share each
    // Gamma^{-1} load (a column of Gamma^{-1}, read coalesced across the
    // threads), sums in q order
    const int ncol = SPLIT ? c.kp : kacc;
    for (int r = threadIdx.x; r < ncol; r += blockDim.x) {
      A acc[kYRows];
#pragma unroll
      for (int aa = 0; aa < kYRows; ++aa) acc[aa] = (A)0;
      if (r < kacc) {
        for (int q = 0; q < kacc; ++q) {
          const A g = (A)Gi[(size_t)q * LGi + r];
          const A* gq = gh + q * kYRows;
#pragma unroll
          for (int aa = 0; aa < kYRows; ++aa) acc[aa] += gq[aa] * g;
        }
      }
      if constexpr (!SPLIT) {
#pragma unroll
        for (int aa = 0; aa < kYRows; ++aa)
          if (Si[aa] >= 0) c.Y[spin][(size_t)r * c.ld + a0 + aa] = (T)acc[aa];
      } else {
        const int KP = c.kp;
#pragma unroll
        for (int aa = 0; aa < kYRows; ++aa) {
          if (Si[aa] < 0) continue;
          float hi = 0.f, lo = 0.f;
          if (r < kacc) split_tf32_y((float)acc[aa], hi, lo);
          c.Yh[spin][(size_t)(a0 + aa) * KP + r] = hi;
          c.Yl[spin][(size_t)(a0 + aa) * KP + r] = lo;
        }
      }
    }
  }
}

// End of block: swap buffers, advance the counter.
template <typename T>
__global__ void k_finish_block(Chain<T>* chains, int n_chains) {
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci >= n_chains) return;
  const Chain<T>& c = chains[ci];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const double n = d.n, ki = d.k_ins, ka = d.k_acc, nn = d.n_new;
  d.work_prep += 2.0 * (2.0 * ki * n * n + 2.0 * n * n * ki + 2.0 * ki * ki * n);
  d.n = d.n_new;
  if (!d.flush_noop) {
    d.work_flush += 2.0 * (2.0 * nn * nn * ka + 2.0 * nn * ka * ka);
    d.bytes_flush += 2.0 * (2.0 * nn * nn + 2.0 * nn * ka) * sizeof(T);
    d.buf = 1 - d.buf;
  }
  d.t += (d.tie_pending == 1) ? d.tie_jj : c.k_max;
  d.sweeps += 1;
}


__global__ void k_philox_test(uint64_t seed, uint32_t chain, int64_t t0, int count, int purpose,
                              double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double u0, u1;
  philox_pair(seed, chain, t0 + i, (uint32_t)purpose, u0, u1);
  out[2 * i] = u0;
  out[2 * i + 1] = u1;
}

void launch_philox_test(uint64_t seed, uint32_t chain, int64_t t0, int count, int purpose,
                        double* out, cudaStream_t st) {
  k_philox_test<<<(count + 255) / 256, 256, 0, st>>>(seed, chain, t0, count, purpose, out);
}

// ----------------------------------------------------------- launchers
template <typename T>
int lu_inverse_smem(const LaunchShape& ls) {
  return (int)(sizeof(T) * 32 * (size_t)ls.max_k);
}

template <typename T>
void launch_block(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st, PhaseTimer* pt,
                  const TcMaps* maps, const BlockFork* fork) {
  const int nch = ls.n_chains;
  pt->begin(0, st);
  k_plan<T><<<nch, 256, 0, st>>>(dchains);
  k_gather<T><<<dim3(ls.gather_slices, 2, nch), 256, 0, st>>>(dchains);
  pt->end(0, st, 2);
  pt->begin(1, st);
  bool prep_tc = false;
  if constexpr (std::is_same<T, float>::value) prep_tc = ls.prep_tc != 0;
  if (prep_tc) {
    if constexpr (std::is_same<T, float>::value) launch_prep_tc(dchains, maps, ls, st);
    pt->end(1, st, 1 + launch_gemm<T>(dchains, ls, PH_GCOL_NEW, st));
  } else {
    int nk = launch_gemm<T>(dchains, ls, PH_RTILDE, st);
    nk += launch_gemm<T>(dchains, ls, PH_GCOL_OLD, st);
    nk += launch_gemm<T>(dchains, ls, PH_GCOL_NEW, st);
    pt->end(1, st, nk);
  }
  if (fork) {
    // side work from here on (the proposals change the spins, the flush writes
    // the other buffer of N and of the configuration)
    cudaEventRecord(fork->ev_fork, st);
    cudaStreamWaitEvent(fork->side, fork->ev_fork, 0);
    fork->fn(fork->arg, fork->side);
    cudaEventRecord(fork->ev_join, fork->side);
  }
  pt->begin(2, st);
  if (ls.gamma_lu) {
    if (ls.gamma_in_smem) k_proposals_smem<T, true><<<nch, 256, ls.prop_smem, st>>>(dchains);
    else k_proposals<T, true><<<nch, 256, ls.prop_smem, st>>>(dchains);
  } else {
    if (ls.gamma_in_smem) k_proposals_smem<T, false><<<nch, 256, ls.prop_smem, st>>>(dchains);
    else k_proposals<T, false><<<nch, 256, ls.prop_smem, st>>>(dchains);
  }
  if (ls.gamma_lu)
    k_lu_inverse<T><<<dim3((ls.max_k + 31) / 32, 2, nch), 32, lu_inverse_smem<T>(ls), st>>>(dchains);
  pt->end(2, st, ls.gamma_lu ? 2 : 1);
  bool tc = false;
  if constexpr (std::is_same<T, float>::value) tc = ls.use_tc != 0;
  pt->begin(4, st);
  k_survivors<T><<<nch, 1024, 0, st>>>(dchains);
  if (tc) {
    if constexpr (std::is_same<T, float>::value)
      k_flush_y<float, true><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
  } else {
    k_flush_y<T, false><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
  }
  pt->end(4, st, 2);
  pt->begin(3, st);
  if (tc) {
    if constexpr (std::is_same<T, float>::value) launch_flush_tc(dchains, maps, ls, st);
    pt->end(3, st, 2);
    if (ls.prep_tc) {   // N'^T for the next block's prep, timed as flush support
      pt->begin(4, st);
      if constexpr (std::is_same<T, float>::value) launch_transpose_n(dchains, ls, st);
      pt->end(4, st, 1);
    }
  } else {
    pt->end(3, st, launch_gemm<T>(dchains, ls, PH_FLUSH, st));
  }
  if (fork) cudaStreamWaitEvent(st, fork->ev_join, 0);   // the side work ends before the block does
  k_finish_block<T><<<(nch + 127) / 128, 128, 0, st>>>(dchains, nch);
  pt->kernels[4] += 1;
}

template <typename T>
cudaError_t configure_block_kernels(const LaunchShape& ls) {
  const cudaFuncAttribute dyn = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_proposals_smem<T, false>, dyn, ls.prop_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_proposals<T, false>, dyn, ls.prop_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_proposals_smem<T, true>, dyn, ls.prop_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_proposals<T, true>, dyn, ls.prop_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lu_inverse<T>, dyn, lu_inverse_smem<T>(ls));
  return e;
}

template int launch_gemm<double>(Chain<double>*, const LaunchShape&, int, cudaStream_t);
template int launch_gemm<float>(Chain<float>*, const LaunchShape&, int, cudaStream_t);
template void launch_block<double>(Chain<double>*, const LaunchShape&, cudaStream_t, PhaseTimer*,
                                   const TcMaps*, const BlockFork*);
template void launch_block<float>(Chain<float>*, const LaunchShape&, cudaStream_t, PhaseTimer*,
                                  const TcMaps*, const BlockFork*);
template cudaError_t configure_block_kernels<double>(const LaunchShape&);
template cudaError_t configure_block_kernels<float>(const LaunchShape&);

}  // namespace ctaux
