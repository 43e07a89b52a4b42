// From-scratch FP64 recomputation of N for every chain (device bodies, shared
// by the refresh kernel and the near-tie fallback of the refinement kernel):
// build
// N^{-1} = e^V - G0 (e^V - 1) (Eq. Nmatrix) from the configuration, invert
// by blocked Gauss-Jordan with partial pivoting, report the drift of the
// running N and replace it.  One cooperative launch: all chains and spins
// advance in lockstep, separated by grid-wide barriers (no spin waits); the
// work of each stage is spread over the whole grid across chains.
//
// Unblocked column step c (pivot row pr) maps X to
//   X[pr][j] / X[pr][c] (j != c), 1 / X[pr][c] at (pr, c),
//   -X[i][c] / X[pr][c] at (i, c), X[i][j] - X[i][c] X[pr][j] / X[pr][c] elsewhere.
// Blocked: for a panel C of 32 columns with pivot rows R, the column steps are
// applied to the panel alone (a copy, ping-pong), giving P' = X'[:, C]; every
// other column then follows in one rank-32 product
//   X'[:, J] = Z[:, J] + P' X[R, J],  Z = X with the rows R set to zero.
// After all panels, N[c][perm[j]] = X[perm[c]][j] and
// log|det N^{-1}| = sum_c log|pivot_c|.
// Pivots: the largest |value| over rows not yet pivoted, folded while the
// previous step writes that column: atomicMax of a 64-bit key (the upper half
// of the float64 magnitude, ties to the lower row) per (chain, spin, column).
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "ctaux_df64.cuh"
#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"

namespace ctaux {

namespace cg = cooperative_groups;

// Pivot key: the upper 32 bits of the float64 pattern of a magnitude (sign 0,
// the whole exponent, 20 significand bits) order like the magnitude for every
// non-negative double, so a normal entry, however small, beats an exact zero;
// ties within 2^-20 go to the lower row.
__device__ __forceinline__ unsigned long long pivot_key_mag(double a, int row) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  return (bits & 0xffffffff00000000ull) | (unsigned long long)(0xffffffffu - (unsigned)row);
}

// Element arithmetic of the elimination: float64, or double-float (df64, the
// mixed form's option) on the float32 pipe.  Both are 8 bytes, so the work
// area layout is the same.
__device__ __forceinline__ double el_from(double x, double*) { return x; }
__device__ __forceinline__ df64 el_from(double x, df64*) { return df_from(x); }
__device__ __forceinline__ double el_to(double a) { return a; }
__device__ __forceinline__ double el_to(df64 a) { return df_to(a); }
__device__ __forceinline__ double el_mul(double a, double b) { return a * b; }
__device__ __forceinline__ df64 el_mul(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ double el_sub(double a, double b) { return a - b; }
__device__ __forceinline__ df64 el_sub(df64 a, df64 b) { return df_sub(a, b); }
__device__ __forceinline__ double el_neg(double a) { return -a; }
__device__ __forceinline__ df64 el_neg(df64 a) { return df_neg(a); }
__device__ __forceinline__ double el_recip(double a) { return 1.0 / a; }
__device__ __forceinline__ df64 el_recip(df64 a) { return df_recip(a); }
__device__ __forceinline__ unsigned long long pivot_key(double v, int row) {
  return pivot_key_mag(fabs(v), row);
}
__device__ __forceinline__ unsigned long long pivot_key(df64 v, int row) {
  return pivot_key_mag(fabs((double)v.hi), row);
}
template <typename E>
__device__ __forceinline__ E el_zero() {
  return el_from(0.0, (E*)nullptr);
}

// acc + sum_k x_k y_k (the rank-32 trailing update)
struct ElDot64 {
  double a;
  __device__ __forceinline__ explicit ElDot64(double init) : a(init) {}
  __device__ __forceinline__ void add(double x, double y) { a = fma(x, y, a); }
  __device__ __forceinline__ double value() const { return a; }
};
struct ElDotDf {
  df64 init;
  DfDot dot;
  __device__ __forceinline__ explicit ElDotDf(df64 i) : init(i) {}
  __device__ __forceinline__ void add(df64 x, df64 y) { dot.add(x, y); }
  __device__ __forceinline__ df64 value() const { return df_add(init, dot.value()); }
};
__device__ __forceinline__ ElDot64 el_dot(double init) { return ElDot64(init); }
__device__ __forceinline__ ElDotDf el_dot(df64 init) { return ElDotDf(init); }

// Trailing-update tile edge: 32 for float64 (the FP64 pipe bounds it), 64 for
// double-float, where each thread keeps a 4 x 4 block of compensated sums so
// that the float32 pipe, not shared-memory loads or latency, bounds it.
template <typename E>
__host__ __device__ constexpr int trail_tile() {
  return std::is_same<E, df64>::value ? 64 : 32;
}

// Compensated sum started from a double-float value: s carries the high
// part and the error-free running sum of the high products, c the low part,
// the rounding errors and the cross terms (Dot2 with the initial value split
// between the two).
struct DfAcc {
  float s, c;
  __device__ __forceinline__ void init(df64 x) {
    s = x.hi;
    c = x.lo;
  }
  __device__ __forceinline__ void add(df64 x, df64 y) {
    float pe, se;
    const float p = two_prod(x.hi, y.hi, pe);
    const float cross = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, pe));
    s = two_sum(s, p, se);
    c = __fadd_rn(c, __fadd_rn(se, cross));
  }
  __device__ __forceinline__ df64 value() const {
    df64 r;
    r.hi = two_sum(s, c, r.lo);
    return r;
  }
};
__device__ __forceinline__ int key_row(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

constexpr int kPB = 32;  // panel width

// Dynamic shared memory of the refresh kernel for element type E.
template <typename E>
__host__ __device__ constexpr int refresh_dyn_smem() {
  return trail_tile<E>() == 32 ? 0
                              : 2 * (int)sizeof(E) * (trail_tile<E>() * (kPB + 1) + kPB * (trail_tile<E>() + 1));
}

// per-spin work area: X (ld x ld), two panel buffers (ld x kPB), pivot rows (ld x kPB)
__host__ __device__ inline size_t refresh_work_per_spin(int ld) {
  return (size_t)ld * ld + (size_t)3 * kPB * ld;
}

// Size of the refresh of chain ci (0 when it does not take part).
template <typename T>
__device__ __forceinline__ int refresh_order(const Chain<T>& c, int ci, int c_lo, int c_hi, int filter) {
  if (ci < c_lo || ci >= c_hi) return 0;
  const Dyn& d = *c.dyn;
  if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) return 0;
  return d.n;
}

// Work of every stage is spread over the grid across all chains: "row units"
// (chain, spin, row or column index; 2m per chain) go to threads or CTAs by a
// prefix sum over chains, "tile units" (chain, spin, 32 x 32 tile) to CTAs.
struct RowUnit {
  int ci, spin, i, m;
};

__device__ __forceinline__ RowUnit row_unit(const int* offr, int n_chains, int u) {
  RowUnit r;
  r.ci = find_chain(offr, n_chains, u);
  r.m = (offr[r.ci + 1] - offr[r.ci]) >> 1;
  const int l = u - offr[r.ci];
  r.spin = l / r.m;
  r.i = l - r.spin * r.m;
  return r;
}

// Trailing update of one panel in double-float, 64 x 64 tiles: each CTA walks
// its tiles (grid stride over the tile units), with the next tile's panel and
// pivot-row values copied into the other shared-memory buffer by cp.async
// while the current tile is computed, and the current tile's X values loaded
// into registers before its products.  Thread (tr, tc) of 16 x 16 owns rows
// tr + 16a and columns tc + 16b (a, b = 0..3): 16 compensated sums, each
// started at zero and added to X at the end.
struct DfTile {
  int ci, spin, m, i0, j0;
};

template <typename T>
__device__ __forceinline__ bool df_tile(Chain<T>* chains, int n_chains, const int* offr,
                                        const int* offt, int c0, int u, DfTile& t) {
  t.ci = find_chain(offt, n_chains, u);
  t.m = (offr[t.ci + 1] - offr[t.ci]) >> 1;
  if (c0 >= t.m) return false;
  const int tb = (t.m + 63) / 64, l = u - offt[t.ci];
  t.spin = l / (tb * tb);
  const int tile = l - t.spin * tb * tb;
  t.i0 = (tile % tb) * 64;
  t.j0 = (tile / tb) * 64;
  return true;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(ok ? 8 : 0)
               : "memory");
}

template <typename T>
__device__ void trail_update_df64(Chain<T>* chains, int n_chains, const int* offr, const int* offt,
                                  int tot_t, int c0, unsigned char* dyn) {
  constexpr int TB = 64;
  using Prow = df64[kPB + 1];
  using Rrow = df64[TB + 1];
  const size_t buf_bytes = sizeof(df64) * (TB * (kPB + 1) + kPB * (TB + 1));
  auto Pbuf = [&](int b) { return reinterpret_cast<Prow*>(dyn + b * buf_bytes); };
  auto Rbuf = [&](int b) {
    return reinterpret_cast<Rrow*>(dyn + b * buf_bytes + sizeof(df64) * TB * (kPB + 1));
  };
  // cp.async of tile t's panel rows and pivot-row columns into buffer b
  auto prefetch = [&](const DfTile& t, int b) {
    const Chain<T>& c = chains[t.ci];
    const int ld = c.ld, bw = min(kPB, t.m - c0);
    const df64* X = reinterpret_cast<const df64*>(c.work + (size_t)t.spin * refresh_work_per_spin(ld));
    const df64* Pa = X + (size_t)ld * ld;
    const df64* Pf = (bw & 1) ? Pa + (size_t)kPB * ld : Pa;  // panel after bw steps
    const df64* Rr = Pa + (size_t)2 * kPB * ld;
    Prow* Ps = Pbuf(b);
    Rrow* Rs = Rbuf(b);
    for (int e = threadIdx.x; e < TB * kPB; e += blockDim.x) {
      const int r = e % TB, k = e / TB;
      const bool okp = t.i0 + r < t.m && k < bw;
      cp_async8(&Ps[r][k], okp ? Pf + (size_t)k * ld + t.i0 + r : Pf, okp);
      const int kk = e % kPB, jj = e / kPB;   // Rr rows are contiguous in k
      const bool okr = t.j0 + jj < t.m;
      cp_async8(&Rs[kk][jj], okr ? Rr + (size_t)(t.j0 + jj) * kPB + kk : Rr, okr);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  const int stride = gridDim.x;
  int u = blockIdx.x;
  DfTile cur;
  while (u < tot_t && !df_tile(chains, n_chains, offr, offt, c0, u, cur)) u += stride;
  if (u >= tot_t) return;
  prefetch(cur, 0);
  const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
  int b = 0;
  while (u < tot_t) {
    // the next tile of this CTA
    int un = u + stride;
    DfTile nxt;
    while (un < tot_t && !df_tile(chains, n_chains, offr, offt, c0, un, nxt)) un += stride;

    const Chain<T>& c = chains[cur.ci];
    const int ld = c.ld, m = cur.m, spin = cur.spin, bw = min(kPB, m - c0), cn = c0 + bw;
    df64* X = reinterpret_cast<df64*>(c.work + (size_t)spin * refresh_work_per_spin(ld));
    unsigned long long* keys = c.pkeys + (size_t)spin * ld;
    const int8_t* used = c.used + spin * ld;
    const int* pcol = c.pcol + spin * ld;
    // X values of this tile (zero for pivot rows, panel columns and padding)
    df64 xin[4][4];
    bool row_ok[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = cur.i0 + tr + 16 * a;
      row_ok[a] = i < m;
      const int pci = row_ok[a] ? pcol[i] : -1;
      const bool in_R = pci >= c0 && pci < cn;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = cur.j0 + tc + 16 * q;
        const bool keep = row_ok[a] && !in_R && j < m && !(j >= c0 && j < cn);
        xin[a][q] = keep ? X[(size_t)j * ld + i] : df_zero();
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // this tile's buffer is complete; the other one is free
    if (un < tot_t) prefetch(nxt, b ^ 1);
    const Prow* Ps = Pbuf(b);
    const Rrow* Rs = Rbuf(b);
    DfAcc acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][q].init(df_zero());
#pragma unroll 1
    for (int k = 0; k < kPB; ++k) {
      df64 pv[4], qv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) pv[a] = Ps[tr + 16 * a][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) qv[q] = Rs[k][tc + 16 * q];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q].add(pv[a], qv[q]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!row_ok[a]) continue;
      const int r = tr + 16 * a, i = cur.i0 + r;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = cur.j0 + tc + 16 * q;
        if (j >= m) continue;
        const df64 v = (j >= c0 && j < cn) ? Ps[r][j - c0] : df_add(xin[a][q], acc[a][q].value());
        X[(size_t)j * ld + i] = v;
        if (j == cn && !used[i]) atomicMax(keys + cn, pivot_key(v, i));
      }
    }
    cur = nxt;
    u = un;
    b ^= 1;
  }
}

template <typename T, typename E>
__device__ void refresh_body(Chain<T>* chains, int n_chains, int only_chain, int filter) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  const int c_lo = only_chain >= 0 ? only_chain : 0;
  const int c_hi = only_chain >= 0 ? only_chain + 1 : n_chains;
  __shared__ int offr[kMaxChains + 1];
  __shared__ int offt[kMaxChains + 1];
  __shared__ int max_m_s;
  constexpr int TB = trail_tile<E>();
  // panel and pivot-row tiles: static for 32 x 32; the 64 x 64 double-float
  // tiles are double-buffered in dynamic shared memory (refresh_dyn_smem bytes)
  __shared__ E Ps[TB == 32 ? 32 : 1][kPB + 1];
  __shared__ E Rs[TB == 32 ? kPB : 1][33];
  extern __shared__ __align__(16) unsigned char refresh_dyn[];
  __shared__ double red[3][8];

  if (threadIdx.x == 0) max_m_s = 0;
  __syncthreads();
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
    const int m = refresh_order(chains[ci], ci, c_lo, c_hi, filter);
    const int tb = (m + TB - 1) / TB;
    offr[ci] = 2 * m;
    offt[ci] = 2 * tb * tb;
    atomicMax(&max_m_s, m);
  }
  __syncthreads();
  block_exclusive_scan(offr, n_chains);
  block_exclusive_scan(offt, n_chains);
  const int tot_r = offr[n_chains], tot_t = offt[n_chains], max_m = max_m_s;
  if (tot_r == 0) return;  // nothing to refresh (same decision in every CTA, before any barrier)

  // ---- stage 1: N^{-1} of the current configuration into X (one column per
  // CTA and unit); pivot key of column 0
  for (int u = blockIdx.x; u < tot_r; u += gridDim.x) {
    const RowUnit ru = row_unit(offr, n_chains, u);
    const Chain<T>& c = chains[ru.ci];
    const int m = ru.m, spin = ru.spin, j = ru.i, buf = c.dyn->buf, ld = c.ld;
    E* X = reinterpret_cast<E*>(c.work + (size_t)spin * refresh_work_per_spin(ld));
    unsigned long long* keys = c.pkeys + (size_t)spin * ld;
    const double evj = c.ev[spin][c.s[buf][j] + 2];
    const double tj = c.tau[buf][j];
    const int sj = c.site[buf][j];
    if (j == 0 && threadIdx.x == 0) c.work_logdet[spin] = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double v = -g0_eval(c, spin, c.tau[buf][i], c.site[buf][i], tj, sj) * (evj - 1.0);
      if (i == j) v += evj;
      const E ve = el_from(v, (E*)nullptr);
      X[(size_t)j * ld + i] = ve;
      if (j == 0) atomicMax(keys, pivot_key(ve, i));
    }
  }
  grid.sync();

  // ---- stage 2: panels
  for (int c0 = 0; c0 < max_m; c0 += kPB) {
    // A0: copy the panel columns ((row unit, panel column) pairs)
    for (int u = gtid; u < tot_r * kPB; u += gthreads) {
      const int k = u / tot_r;
      const RowUnit ru = row_unit(offr, n_chains, u - k * tot_r);
      if (c0 + k >= ru.m) continue;
      const Chain<T>& c = chains[ru.ci];
      const int ld = c.ld;
      E* X = reinterpret_cast<E*>(c.work + (size_t)ru.spin * refresh_work_per_spin(ld));
      E* Pa = X + (size_t)ld * ld;
      Pa[(size_t)k * ld + ru.i] = X[(size_t)(c0 + k) * ld + ru.i];
    }
    grid.sync();
    // A1: the column steps, on the panel only.  Work unit = (row unit, group
    // of W = 32 / G panel columns), G the largest power of two <= 32 with
    // rows x G <= threads: few rows spread their columns over more threads,
    // many rows take whole panel rows.  A unit's panel values are loaded in
    // batches of 4 before they are transformed; the next column's pivot key
    // is reduced per warp before its atomic.
    int G = 1;
    while (G < kPB && tot_r * (2 * G) <= gthreads) G *= 2;
    const int W = kPB / G;
    for (int k = 0; k < kPB; ++k) {
      for (int ub = gtid - (int)(threadIdx.x & 31); ub < tot_r * G; ub += gthreads) {
        const int u = ub + (int)(threadIdx.x & 31);
        unsigned long long* kaddr = nullptr;
        unsigned long long cand = 0ull;
        if (u < tot_r * G) {
          const int grp = u / tot_r;
          const RowUnit ru = row_unit(offr, n_chains, u - grp * tot_r);
          if (c0 + k < ru.m) {
            const Chain<T>& c = chains[ru.ci];
            const int ld = c.ld, col = c0 + k, i = ru.i, spin = ru.spin;
            const int nkk = min(kPB, ru.m - c0);
            E* X = reinterpret_cast<E*>(c.work + (size_t)spin * refresh_work_per_spin(ld));
            E* Pa = X + (size_t)ld * ld;
            E* Pb = Pa + (size_t)kPB * ld;
            const E* src = (k & 1) ? Pb : Pa;
            E* dst = (k & 1) ? Pa : Pb;
            unsigned long long* keys = c.pkeys + (size_t)spin * ld;
            int8_t* used = c.used + spin * ld;
            const int pr = key_row(keys[col]);
            const E piv = src[(size_t)k * ld + pr];
            if (i == 0 && grp == 0) {
              const double pd = el_to(piv);
              c.perm[spin * ld + col] = pr;
              used[pr] = 1;  // read below only for rows other than pr
              c.pcol[spin * ld + pr] = col;
              if (!(fabs(pd) > 0.0) || !isfinite(pd)) atomicOr(&c.dyn->status, DS_SINGULAR);
              c.work_logdet[spin] += log(fabs(pd));
            }
            const E ipiv = el_recip(piv);
            const E xic = src[(size_t)k * ld + i];
            E vnext = el_zero<E>();
            for (int kb = grp * W; kb < grp * W + W; kb += 4) {
              E xs[4], xp[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int kk = kb + q;
                const bool in = q < W && kk < nkk;
                xs[q] = in ? src[(size_t)kk * ld + i] : el_zero<E>();
                xp[q] = in ? src[(size_t)kk * ld + pr] : el_zero<E>();
              }
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int kk = kb + q;
                if (q >= W || kk >= nkk) continue;
                E v;
                if (i == pr) v = (kk == k) ? ipiv : el_mul(xp[q], ipiv);
                else if (kk == k) v = el_neg(el_mul(xic, ipiv));
                else v = el_sub(xs[q], el_mul(xic, el_mul(xp[q], ipiv)));
                dst[(size_t)kk * ld + i] = v;
                if (kk == k + 1) vnext = v;
              }
            }
            if (k + 1 < nkk && (k + 1) / W == grp && i != pr && !used[i]) {
              kaddr = keys + col + 1;
              cand = pivot_key(vnext, i);
            }
          }
        }
        // one atomic per warp where every lane with a candidate shares the key
        const unsigned want = __ballot_sync(0xffffffffu, kaddr != nullptr);
        if (want) {
          const int lead = __ffs(want) - 1;
          const unsigned long long* a0 = reinterpret_cast<const unsigned long long*>(
              __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(kaddr), lead));
          if (__all_sync(0xffffffffu, kaddr == nullptr || kaddr == a0)) {
            unsigned long long mx = cand;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
              mx = y > mx ? y : mx;
            }
            if ((int)(threadIdx.x & 31) == lead) atomicMax(kaddr, mx);
          } else if (kaddr) {
            atomicMax(kaddr, cand);
          }
        }
      }
      grid.sync();
    }
    // B0: pivot rows of this panel, outside it, from X before the update:
    // Rr[j][k] = X[R_k][j] ((row unit = column j, k) pairs)
    for (int u = gtid; u < tot_r * kPB; u += gthreads) {
      const int k = u % kPB;
      const RowUnit ru = row_unit(offr, n_chains, u / kPB);
      if (c0 >= ru.m) continue;
      const Chain<T>& c = chains[ru.ci];
      const int ld = c.ld, j = ru.i;
      E* X = reinterpret_cast<E*>(c.work + (size_t)ru.spin * refresh_work_per_spin(ld));
      E* Rr = X + (size_t)ld * ld + (size_t)2 * kPB * ld;
      const int* perm = c.perm + ru.spin * ld;
      Rr[(size_t)j * kPB + k] = (c0 + k < ru.m) ? X[(size_t)j * ld + perm[c0 + k]] : el_zero<E>();
    }
    grid.sync();
    // B1: trailing rank-bw update in TB x TB tiles (tile units), panel written
    // back, pivot key of the next panel's first column
    if constexpr (TB == 64) {
      trail_update_df64<T>(chains, n_chains, offr, offt, tot_t, c0, refresh_dyn);
    } else {
    for (int u = blockIdx.x; u < tot_t; u += gridDim.x) {
      const int ci = find_chain(offt, n_chains, u);
      const int m = (offr[ci + 1] - offr[ci]) >> 1;
      if (c0 >= m) continue;  // uniform over the CTA
      const Chain<T>& c = chains[ci];
      const int tb = (m + TB - 1) / TB, l = u - offt[ci];
      const int spin = l / (tb * tb), tile = l - spin * tb * tb;
      const int ld = c.ld, bw = min(kPB, m - c0), cn = c0 + bw;
      E* X = reinterpret_cast<E*>(c.work + (size_t)spin * refresh_work_per_spin(ld));
      E* Pa = X + (size_t)ld * ld;
      const E* Pf = (bw & 1) ? Pa + (size_t)kPB * ld : Pa;  // panel after bw steps
      const E* Rr = Pa + (size_t)2 * kPB * ld;
      unsigned long long* keys = c.pkeys + (size_t)spin * ld;
      const int8_t* used = c.used + spin * ld;
      const int* pcol = c.pcol + spin * ld;
      const int i0 = (tile % tb) * TB, j0 = (tile / tb) * TB;
      __syncthreads();
      for (int e = threadIdx.x; e < TB * kPB; e += blockDim.x) {
        const int r = e % TB, k = e / TB;
        Ps[r][k] = (i0 + r < m && k < bw) ? Pf[(size_t)k * ld + i0 + r] : el_zero<E>();
        const int kk = e % kPB, jj = e / kPB;   // Rr rows are contiguous in k
        Rs[kk][jj] = (j0 + jj < m) ? Rr[(size_t)(j0 + jj) * kPB + kk] : el_zero<E>();
      }
      __syncthreads();
      {
      // thread (row r, column group g): columns q = g + 8c, c = 0..3, so that
      // each panel value Ps[r][k] is loaded once for four products
      const int r = threadIdx.x % 32, i = i0 + r, g = threadIdx.x / 32;
      static_assert(kPB == 32 && TB == 32, "a 32 x 32 tile per 256 threads");
      if (i < m) {
        const int pci = pcol[i];
        const bool in_R = pci >= c0 && pci < cn;
        decltype(el_dot(el_zero<E>())) acc[4] = {el_dot(el_zero<E>()), el_dot(el_zero<E>()),
                                                 el_dot(el_zero<E>()), el_dot(el_zero<E>())};
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) {
          const int j = j0 + g + 8 * cq;
          if (!in_R && j < m && !(j >= c0 && j < cn)) acc[cq] = el_dot(X[(size_t)j * ld + i]);
        }
#pragma unroll 4
        for (int k = 0; k < kPB; ++k) {
          const E pk = Ps[r][k];
#pragma unroll
          for (int cq = 0; cq < 4; ++cq) acc[cq].add(pk, Rs[k][g + 8 * cq]);
        }
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) {
          const int q = g + 8 * cq, j = j0 + q;
          if (j >= m) continue;
          const E v = (j >= c0 && j < cn) ? Ps[r][j - c0] : acc[cq].value();
          X[(size_t)j * ld + i] = v;
          if (j == cn && !used[i]) atomicMax(keys + cn, pivot_key(v, i));
        }
      }
      }
    }
    }
    grid.sync();
  }

  // ---- stage 3: unscramble, drift against the running N (reduced per CTA
  // and column), replace it; clear the pivot keys and flags for the next refresh
  for (int u = blockIdx.x; u < tot_r; u += gridDim.x) {
    const RowUnit ru = row_unit(offr, n_chains, u);
    const Chain<T>& c = chains[ru.ci];
    const int m = ru.m, spin = ru.spin, j = ru.i, ld = c.ld, buf = c.dyn->buf;
    const E* X = reinterpret_cast<const E*>(c.work + (size_t)spin * refresh_work_per_spin(ld));
    const int* perm = c.perm + spin * ld;
    T* Nr = c.N[buf][spin];
    float* NTr = c.NT[buf][spin];   // N^T kept for the tensor-core prep (mixed form), or null
    double* N64 = (filter == 1) ? c.N64[spin] : nullptr;
    const int pj = perm[j];
    double dmax = 0.0, dsq = 0.0, nmax = 0.0;
    for (int cc = threadIdx.x; cc < m; cc += blockDim.x) {
      const double v = el_to(X[(size_t)j * ld + perm[cc]]);  // N[cc][perm[j]]
      const long o = (long)pj * ld + cc;
      if (N64) N64[o] = v;
      const double diff = fabs((double)Nr[o] - v);
      dmax = fmax(dmax, diff);
      dsq += diff * diff;
      nmax = fmax(nmax, fabs(v));
      Nr[o] = (T)v;
      if (NTr) NTr[(long)cc * ld + pj] = (float)v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      dsq += __shfl_xor_sync(0xffffffffu, dsq, o);
      nmax = fmax(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = dmax;
      red[1][threadIdx.x >> 5] = dsq;
      red[2][threadIdx.x >> 5] = nmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bm = 0.0, bs = 0.0, bn = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        bm = fmax(bm, red[0][w]);
        bs += red[1][w];
        bn = fmax(bn, red[2][w]);
      }
      // non-negative doubles order like their bit patterns
      if (bm > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(&c.work_drift[0]),
                  (unsigned long long)__double_as_longlong(bm));
      if (bs > 0.0) atomicAdd(&c.work_drift[1], bs);
      if (bn > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(&c.work_drift[2]),
                  (unsigned long long)__double_as_longlong(bn));
    }
  }
  grid.sync();  // every column has read perm before the flags are cleared
  for (int u = gtid; u < tot_r; u += gthreads) {
    const RowUnit ru = row_unit(offr, n_chains, u);
    const Chain<T>& c = chains[ru.ci];
    const int ld = c.ld;
    c.pkeys[(size_t)ru.spin * ld + ru.i] = 0ull;
    c.used[ru.spin * ld + ru.i] = 0;
    c.pcol[ru.spin * ld + ru.i] = -1;
  }
}

// Permutation signs, log det and drift of a refreshed chain into its stats.
template <typename T>
__device__ __forceinline__ void refresh_finish_one(const Chain<T>& c, int filter) {
  Dyn& d = *c.dyn;
  if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) return;
  d.refreshes += 1;
  d.work_refresh += 4.0 * (double)d.n * (double)d.n * (double)d.n;  // 2 m^3 per spin
  d.drift_max = c.work_drift[0];
  d.drift_fro = sqrt(c.work_drift[1]);
  d.drift_rel = c.work_drift[2] > 0.0 ? c.work_drift[0] / c.work_drift[2] : 0.0;
  if (c.drift_limit > 0.0 && d.drift_rel > c.drift_limit) d.drift_exceeded = 1;
  c.work_drift[0] = 0.0;
  c.work_drift[1] = 0.0;
  c.work_drift[2] = 0.0;
  for (int spin = 0; spin < 2; ++spin) d.logdet[spin] = c.work_logdet[spin];
}

}  // namespace ctaux
