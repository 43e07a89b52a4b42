// From-scratch FP64 recomputation of N for every chain: build
// N^{-1} = e^V - G0 (e^V - 1) (Eq. Nmatrix) from the configuration, invert
// by blocked Gauss-Jordan with partial pivoting, report the drift of the
// running N and replace it.  One cooperative launch: all chains and spins
// advance in lockstep, separated by grid-wide barriers (no spin waits).
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
// previous step writes that column: atomicMax of a 64-bit key (float
// magnitude, ties to the lower row) per (chain, spin, column).
#include <cooperative_groups.h>

#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"

namespace cg = cooperative_groups;

namespace ctaux {

__device__ __forceinline__ unsigned long long pivot_key(double v, int row) {
  const float a = (float)fabs(v);
  return ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)(0xffffffffu - (unsigned)row);
}
__device__ __forceinline__ int key_row(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

constexpr int kPB = 32;  // panel width

// per-spin work area: X (ld x ld), two panel buffers (ld x kPB), pivot rows (ld x kPB)
__host__ __device__ inline size_t refresh_work_per_spin(int ld) {
  return (size_t)ld * ld + (size_t)3 * kPB * ld;
}

template <typename T>
__global__ void __launch_bounds__(256) k_refresh(Chain<T>* chains, int n_chains, int only_chain,
                                                 int filter) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  const int c_lo = only_chain >= 0 ? only_chain : 0;
  const int c_hi = only_chain >= 0 ? only_chain + 1 : n_chains;
  __shared__ double Ps[32][kPB + 1];
  __shared__ double Rs[kPB][33];

  // ---- stage 1: N^{-1} of the current configuration into X; pivot of column 0
  int max_m = 0;
  for (int ci = c_lo; ci < c_hi; ++ci) {
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
    const int m = d.n, buf = d.buf, ld = c.ld;
    max_m = max(max_m, m);
    if (gtid == 0) c.work_logdet[0] = c.work_logdet[1] = 0.0;
    for (int spin = 0; spin < 2; ++spin) {
      double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
      unsigned long long* keys = c.pkeys + (size_t)spin * ld;
      for (int j = blockIdx.x; j < m; j += gridDim.x) {
        const double evj = c.ev[spin][c.s[buf][j] + 2];
        const double tj = c.tau[buf][j];
        const int sj = c.site[buf][j];
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          double v = -g0_eval(c, spin, c.tau[buf][i], c.site[buf][i], tj, sj) * (evj - 1.0);
          if (i == j) v += evj;
          X[(size_t)j * ld + i] = v;
          if (j == 0) atomicMax(keys, pivot_key(v, i));
        }
      }
    }
  }
  grid.sync();

  // ---- stage 2: panels
  for (int c0 = 0; c0 < max_m; c0 += kPB) {
    // A0: copy the panel columns
    for (int ci = c_lo; ci < c_hi; ++ci) {
      const Chain<T>& c = chains[ci];
      const Dyn& d = *c.dyn;
      if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
      const int m = d.n, ld = c.ld;
      if (c0 >= m) continue;
      const int bw = min(kPB, m - c0);
      for (int spin = 0; spin < 2; ++spin) {
        const double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
        double* Pa = const_cast<double*>(X) + (size_t)ld * ld;
        for (int e = gtid; e < m * bw; e += gthreads) {
          const int i = e % m, k = e / m;
          Pa[(size_t)k * ld + i] = X[(size_t)(c0 + k) * ld + i];
        }
      }
    }
    grid.sync();
    // A1: the column steps, on the panel only
    for (int k = 0; k < kPB; ++k) {
      for (int ci = c_lo; ci < c_hi; ++ci) {
        const Chain<T>& c = chains[ci];
        const Dyn& d = *c.dyn;
        if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
        const int m = d.n, ld = c.ld;
        if (c0 + k >= m) continue;
        const int bw = min(kPB, m - c0), col = c0 + k;
        for (int spin = 0; spin < 2; ++spin) {
          double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
          double* Pa = X + (size_t)ld * ld;
          double* Pb = Pa + (size_t)kPB * ld;
          const double* src = (k & 1) ? Pb : Pa;
          double* dst = (k & 1) ? Pa : Pb;
          unsigned long long* keys = c.pkeys + (size_t)spin * ld;
          int8_t* used = c.used + spin * ld;
          const int pr = key_row(keys[col]);
          const double piv = src[(size_t)k * ld + pr];
          if (gtid == 0) {
            c.perm[spin * ld + col] = pr;
            used[pr] = 1;
            c.pcol[spin * ld + pr] = col;
            if (!(fabs(piv) > 0.0) || !isfinite(piv)) atomicOr(&c.dyn->status, DS_SINGULAR);
            c.work_logdet[spin] += log(fabs(piv));
          }
          const double ipiv = 1.0 / piv;
          // one (row, panel column) pair per thread
          for (int e = gtid; e < m * bw; e += gthreads) {
            const int i = e % m, kk = e / m;
            const double xic = src[(size_t)k * ld + i];
            double v;
            if (i == pr) v = (kk == k) ? ipiv : src[(size_t)kk * ld + pr] * ipiv;
            else if (kk == k) v = -xic * ipiv;
            else v = src[(size_t)kk * ld + i] - xic * (src[(size_t)kk * ld + pr] * ipiv);
            dst[(size_t)kk * ld + i] = v;
            if (kk == k + 1 && i != pr && !used[i]) atomicMax(keys + col + 1, pivot_key(v, i));
          }
        }
      }
      grid.sync();
    }
    // B0: pivot rows of this panel, outside it, from X before the update: Rr[j][k] = X[R_k][j]
    for (int ci = c_lo; ci < c_hi; ++ci) {
      const Chain<T>& c = chains[ci];
      const Dyn& d = *c.dyn;
      if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
      const int m = d.n, ld = c.ld;
      if (c0 >= m) continue;
      const int bw = min(kPB, m - c0);
      for (int spin = 0; spin < 2; ++spin) {
        const double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
        double* Rr = const_cast<double*>(X) + (size_t)ld * ld + (size_t)2 * kPB * ld;
        const int* perm = c.perm + spin * ld;
        for (int e = gtid; e < m * kPB; e += gthreads) {
          const int k = e % kPB, j = e / kPB;
          Rr[(size_t)j * kPB + k] = (k < bw) ? X[(size_t)j * ld + perm[c0 + k]] : 0.0;
        }
      }
    }
    grid.sync();
    // B1: trailing rank-bw update in 32 x 32 tiles, panel written back,
    // pivot key of the next panel's first column
    for (int ci = c_lo; ci < c_hi; ++ci) {
      const Chain<T>& c = chains[ci];
      const Dyn& d = *c.dyn;
      if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
      const int m = d.n, ld = c.ld;
      if (c0 >= m) continue;
      const int bw = min(kPB, m - c0), cn = c0 + bw;
      const int tb = (m + 31) / 32;
      for (int spin = 0; spin < 2; ++spin) {
        double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
        double* Pa = X + (size_t)ld * ld;
        const double* Pf = (bw & 1) ? Pa + (size_t)kPB * ld : Pa;  // panel after bw steps
        const double* Rr = Pa + (size_t)2 * kPB * ld;
        unsigned long long* keys = c.pkeys + (size_t)spin * ld;
        const int8_t* used = c.used + spin * ld;
        const int* pcol = c.pcol + spin * ld;
        for (int tile = blockIdx.x; tile < tb * tb; tile += gridDim.x) {
          const int i0 = (tile % tb) * 32, j0 = (tile / tb) * 32;
          __syncthreads();
          for (int e = threadIdx.x; e < 32 * kPB; e += blockDim.x) {
            const int r = e % 32, k = e / 32;
            Ps[r][k] = (i0 + r < m && k < bw) ? Pf[(size_t)k * ld + i0 + r] : 0.0;
            const int jj = e % 32, kk = e / 32;
            Rs[kk][jj] = (j0 + jj < m) ? Rr[(size_t)(j0 + jj) * kPB + kk] : 0.0;
          }
          __syncthreads();
          const int r = threadIdx.x % 32, i = i0 + r;
          if (i < m) {
            const int pci = pcol[i];
            const bool in_R = pci >= c0 && pci < cn;
            for (int q = threadIdx.x / 32; q < 32; q += blockDim.x / 32) {
              const int j = j0 + q;
              if (j >= m) continue;
              double v;
              if (j >= c0 && j < cn) {
                v = Ps[r][j - c0];
              } else {
                double acc = in_R ? 0.0 : X[(size_t)j * ld + i];
#pragma unroll 8
                for (int k = 0; k < kPB; ++k) acc += Ps[r][k] * Rs[k][q];
                v = acc;
              }
              X[(size_t)j * ld + i] = v;
              if (j == cn && !used[i]) atomicMax(keys + cn, pivot_key(v, i));
            }
          }
        }
      }
    }
    grid.sync();
  }

  // ---- stage 3: unscramble, drift against the running N, replace it;
  // clear the pivot keys and flags for the next refresh
  for (int ci = c_lo; ci < c_hi; ++ci) {
    const Chain<T>& c = chains[ci];
    Dyn& d = *c.dyn;
    if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) continue;
    const int m = d.n, ld = c.ld, buf = d.buf;
    for (int spin = 0; spin < 2; ++spin) {
      const double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
      const int* perm = c.perm + spin * ld;
      T* Nr = c.N[buf][spin];
      double* N64 = (filter == 1) ? c.N64[spin] : nullptr;
      for (int j = blockIdx.x; j < m; j += gridDim.x) {
        const int pj = perm[j];
        for (int cc = threadIdx.x; cc < m; cc += blockDim.x) {
          const double v = X[(size_t)j * ld + perm[cc]];  // N[cc][perm[j]]
          const long o = (long)pj * ld + cc;
          if (N64) N64[o] = v;
          const double diff = fabs((double)Nr[o] - v);
          if (diff > 0.0) {
            atomicMax(reinterpret_cast<unsigned long long*>(&c.work_drift[0]),
                      (unsigned long long)__double_as_longlong(diff));
            atomicAdd(&c.work_drift[1], diff * diff);
          }
          Nr[o] = (T)v;
        }
      }
      for (int e = gtid; e < m; e += gthreads) {
        c.pkeys[(size_t)spin * ld + e] = 0ull;
        c.used[spin * ld + e] = 0;
        c.pcol[spin * ld + e] = -1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Batched form: one CTA per (chain, spin), the same blocked Gauss-Jordan with
// block-level barriers.  The panel (m x 16 float64) lives in shared memory and
// is updated in place (the pivot row is copied first); pivots come from a
// block reduction; the trailing rank-16 update streams X through the CTA,
// with the pivot rows X[R, :] saved in the work area beforehand.
constexpr int kPBc = 16;

__device__ __forceinline__ void block_argmax(double v, int row, double* rv, int* ri) {
  // max |v| (ties to the lower row) over the block; result in rv[0], ri[0]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int r2 = __shfl_down_sync(0xffffffffu, row, o);
    if (v2 > v || (v2 == v && r2 < row)) {
      v = v2;
      row = r2;
    }
  }
  __syncthreads();
  if (lane == 0) {
    rv[w] = v;
    ri[w] = row;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (rv[k] > rv[0] || (rv[k] == rv[0] && ri[k] < ri[0])) {
        rv[0] = rv[k];
        ri[0] = ri[k];
      }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) k_refresh_cta(Chain<T>* chains, int n_chains, int filter) {
  const int ci = blockIdx.x >> 1, spin = blockIdx.x & 1;
  if (ci >= n_chains) return;
  const Chain<T>& c = chains[ci];
  Dyn& d = *c.dyn;
  if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) return;
  const int m = d.n, ld = c.ld, buf = d.buf;
  double* X = c.work + (size_t)spin * refresh_work_per_spin(ld);
  double* Rr = X + (size_t)ld * ld;       // pivot rows of the current panel, [j][k]
  int* perm = c.perm + spin * ld;
  int8_t* used = c.used + spin * ld;
  int* pcol = c.pcol + spin * ld;
  extern __shared__ __align__(16) double panel[];  // [k][i], kPBc x m
  __shared__ double prow[kPBc];
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ double logdet_s;
  if (threadIdx.x == 0) logdet_s = 0.0;
  // N^{-1} of the configuration
  for (int j = 0; j < m; ++j) {
    const double evj = c.ev[spin][c.s[buf][j] + 2];
    const double tj = c.tau[buf][j];
    const int sj = c.site[buf][j];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double v = -g0_eval(c, spin, c.tau[buf][i], c.site[buf][i], tj, sj) * (evj - 1.0);
      if (i == j) v += evj;
      X[(size_t)j * ld + i] = v;
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    used[i] = 0;
    pcol[i] = -1;
  }
  __syncthreads();
  for (int c0 = 0; c0 < m; c0 += kPBc) {
    const int bw = min(kPBc, m - c0);
    for (int e = threadIdx.x; e < m * bw; e += blockDim.x) {
      const int i = e % m, k = e / m;
      panel[(size_t)k * m + i] = X[(size_t)(c0 + k) * ld + i];
    }
    __syncthreads();
    for (int k = 0; k < bw; ++k) {
      const int col = c0 + k;
      double best = -1.0;
      int brow = 0x7fffffff;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double a = used[i] ? -1.0 : fabs(panel[(size_t)k * m + i]);
        if (a > best || (a == best && i < brow)) {
          best = a;
          brow = i;
        }
      }
      block_argmax(best, brow, rv, ri);
      const int pr = ri[0];
      const double piv = panel[(size_t)k * m + pr];
      if (threadIdx.x == 0) {
        perm[col] = pr;
        used[pr] = 1;
        pcol[pr] = col;
        if (!(fabs(piv) > 0.0) || !isfinite(piv)) atomicOr(&d.status, DS_SINGULAR);
        logdet_s += log(fabs(piv));
      }
      const double ipiv = 1.0 / piv;
      if (threadIdx.x < bw) prow[threadIdx.x] = panel[(size_t)threadIdx.x * m + pr] * ipiv;
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double xic = panel[(size_t)k * m + i];
        for (int kk = 0; kk < bw; ++kk) {
          double v;
          if (i == pr) v = (kk == k) ? ipiv : prow[kk];
          else if (kk == k) v = -xic * ipiv;
          else v = panel[(size_t)kk * m + i] - xic * prow[kk];
          panel[(size_t)kk * m + i] = v;
        }
      }
      __syncthreads();
    }
    // pivot rows outside the panel, before the update
    for (int e = threadIdx.x; e < m * bw; e += blockDim.x) {
      const int k = e % bw, j = e / bw;
      Rr[(size_t)j * kPBc + k] = X[(size_t)j * ld + perm[c0 + k]];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      double* Xj = X + (size_t)j * ld;
      if (j >= c0 && j < c0 + bw) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) Xj[i] = panel[(size_t)(j - c0) * m + i];
        continue;
      }
      double r[kPBc];
#pragma unroll
      for (int k = 0; k < kPBc; ++k) r[k] = (k < bw) ? Rr[(size_t)j * kPBc + k] : 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int pci = pcol[i];
        double acc = (pci >= c0 && pci < c0 + bw) ? 0.0 : Xj[i];
#pragma unroll
        for (int k = 0; k < kPBc; ++k)
          if (k < bw) acc += panel[(size_t)k * m + i] * r[k];
        Xj[i] = acc;
      }
    }
    __syncthreads();
  }
  // unscramble, drift, replace
  T* Nr = c.N[buf][spin];
  double* N64 = (filter == 1) ? c.N64[spin] : nullptr;
  double dmax = 0.0, dsq = 0.0;
  for (int j = 0; j < m; ++j) {
    const int pj = perm[j];
    for (int cc = threadIdx.x; cc < m; cc += blockDim.x) {
      const double v = X[(size_t)j * ld + perm[cc]];
      const long o = (long)pj * ld + cc;
      if (N64) N64[o] = v;
      const double diff = fabs((double)Nr[o] - v);
      dmax = fmax(dmax, diff);
      dsq += diff * diff;
      Nr[o] = (T)v;
    }
  }
  if (dmax > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&c.work_drift[0]),
              (unsigned long long)__double_as_longlong(dmax));
  if (dsq > 0.0) atomicAdd(&c.work_drift[1], dsq);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    used[i] = 0;
    pcol[i] = -1;
    c.pkeys[(size_t)spin * ld + i] = 0ull;
  }
  __syncthreads();
  if (threadIdx.x == 0) c.work_logdet[spin] = logdet_s;
}

// Small follow-up kernel: permutation signs, log det, drift into the stats.
template <typename T>
__global__ void k_refresh_finish(Chain<T>* chains, int n_chains, int only_chain, int filter) {
  const int ci = (only_chain >= 0) ? only_chain : (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (ci >= n_chains) return;
  if (only_chain >= 0 && (blockIdx.x | threadIdx.x)) return;
  const Chain<T>& c = chains[ci];
  Dyn& d = *c.dyn;
  if ((d.status & ~DS_SINGULAR) || (filter && d.tie_pending != filter)) return;
  d.refreshes += 1;
  d.drift_max = c.work_drift[0];
  d.drift_fro = sqrt(c.work_drift[1]);
  c.work_drift[0] = 0.0;
  c.work_drift[1] = 0.0;
  for (int spin = 0; spin < 2; ++spin) d.logdet[spin] = c.work_logdet[spin];
}

template <typename T>
cudaError_t launch_refresh(Chain<T>* dchains, const LaunchShape& ls, int only_chain,
                           cudaStream_t st, PhaseTimer* pt, int filter) {
  pt->begin(6, st);
  int nch = ls.n_chains;
  cudaError_t e = cudaSuccess;
  if (only_chain < 0 && ls.refresh_per_cta) {
    k_refresh_cta<T><<<2 * nch, 512, ls.refresh_cta_smem, st>>>(dchains, nch, filter);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      k_refresh_finish<T><<<(nch + 127) / 128, 128, 0, st>>>(dchains, nch, -1, filter);
    e = cudaGetLastError();
    pt->end(6, st, 2);
    return e;
  }
  void* args[] = {&dchains, &nch, &only_chain, &filter};
  e = cudaLaunchCooperativeKernel((const void*)k_refresh<T>, dim3(ls.refresh_grid), dim3(256),
                                  args, 0, st);
  if (e == cudaSuccess) {
    if (only_chain >= 0)
      k_refresh_finish<T><<<1, 1, 0, st>>>(dchains, nch, only_chain, filter);
    else
      k_refresh_finish<T><<<(nch + 127) / 128, 128, 0, st>>>(dchains, nch, -1, filter);
    e = cudaGetLastError();
  }
  pt->end(6, st, 2);
  return e;
}

template <typename T>
cudaError_t configure_refresh_cta(int smem) {
  return cudaFuncSetAttribute(k_refresh_cta<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template cudaError_t configure_refresh_cta<double>(int);
template cudaError_t configure_refresh_cta<float>(int);

template <typename T>
int refresh_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refresh<T>, 256, 0);
  return nb;
}

template cudaError_t launch_refresh<double>(Chain<double>*, const LaunchShape&, int, cudaStream_t,
                                            PhaseTimer*, int);
template cudaError_t launch_refresh<float>(Chain<float>*, const LaunchShape&, int, cudaStream_t,
                                           PhaseTimer*, int);
size_t refresh_work_doubles(int ld) { return 2 * refresh_work_per_spin(ld); }

template int refresh_blocks_per_sm<double>();
template int refresh_blocks_per_sm<float>();

}  // namespace ctaux
