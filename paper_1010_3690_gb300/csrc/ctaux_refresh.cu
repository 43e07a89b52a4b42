// From-scratch FP64 recomputation of N for every chain: build
// N^{-1} = e^V - G0 (e^V - 1) (Eq. Nmatrix) from the configuration, invert
// by Gauss-Jordan with partial pivoting, report the drift of the running N
// and replace it.  One cooperative launch: the column steps of all chains
// and spins run in lockstep, separated by grid-wide barriers (no spin waits).
//
// Column step c reads matrix X and writes Y (ping-pong), with pivot row pr:
//   Y[pr][j] = X[pr][j] / X[pr][c]            (j != c),  Y[pr][c] = 1 / X[pr][c]
//   Y[i][j]  = X[i][j] - X[i][c] X[pr][j] / X[pr][c]   (i != pr, j != c)
//   Y[i][c]  = -X[i][c] / X[pr][c]                      (i != pr)
// After m steps with pivot rows perm[c], N[c][perm[j]] = X[perm[c]][j] and
// det N^{-1} = sign(perm) prod_c X_c[perm[c]][c].
// The pivot of the next column is found while a step writes it: each CTA
// folds max |Y[i][c+1]| over not-yet-pivoted rows into one 64-bit key per
// (chain, spin, step) with atomicMax (float magnitude, ties to the lower row).
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

template <typename T>
__global__ void __launch_bounds__(256) k_refresh(Chain<T>* chains, int n_chains, int only_chain) {
  cg::grid_group grid = cg::this_grid();
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gthreads = (long)gridDim.x * blockDim.x;
  const int c_lo = only_chain >= 0 ? only_chain : 0;
  const int c_hi = only_chain >= 0 ? only_chain + 1 : n_chains;

  // ---- stage 1: N^{-1} of the current configuration into work[0]; pivot of column 0
  int max_m = 0;
  for (int ci = c_lo; ci < c_hi; ++ci) {
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    if (d.status & ~DS_SINGULAR) continue;
    const int m = d.n, buf = d.buf, ld = c.ld;
    max_m = max(max_m, m);
    if (gtid == 0) c.work_logdet[0] = c.work_logdet[1] = 0.0;
    for (int spin = 0; spin < 2; ++spin) {
      double* X = c.work + (size_t)spin * 2 * ld * ld;
      unsigned long long* keys = c.pkeys + (size_t)spin * ld;
      int8_t* used = c.used + spin * ld;
      for (long e = gtid; e < (long)m * m; e += gthreads) {
        const int i = (int)(e % m), j = (int)(e / m);
        const double evj = c.ev[spin][c.s[buf][j] + 2];
        double v = -g0_eval(c, spin, c.tau[buf][i], c.site[buf][i], c.tau[buf][j], c.site[buf][j]) *
                   (evj - 1.0);
        if (i == j) v += evj;
        X[(size_t)j * ld + i] = v;
        if (j == 0) atomicMax(keys, pivot_key(v, i));
      }
    }
  }
  grid.sync();

  // ---- stage 2: m Gauss-Jordan column steps
  for (int col = 0; col < max_m; ++col) {
    for (int ci = c_lo; ci < c_hi; ++ci) {
      const Chain<T>& c = chains[ci];
      const Dyn& d = *c.dyn;
      if (d.status & ~DS_SINGULAR) continue;
      const int m = d.n, ld = c.ld;
      if (col >= m) continue;
      for (int spin = 0; spin < 2; ++spin) {
        const double* X = c.work + (size_t)spin * 2 * ld * ld + (size_t)(col & 1) * ld * ld;
        double* Y = c.work + (size_t)spin * 2 * ld * ld + (size_t)((col + 1) & 1) * ld * ld;
        unsigned long long* keys = c.pkeys + (size_t)spin * ld;
        int8_t* used = c.used + spin * ld;
        const int pr = key_row(keys[col]);
        const double piv = X[(size_t)col * ld + pr];
        if (gtid == 0) {
          c.perm[spin * ld + col] = pr;
          used[pr] = 1;
          if (!(fabs(piv) > 0.0) || !isfinite(piv)) atomicOr(&c.dyn->status, DS_SINGULAR);
          c.work_logdet[spin] += log(fabs(piv));
        }
        const double ipiv = 1.0 / piv;
        // columns over CTAs, rows over threads
        for (int j = blockIdx.x; j < m; j += gridDim.x) {
          const double xpj = X[(size_t)j * ld + pr] * ipiv;
          const double* Xj = X + (size_t)j * ld;
          const double* Xc = X + (size_t)col * ld;
          double* Yj = Y + (size_t)j * ld;
          for (int i = threadIdx.x; i < m; i += blockDim.x) {
            double v;
            if (i == pr) v = (j == col) ? ipiv : xpj;
            else if (j == col) v = -Xc[i] * ipiv;
            else v = Xj[i] - Xc[i] * xpj;
            Yj[i] = v;
            if (j == col + 1 && i != pr && !used[i]) atomicMax(keys + col + 1, pivot_key(v, i));
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
    if (d.status & ~DS_SINGULAR) continue;
    const int m = d.n, ld = c.ld, buf = d.buf;
    for (int spin = 0; spin < 2; ++spin) {
      const double* X = c.work + (size_t)spin * 2 * ld * ld + (size_t)(m & 1) * ld * ld;
      const int* perm = c.perm + spin * ld;
      T* Nr = c.N[buf][spin];
      for (long e = gtid; e < (long)m * m; e += gthreads) {
        const int cc = (int)(e % m), j = (int)(e / m);
        const double v = X[(size_t)j * ld + perm[cc]];  // N[cc][perm[j]]
        const long o = (long)perm[j] * ld + cc;
        const double diff = fabs((double)Nr[o] - v);
        if (diff > 0.0) {
          atomicMax(reinterpret_cast<unsigned long long*>(&c.work_drift[0]),
                    (unsigned long long)__double_as_longlong(diff));
          atomicAdd(&c.work_drift[1], diff * diff);
        }
        Nr[o] = (T)v;
      }
      for (long e = gtid; e < m; e += gthreads) {
        c.pkeys[(size_t)spin * ld + e] = 0ull;
        c.used[spin * ld + e] = 0;
      }
    }
  }
}

// Small follow-up kernel: permutation signs, log det, drift into the stats.
template <typename T>
__global__ void k_refresh_finish(Chain<T>* chains, int n_chains, int only_chain) {
  const int ci = (only_chain >= 0) ? only_chain : (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (ci >= n_chains) return;
  if (only_chain >= 0 && (blockIdx.x | threadIdx.x)) return;
  const Chain<T>& c = chains[ci];
  Dyn& d = *c.dyn;
  if (d.status & ~DS_SINGULAR) return;
  d.refreshes += 1;
  d.drift_max = c.work_drift[0];
  d.drift_fro = sqrt(c.work_drift[1]);
  c.work_drift[0] = 0.0;
  c.work_drift[1] = 0.0;
  for (int spin = 0; spin < 2; ++spin) d.logdet[spin] = c.work_logdet[spin];
}

template <typename T>
cudaError_t launch_refresh(Chain<T>* dchains, const LaunchShape& ls, int only_chain,
                           cudaStream_t st, PhaseTimer* pt) {
  pt->begin(6, st);
  int nch = ls.n_chains;
  void* args[] = {&dchains, &nch, &only_chain};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_refresh<T>, dim3(ls.refresh_grid),
                                              dim3(256), args, 0, st);
  if (e == cudaSuccess) {
    if (only_chain >= 0)
      k_refresh_finish<T><<<1, 1, 0, st>>>(dchains, nch, only_chain);
    else
      k_refresh_finish<T><<<(nch + 127) / 128, 128, 0, st>>>(dchains, nch, -1);
    e = cudaGetLastError();
  }
  pt->end(6, st, 2);
  return e;
}

template <typename T>
int refresh_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refresh<T>, 256, 0);
  return nb;
}

template cudaError_t launch_refresh<double>(Chain<double>*, const LaunchShape&, int, cudaStream_t,
                                            PhaseTimer*);
template cudaError_t launch_refresh<float>(Chain<float>*, const LaunchShape&, int, cudaStream_t,
                                           PhaseTimer*);
template int refresh_blocks_per_sm<double>();
template int refresh_blocks_per_sm<float>();

}  // namespace ctaux
