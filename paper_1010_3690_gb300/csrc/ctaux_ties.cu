// FP64 decisions of near ties in the mixed form (one cooperative launch per block).
#include <cooperative_groups.h>

#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"
#include "ctaux_refresh.cuh"

namespace ctaux {

// Mixed form: the proposal d.t that the float32 block stopped at is decided in
// FP64 with the first-touch formula ratio_sigma = 1 + lambda (1 - G_pp)
// (Eq. Akp1Ak, reading C2):
//   removal / flip of slot p: G_pp = (N_pp e^{V_p} - 1) / (e^{V_p} - 1) (Eq. NfromG);
//   insertion of a vertex p:  G_pp = G0(p,p) + sum_l G0(p,l)(e^{V_l}-1) (N g)_l,
//                             g_k = G0(k,p) (the s=0 row of N_ext, Sec. IV A).
// The decision is stored (forced_t) and the next block applies the move
// through the float32 path.  k_tie_refine obtains N e_p or N g to FP64
// accuracy by iterative refinement, A x = b with A = N^{-1} rebuilt in FP64
// from the configuration (Eq. Nmatrix) and the float32 N as preconditioner;
// where that does not converge within max_iter iterations, the same launch
// refreshes the pending chains from scratch in FP64, keeping the FP64 N, and
// decides from it (tie_eval_chain).
struct TieProposal {
  int move, p, s_new, site_new, none;
  double f, tau_new;
  Draws dr;
};

__device__ __forceinline__ TieProposal tie_proposal(const Chain<float>& c, const Dyn& d) {
  TieProposal q;
  q.dr = draw(c.seed, c.chain_id, d.t);
  q.move = move_of(q.dr.u_move, c.p_insert, c.p_remove);
  q.p = -1;
  q.s_new = 0;
  q.site_new = 0;
  q.tau_new = 0.0;
  q.f = 0.0;
  const int n = d.n;
  const int8_t* sv = c.s[d.buf];
  if (q.move == MV_INSERT) {
    q.tau_new = q.dr.u_tau * c.beta;
    q.site_new = (int)floor(q.dr.u_site * (double)c.n_c);
    if (q.site_new > c.n_c - 1) q.site_new = c.n_c - 1;
    q.s_new = (q.dr.u_spin < 0.5) ? 1 : -1;
    q.f = c.K / (double)(n + 1);
  } else if (n > 0) {
    int idx = (int)floor(q.dr.u_idx * (double)n);
    if (idx > n - 1) idx = n - 1;
    q.p = idx;
    q.s_new = (q.move == MV_REMOVE) ? 0 : -(int)sv[q.p];
    q.f = (q.move == MV_REMOVE) ? (double)n / c.K : 1.0;
  }
  q.none = (q.move != MV_INSERT && n == 0);
  return q;
}

__device__ __forceinline__ void set_forced(const Chain<float>& c, Dyn& d, const TieProposal& q,
                                           const double* ratio) {
  const double R = q.none ? 0.0 : q.f * ratio[0] * ratio[1];
  const bool finite = isfinite(R);
  d.forced_accept = (!q.none && finite && q.dr.u_acc < fmin(1.0, fabs(R))) ? 1 : 0;
  d.forced_ratio[0] = q.none ? 0.0 : ratio[0];
  d.forced_ratio[1] = q.none ? 0.0 : ratio[1];
  d.forced_R = R;
  d.forced_t = d.t;
  d.tie_pending = 0;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  return tot;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  return mx;
}

// Fallback: decide from the FP64 N of a from-scratch refresh (N64).
__device__ void tie_eval_chain(const Chain<float>& c) {
  Dyn& d = *c.dyn;
  if (d.status || d.tie_pending != 1) return;  // the same in every thread of the CTA
  const TieProposal q = tie_proposal(c, d);
  __shared__ double red[8];
  __shared__ double ratio[2];
  __syncthreads();  // the previous chain's readers of ratio are done
  const int n = d.n, buf = d.buf, ld = c.ld;
  const double* tau = c.tau[buf];
  const int* site = c.site[buf];
  const int8_t* sv = c.s[buf];
  for (int spin = 0; spin < 2 && !q.none; ++spin) {
    const double* N64 = c.N64[spin];
    double gpp, lam;
    if (q.move == MV_INSERT) {
      double* gvec = c.work + (size_t)spin * ((size_t)ld * ld + (size_t)96 * ld);  // scratch
      for (int k = threadIdx.x; k < n; k += blockDim.x)
        gvec[k] = g0_eval(c, spin, tau[k], site[k], q.tau_new, q.site_new);
      __syncthreads();
      double part = 0.0;
      for (int l = threadIdx.x; l < n; l += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < n; ++k) v += N64[(size_t)k * ld + l] * gvec[k];
        part += g0_eval(c, spin, q.tau_new, q.site_new, tau[l], site[l]) * (c.ev[spin][sv[l] + 2] - 1.0) * v;
      }
      gpp = g0_eval(c, spin, q.tau_new, q.site_new, q.tau_new, q.site_new) + block_sum(part, red);
      lam = c.ev[spin][q.s_new + 2] - 1.0;
    } else {
      const int k = sv[q.p] + 2;
      gpp = (N64[(size_t)q.p * ld + q.p] * c.ev[spin][k] - 1.0) * c.inv_em1[spin][k];
      lam = c.ev[spin][q.s_new - sv[q.p] + 2] - 1.0;
    }
    if (threadIdx.x == 0) ratio[spin] = 1.0 + lam * (1.0 - gpp);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (q.none) ratio[0] = ratio[1] = 0.0;
    set_forced(c, d, q, ratio);
    d.tie_refreshes += 1;
  }
}


// y_s = M_s v_s for both spins s over the whole grid, M_s column-major with
// leading dimension ld: slice sl of the columns of spin s writes its partial
// sums to P_s[sl*ld + i] (P_s = P + s*kTieSlices*ld); the caller adds the ns
// partials in slice order after a grid barrier (deterministic).
template <typename Tm>
__device__ __forceinline__ void grid_gemv_partials2(const Tm* M0, const Tm* M1, int ld, int n,
                                                    const double* v0, const double* v1, double* P,
                                                    int ns, int gtid, int gthreads) {
  const int rp = (n + 31) & ~31;
  const int per_spin = ns * rp;
  for (int idx = gtid; idx < 2 * per_spin; idx += gthreads) {
    const int spin = idx / per_spin, l = idx - spin * per_spin;
    const int i = l % rp, sl = l / rp;
    if (i >= n) continue;
    const Tm* M = spin ? M1 : M0;
    const double* v = spin ? v1 : v0;
    const int j0 = (int)((long long)sl * n / ns), j1 = (int)((long long)(sl + 1) * n / ns);
    double a0 = 0.0, a1 = 0.0;
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      a0 += (double)M[(size_t)j * ld + i] * v[j];
      a1 += (double)M[(size_t)(j + 1) * ld + i] * v[j + 1];
    }
    if (j < j1) a0 += (double)M[(size_t)j * ld + i] * v[j];
    P[(size_t)spin * kTieSlices * ld + (size_t)sl * ld + i] = a0 + a1;
  }
}

__device__ __forceinline__ double slice_sum(const double* P, int ld, int ns, int spin, int i) {
  const double* Ps = P + (size_t)spin * kTieSlices * ld;
  double t = 0.0;
  for (int sl = 0; sl < ns; ++sl) t += Ps[(size_t)sl * ld + i];
  return t;
}

// Cooperative over the whole GPU, one pending tie at a time, both spins at
// once: A_s (FP64) is built across all CTAs, then x_s <- x_s + N_s (b_s - A_s
// x_s) iterates until both spins have converged; each matrix-vector product
// is split over column slices, and the convergence maxima go through per-CTA
// partials read in CTA order.
__global__ void __launch_bounds__(256) k_tie_refine(Chain<float>* chains, int n_chains,
                                                    double* part, double* slices, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  __shared__ double red[8];
  __shared__ unsigned pend[kMaxChains / 32];  // chains with a pending tie, as bits
  const int nwords = (n_chains + 31) / 32;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) pend[w] = 0u;
  __syncthreads();
  // every CTA reads the same flags: they change only after the first grid barrier
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
    const Dyn& d = *chains[ci].dyn;
    if (!d.status && d.tie_pending == 1) atomicOr(&pend[ci >> 5], 1u << (ci & 31));
  }
  __syncthreads();
  bool any_fail = false;
  for (int wd = 0; wd < nwords; ++wd)
  for (unsigned bits = pend[wd]; bits; bits &= bits - 1) {
    const int ci = wd * 32 + __ffs(bits) - 1;  // increasing chain order in every CTA
    const Chain<float>& c = chains[ci];
    Dyn& d = *c.dyn;
    const TieProposal q = tie_proposal(c, d);
    const int n = d.n, buf = d.buf, ld = c.ld;
    const int ns = max(1, min(kTieSlices, gthreads / (2 * ((n + 31) & ~31))));
    const double* tau = c.tau[buf];
    const int* site = c.site[buf];
    const int8_t* sv = c.s[buf];
    double ratio[2] = {0.0, 0.0};
    bool ok = max_iter > 0;
    if (!q.none && ok) {
      const float* N0 = c.N[buf][0];
      const float* N1 = c.N[buf][1];
      double* A[2];
      double *x[2], *r[2], *b[2];
      for (int spin = 0; spin < 2; ++spin) {
        A[spin] = c.work + (size_t)spin * ((size_t)ld * ld + (size_t)96 * ld);
        x[spin] = A[spin] + (size_t)ld * ld;
        r[spin] = x[spin] + ld;
        b[spin] = r[spin] + ld;
      }
      for (int u = blockIdx.x; u < 2 * n; u += gridDim.x) {
        const int spin = u / n, j = u - spin * n;
        const double emj = c.ev[spin][sv[j] + 2] - 1.0;
        double* Aj = A[spin] + (size_t)j * ld;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          double v = -g0_eval(c, spin, tau[i], site[i], tau[j], site[j]) * emj;
          if (i == j) v += emj + 1.0;
          Aj[i] = v;
        }
      }
      for (int k = gtid; k < 2 * n; k += gthreads) {
        const int spin = k / n, kk = k - spin * n;
        b[spin][kk] = (q.move == MV_INSERT)
                          ? g0_eval(c, spin, tau[kk], site[kk], q.tau_new, q.site_new)
                          : (kk == q.p ? 1.0 : 0.0);
      }
      grid.sync();
      if (q.move == MV_INSERT) {
        grid_gemv_partials2(N0, N1, ld, n, b[0], b[1], slices, ns, gtid, gthreads);
        grid.sync();
        for (int k = gtid; k < 2 * n; k += gthreads) {
          const int spin = k / n, i = k - spin * n;
          x[spin][i] = slice_sum(slices, ld, ns, spin, i);
        }
      } else {
        for (int k = gtid; k < 2 * n; k += gthreads) {
          const int spin = k / n, i = k - spin * n;
          x[spin][i] = (double)c.N[buf][spin][(size_t)q.p * ld + i];
        }
      }
      grid.sync();
      bool conv[2] = {false, false};
      double dprev[2] = {1e300, 1e300};
      for (int it = 0; it < max_iter && !(conv[0] && conv[1]); ++it) {
        grid_gemv_partials2(A[0], A[1], ld, n, x[0], x[1], slices, ns, gtid, gthreads);
        grid.sync();
        for (int k = gtid; k < 2 * n; k += gthreads) {
          const int spin = k / n, i = k - spin * n;
          r[spin][i] = b[spin][i] - slice_sum(slices, ld, ns, spin, i);
        }
        grid.sync();
        grid_gemv_partials2(N0, N1, ld, n, r[0], r[1], slices, ns, gtid, gthreads);
        grid.sync();
        double dmax[2] = {0.0, 0.0}, xmax[2] = {0.0, 0.0};
        for (int k = gtid; k < 2 * n; k += gthreads) {
          const int spin = k / n, i = k - spin * n;
          const double dx = slice_sum(slices, ld, ns, spin, i);
          const double xn = conv[spin] ? x[spin][i] : x[spin][i] + dx;  // converged: frozen
          x[spin][i] = xn;
          dmax[spin] = fmax(dmax[spin], fabs(dx));
          xmax[spin] = fmax(xmax[spin], fabs(xn));
        }
        for (int spin = 0; spin < 2; ++spin) {
          const double bd = block_max(dmax[spin], red);
          const double bx = block_max(xmax[spin], red);
          if (threadIdx.x == 0) {
            part[4 * blockIdx.x + 2 * spin] = bd;
            part[4 * blockIdx.x + 2 * spin + 1] = bx;
          }
        }
        grid.sync();
        for (int spin = 0; spin < 2; ++spin) {
          double dm = 0.0, xm = 0.0;
          for (int k = 0; k < (int)gridDim.x; ++k) {
            dm = fmax(dm, part[4 * k + 2 * spin]);
            xm = fmax(xm, part[4 * k + 2 * spin + 1]);
          }
          // converged at 1e-14, or stagnating at the float64 rounding level
          if (!conv[spin])
            conv[spin] = dm <= 1e-14 * xm || (it >= 2 && dm <= 1e-10 * xm && dm >= 0.5 * dprev[spin]);
          dprev[spin] = dm;
        }
        grid.sync();  // partials are rewritten in the next iteration
      }
      ok = conv[0] && conv[1];
      if (ok) {
        double gpp[2], lam[2];
        if (q.move == MV_INSERT) {
          double v[2] = {0.0, 0.0};
          for (int k = gtid; k < 2 * n; k += gthreads) {
            const int spin = k / n, l = k - spin * n;
            v[spin] += g0_eval(c, spin, q.tau_new, q.site_new, tau[l], site[l]) *
                       (c.ev[spin][sv[l] + 2] - 1.0) * x[spin][l];
          }
          for (int spin = 0; spin < 2; ++spin) {
            const double bs = block_sum(v[spin], red);
            if (threadIdx.x == 0) part[4 * blockIdx.x + spin] = bs;
          }
          grid.sync();
          for (int spin = 0; spin < 2; ++spin) {
            double tot = 0.0;
            for (int k = 0; k < (int)gridDim.x; ++k) tot += part[4 * k + spin];
            gpp[spin] = g0_eval(c, spin, q.tau_new, q.site_new, q.tau_new, q.site_new) + tot;
            lam[spin] = c.ev[spin][q.s_new + 2] - 1.0;
          }
          grid.sync();
        } else {
          const int k = sv[q.p] + 2;
          for (int spin = 0; spin < 2; ++spin) {
            gpp[spin] = (x[spin][q.p] * c.ev[spin][k] - 1.0) * c.inv_em1[spin][k];
            lam[spin] = c.ev[spin][q.s_new - sv[q.p] + 2] - 1.0;
          }
        }
        for (int spin = 0; spin < 2; ++spin) ratio[spin] = 1.0 + lam[spin] * (1.0 - gpp[spin]);
      }
    }
    grid.sync();  // every CTA has read the pending state before it changes
    if (gtid == 0 && ok) set_forced(c, d, q, ratio);
    any_fail = any_fail || !ok;  // the same in every CTA
    grid.sync();
  }
  if (!any_fail) return;
  // fallback for the chains still pending: from-scratch FP64 refresh keeping
  // the FP64 N (N64), its stats, then the decision from N64
  refresh_body<float, double>(chains, n_chains, -1, 1);
  grid.sync();
  for (int ci = gtid; ci < n_chains; ci += gthreads) refresh_finish_one(chains[ci], 1);
  grid.sync();
  for (int ci = blockIdx.x; ci < n_chains; ci += gridDim.x) tie_eval_chain(chains[ci]);
}

cudaError_t launch_tie_refine(Chain<float>* dchains, const LaunchShape& ls, double* part,
                              cudaStream_t st) {
  int nch = ls.n_chains;
  double* slices = part + 4 * (size_t)ls.tie_grid;
  int max_iter = ls.tie_iters;
  void* args[] = {&dchains, &nch, &part, &slices, &max_iter};
  return cudaLaunchCooperativeKernel((const void*)k_tie_refine, dim3(ls.tie_grid), dim3(256), args,
                                     0, st);
}


}  // namespace ctaux
