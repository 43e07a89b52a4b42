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


// y = M v over the whole grid, M column-major with leading dimension ld:
// slice sl of the columns writes its partial sums to P[sl*ld + i]; the caller
// adds the ns partials in slice order after a grid barrier (deterministic).
template <typename Tm>
__device__ __forceinline__ void grid_gemv_partials(const Tm* M, int ld, int n, const double* v,
                                                   double* P, int ns, int gtid, int gthreads) {
  const int rp = (n + 31) & ~31;
  for (int idx = gtid; idx < ns * rp; idx += gthreads) {
    const int i = idx % rp, sl = idx / rp;
    if (i >= n) continue;
    const int j0 = (int)((long long)sl * n / ns), j1 = (int)((long long)(sl + 1) * n / ns);
    double a0 = 0.0, a1 = 0.0;
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      a0 += (double)M[(size_t)j * ld + i] * v[j];
      a1 += (double)M[(size_t)(j + 1) * ld + i] * v[j + 1];
    }
    if (j < j1) a0 += (double)M[(size_t)j * ld + i] * v[j];
    P[(size_t)sl * ld + i] = a0 + a1;
  }
}

__device__ __forceinline__ double slice_sum(const double* P, int ld, int ns, int i) {
  double t = 0.0;
  for (int sl = 0; sl < ns; ++sl) t += P[(size_t)sl * ld + i];
  return t;
}

// Cooperative over the whole GPU, one pending tie at a time: A (FP64) is
// built once across all CTAs, then x <- x + N (b - A x) iterates; each
// matrix-vector product is split over column slices, and the convergence
// maxima go through per-CTA partials read in CTA order.
__global__ void __launch_bounds__(256) k_tie_refine(Chain<float>* chains, int n_chains,
                                                    double* part, double* slices, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  __shared__ double red[8];
  bool any_fail = false;
  for (int ci = 0; ci < n_chains; ++ci) {
    const Chain<float>& c = chains[ci];
    Dyn& d = *c.dyn;
    if (d.status || d.tie_pending != 1) continue;  // same decision in every CTA
    const TieProposal q = tie_proposal(c, d);
    const int n = d.n, buf = d.buf, ld = c.ld;
    const int ns = max(1, min(kTieSlices, gthreads / ((n + 31) & ~31)));
    const double* tau = c.tau[buf];
    const int* site = c.site[buf];
    const int8_t* sv = c.s[buf];
    double ratio[2] = {0.0, 0.0};
    bool ok = max_iter > 0;
    for (int spin = 0; spin < 2 && !q.none && ok; ++spin) {
      const float* N = c.N[buf][spin];
      double* A = c.work + (size_t)spin * ((size_t)ld * ld + (size_t)96 * ld);
      double* x = A + (size_t)ld * ld;
      double* r = x + ld;
      double* b = r + ld;
      for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const double emj = c.ev[spin][sv[j] + 2] - 1.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          double v = -g0_eval(c, spin, tau[i], site[i], tau[j], site[j]) * emj;
          if (i == j) v += emj + 1.0;
          A[(size_t)j * ld + i] = v;
        }
      }
      for (int k = gtid; k < n; k += gthreads)
        b[k] = (q.move == MV_INSERT) ? g0_eval(c, spin, tau[k], site[k], q.tau_new, q.site_new)
                                     : (k == q.p ? 1.0 : 0.0);
      grid.sync();
      if (q.move == MV_INSERT) {
        grid_gemv_partials(N, ld, n, b, slices, ns, gtid, gthreads);
        grid.sync();
        for (int i = gtid; i < n; i += gthreads) x[i] = slice_sum(slices, ld, ns, i);
      } else {
        for (int i = gtid; i < n; i += gthreads) x[i] = (double)N[(size_t)q.p * ld + i];
      }
      grid.sync();
      bool conv = false;
      double dprev = 1e300;
      for (int it = 0; it < max_iter && !conv; ++it) {
        grid_gemv_partials(A, ld, n, x, slices, ns, gtid, gthreads);
        grid.sync();
        for (int i = gtid; i < n; i += gthreads) r[i] = b[i] - slice_sum(slices, ld, ns, i);
        grid.sync();
        grid_gemv_partials(N, ld, n, r, slices, ns, gtid, gthreads);
        grid.sync();
        double dmax = 0.0, xmax = 0.0;
        for (int i = gtid; i < n; i += gthreads) {
          const double dx = slice_sum(slices, ld, ns, i);
          const double xn = x[i] + dx;
          x[i] = xn;
          dmax = fmax(dmax, fabs(dx));
          xmax = fmax(xmax, fabs(xn));
        }
        const double bd = block_max(dmax, red);
        const double bx = block_max(xmax, red);
        if (threadIdx.x == 0) {
          part[2 * blockIdx.x] = bd;
          part[2 * blockIdx.x + 1] = bx;
        }
        grid.sync();
        double dm = 0.0, xm = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) {
          dm = fmax(dm, part[2 * k]);
          xm = fmax(xm, part[2 * k + 1]);
        }
        // converged at 1e-14, or stagnating at the float64 rounding level
        conv = dm <= 1e-14 * xm || (it >= 2 && dm <= 1e-10 * xm && dm >= 0.5 * dprev);
        dprev = dm;
        grid.sync();  // partials are rewritten in the next iteration
      }
      if (!conv) {
        ok = false;
        break;
      }
      double gpp, lam;
      if (q.move == MV_INSERT) {
        double v = 0.0;
        for (int l = gtid; l < n; l += gthreads)
          v += g0_eval(c, spin, q.tau_new, q.site_new, tau[l], site[l]) * (c.ev[spin][sv[l] + 2] - 1.0) * x[l];
        const double bs = block_sum(v, red);
        if (threadIdx.x == 0) part[blockIdx.x] = bs;
        grid.sync();
        double tot = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) tot += part[k];
        gpp = g0_eval(c, spin, q.tau_new, q.site_new, q.tau_new, q.site_new) + tot;
        lam = c.ev[spin][q.s_new + 2] - 1.0;
        grid.sync();
      } else {
        const int k = sv[q.p] + 2;
        gpp = (x[q.p] * c.ev[spin][k] - 1.0) * c.inv_em1[spin][k];
        lam = c.ev[spin][q.s_new - sv[q.p] + 2] - 1.0;
      }
      ratio[spin] = 1.0 + lam * (1.0 - gpp);
    }
    grid.sync();  // every CTA has read the pending state before it changes
    if (gtid == 0 && ok) set_forced(c, d, q, ratio);
    any_fail = any_fail || !ok;  // the same in every CTA
    grid.sync();
  }
  if (!any_fail) return;
  // fallback for the chains still pending: from-scratch FP64 refresh keeping
  // the FP64 N (N64), its stats, then the decision from N64
  refresh_body<float>(chains, n_chains, -1, 1);
  grid.sync();
  for (int ci = gtid; ci < n_chains; ci += gthreads) refresh_finish_one(chains[ci], 1);
  grid.sync();
  for (int ci = blockIdx.x; ci < n_chains; ci += gridDim.x) tie_eval_chain(chains[ci]);
}

cudaError_t launch_tie_refine(Chain<float>* dchains, const LaunchShape& ls, double* part,
                              cudaStream_t st) {
  int nch = ls.n_chains;
  double* slices = part + 2 * (size_t)ls.tie_grid;
  int max_iter = ls.tie_iters;
  void* args[] = {&dchains, &nch, &part, &slices, &max_iter};
  return cudaLaunchCooperativeKernel((const void*)k_tie_refine, dim3(ls.tie_grid), dim3(256), args,
                                     0, st);
}


}  // namespace ctaux
