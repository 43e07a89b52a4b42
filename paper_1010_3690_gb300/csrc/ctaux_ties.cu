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
  // the float32 ratio this proposal had against its FP64 value: a sample of
  // the form's ratio error, from which the chain's guard band follows
  // (16 x the largest error seen, at least the configured guard, at most 0.05)
  if (!q.none && finite && fabs(R) > 0.0 && isfinite(d.tie_R32)) {
    const double err = fabs(d.tie_R32 - R) / fabs(R);
    d.tie_err_max = fmax(d.tie_err_max, err);
    d.guard_eff = fmax(c.tie_guard, fmin(0.05, 16.0 * d.tie_err_max));
  }
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


// All chains with a pending tie are refined together, in groups of up to
// kTiePend in increasing chain order (the same in every CTA).  Per chain and
// spin the work area holds A (ld x ld), x, r, b (ld each), the column-slice
// partial sums of the matrix-vector products (kTieSlices x ld) and five
// statistics: two pairs of convergence maxima (|dx|, |x|), used in alternate
// iterations so that one pair is reset while the other is read, and G_pp.
// Work goes to threads or CTAs through prefix sums over the group: "row
// units" (chain, spin, row or column; 2n per chain) and "product units"
// (chain, spin, column slice, row; 2 ns rp per chain, ns column slices that
// depend only on the chain's order, rp = n rounded up to 32).  Reductions are
// maxima (atomicMax on non-negative values) or sums in a fixed order, so the
// results do not depend on timing.
constexpr int kTiePend = 64;
static_assert(3 * kPB >= kTieSlices + 4, "tie work area exceeds the refresh work area");

struct TieWork {
  double *A, *x, *r, *b, *P, *st;
};

__device__ __forceinline__ TieWork tie_work(const Chain<float>& c, int spin) {
  const int ld = c.ld;
  TieWork w;
  w.A = c.work + (size_t)spin * refresh_work_per_spin(ld);
  w.x = w.A + (size_t)ld * ld;
  w.r = w.x + ld;
  w.b = w.r + ld;
  w.P = w.b + ld;
  w.st = w.P + (size_t)kTieSlices * ld;
  return w;
}

__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
  // non-negative doubles order like their bit patterns
  if (v != 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(256) k_tie_refine(Chain<float>* chains, int n_chains, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gthreads = gridDim.x * blockDim.x;
  __shared__ unsigned pend[kMaxChains / 32];  // chains with a pending tie, as bits
  __shared__ int gl[kTiePend];                // chain of each group member
  __shared__ int offr[kTiePend + 1];          // prefix of 2 n
  __shared__ int offg[kTiePend + 1];          // prefix of 2 ns rp
  __shared__ int nn_s[kTiePend], ns_s[kTiePend];
  __shared__ TieProposal q_s[kTiePend];
  __shared__ unsigned char conv_s[kTiePend][2];
  __shared__ double dprev_s[kTiePend][2];
  __shared__ int g_s, all_s, fail_s;
  const int nwords = (n_chains + 31) / 32;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) pend[w] = 0u;
  if (threadIdx.x == 0) fail_s = 0;
  __syncthreads();
  // every CTA reads the same flags: they change only after the first grid barrier
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
    const Dyn& d = *chains[ci].dyn;
    if (!d.status && d.tie_pending == 1) atomicOr(&pend[ci >> 5], 1u << (ci & 31));
  }
  int wd = 0;
  unsigned bits = 0u;
  bool first = true;
  for (;;) {
    // ---- next group of pending chains, in chain order
    __syncthreads();
    if (threadIdx.x == 0) {
      if (first && nwords > 0) bits = pend[0];
      first = false;
      int g = 0;
      while (g < kTiePend) {
        while (!bits && wd + 1 < nwords) bits = pend[++wd];
        if (!bits) break;
        gl[g++] = wd * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
      }
      g_s = g;
    }
    __syncthreads();
    const int G = g_s;
    if (G == 0) break;
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
      const Chain<float>& c = chains[gl[i]];
      const int n = c.dyn->n;
      const TieProposal q = tie_proposal(c, *c.dyn);
      const bool work = !q.none && max_iter > 0;
      q_s[i] = q;
      nn_s[i] = n;
      ns_s[i] = max(1, min(kTieSlices, gthreads / (2 * ((n + 31) & ~31))));
      conv_s[i][0] = conv_s[i][1] = work ? 0 : 1;
      dprev_s[i][0] = dprev_s[i][1] = 1e300;
      offr[i + 1] = work ? 2 * n : 0;
      offg[i + 1] = work ? 2 * ns_s[i] * ((n + 31) & ~31) : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      offr[0] = offg[0] = 0;
      for (int i = 0; i < G; ++i) {
        offr[i + 1] += offr[i];
        offg[i + 1] += offg[i];
      }
    }
    __syncthreads();
    const int tot_r = offr[G], tot_g = offg[G];

    // ---- A_s = N^{-1} (Eq. Nmatrix), one column per CTA step
    for (int u = blockIdx.x; u < tot_r; u += gridDim.x) {
      const int i = find_chain(offr, G, u);
      const Chain<float>& c = chains[gl[i]];
      const int n = nn_s[i], l = u - offr[i], spin = l / n, j = l - spin * n, buf = c.dyn->buf;
      const double* tau = c.tau[buf];
      const int* site = c.site[buf];
      const double emj = c.ev[spin][c.s[buf][j] + 2] - 1.0;
      double* Aj = tie_work(c, spin).A + (size_t)j * c.ld;
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double v = -g0_eval(c, spin, tau[r], site[r], tau[j], site[j]) * emj;
        if (r == j) v += emj + 1.0;
        Aj[r] = v;
      }
    }
    // ---- right-hand sides: G0 column of the new vertex (insertion, Eq. Rins)
    // or e_p (removal, flip: x is then column p of N); the start x is N b
    for (int u = gtid; u < tot_r; u += gthreads) {
      const int i = find_chain(offr, G, u);
      const Chain<float>& c = chains[gl[i]];
      const TieProposal& q = q_s[i];
      const int n = nn_s[i], l = u - offr[i], spin = l / n, k = l - spin * n, buf = c.dyn->buf;
      const TieWork w = tie_work(c, spin);
      if (q.move == MV_INSERT) {
        w.b[k] = g0_eval(c, spin, c.tau[buf][k], c.site[buf][k], q.tau_new, q.site_new);
        w.r[k] = w.b[k];
      } else {
        w.b[k] = k == q.p ? 1.0 : 0.0;
        w.x[k] = (double)c.N[buf][spin][(size_t)q.p * c.ld + k];
      }
      if (k == 0)
        for (int e = 0; e < 5; ++e) w.st[e] = 0.0;
    }
    grid.sync();
    // partial sums over column slices of A x (a_matrix) or N r
    auto products = [&](bool a_matrix, bool insert_only) {
      for (int u = gtid; u < tot_g; u += gthreads) {
        const int i = find_chain(offg, G, u);
        const Chain<float>& c = chains[gl[i]];
        const int n = nn_s[i], ns = ns_s[i], rp = (n + 31) & ~31, ld = c.ld;
        const int l = u - offg[i], spin = l / (ns * rp), l2 = l - spin * ns * rp;
        const int sl = l2 / rp, row = l2 - sl * rp;
        if (row >= n || conv_s[i][spin] || (insert_only && q_s[i].move != MV_INSERT)) continue;
        const TieWork w = tie_work(c, spin);
        const int j0 = (int)((long long)sl * n / ns), j1 = (int)((long long)(sl + 1) * n / ns);
        double a0 = 0.0, a1 = 0.0;
        int j = j0;
        if (a_matrix) {
          for (; j + 1 < j1; j += 2) {
            a0 += w.A[(size_t)j * ld + row] * w.x[j];
            a1 += w.A[(size_t)(j + 1) * ld + row] * w.x[j + 1];
          }
          if (j < j1) a0 += w.A[(size_t)j * ld + row] * w.x[j];
        } else {
          const float* N = c.N[c.dyn->buf][spin];
          for (; j + 1 < j1; j += 2) {
            a0 += (double)N[(size_t)j * ld + row] * w.r[j];
            a1 += (double)N[(size_t)(j + 1) * ld + row] * w.r[j + 1];
          }
          if (j < j1) a0 += (double)N[(size_t)j * ld + row] * w.r[j];
        }
        w.P[(size_t)sl * ld + row] = a0 + a1;
      }
    };
    // slice partials of a row, added in slice order
    auto slice_total = [&](const TieWork& w, int ld, int ns, int k) {
      double t = 0.0;
      for (int sl = 0; sl < ns; ++sl) t += w.P[(size_t)sl * ld + k];
      return t;
    };
    products(false, true);
    grid.sync();
    for (int u = gtid; u < tot_r; u += gthreads) {
      const int i = find_chain(offr, G, u);
      if (q_s[i].move != MV_INSERT) continue;
      const Chain<float>& c = chains[gl[i]];
      const int n = nn_s[i], l = u - offr[i], spin = l / n, k = l - spin * n;
      const TieWork w = tie_work(c, spin);
      w.x[k] = slice_total(w, c.ld, ns_s[i], k);
    }
    grid.sync();
    // ---- x <- x + N (b - A x) until every member has converged
    for (int it = 0; it < max_iter; ++it) {
      const int pr = 2 * (it & 1);  // statistics pair of this iteration
      __syncthreads();
      if (threadIdx.x == 0) {
        int all = 1;
        for (int i = 0; i < G; ++i) all &= conv_s[i][0] & conv_s[i][1];
        all_s = all;
      }
      __syncthreads();
      if (all_s) break;
      products(true, false);
      grid.sync();
      for (int u = gtid; u < tot_r; u += gthreads) {
        const int i = find_chain(offr, G, u);
        const Chain<float>& c = chains[gl[i]];
        const int n = nn_s[i], l = u - offr[i], spin = l / n, k = l - spin * n;
        const TieWork w = tie_work(c, spin);
        // the other pair was read by every CTA before the last barrier
        if (k == 0) w.st[2 - pr] = w.st[3 - pr] = 0.0;
        if (conv_s[i][spin]) continue;
        w.r[k] = w.b[k] - slice_total(w, c.ld, ns_s[i], k);
      }
      grid.sync();
      products(false, false);
      grid.sync();
      for (int u = gtid; u < tot_r; u += gthreads) {
        const int i = find_chain(offr, G, u);
        const Chain<float>& c = chains[gl[i]];
        const int n = nn_s[i], l = u - offr[i], spin = l / n, k = l - spin * n;
        if (conv_s[i][spin]) continue;
        const TieWork w = tie_work(c, spin);
        const double dx = slice_total(w, c.ld, ns_s[i], k);
        const double xn = w.x[k] + dx;
        w.x[k] = xn;
        atomic_max_nonneg(&w.st[pr], fabs(dx));
        atomic_max_nonneg(&w.st[pr + 1], fabs(xn));
      }
      grid.sync();
      for (int u = threadIdx.x; u < 2 * G; u += blockDim.x) {
        const int i = u >> 1, spin = u & 1;
        if (conv_s[i][spin]) continue;
        const TieWork w = tie_work(chains[gl[i]], spin);
        const double dm = w.st[pr], xm = w.st[pr + 1];
        // converged at 1e-14, or stagnating at the float64 rounding level
        if (dm <= 1e-14 * xm || (it >= 2 && dm <= 1e-10 * xm && dm >= 0.5 * dprev_s[i][spin]))
          conv_s[i][spin] = 1;
        dprev_s[i][spin] = dm;
      }
    }
    // ---- insertion: G_pp = G0(p,p) + sum_l G0(p,l)(e^{V_l}-1) x_l (Eq. Rins);
    // the terms go to r, one warp per (chain, spin) adds them in a fixed order
    for (int u = gtid; u < tot_r; u += gthreads) {
      const int i = find_chain(offr, G, u);
      const TieProposal& q = q_s[i];
      if (q.move != MV_INSERT) continue;
      const Chain<float>& c = chains[gl[i]];
      const int n = nn_s[i], l = u - offr[i], spin = l / n, k = l - spin * n, buf = c.dyn->buf;
      const TieWork w = tie_work(c, spin);
      w.r[k] = g0_eval(c, spin, q.tau_new, q.site_new, c.tau[buf][k], c.site[buf][k]) *
               (c.ev[spin][c.s[buf][k] + 2] - 1.0) * w.x[k];
    }
    grid.sync();
    {
      const int wg = gtid >> 5, lane = threadIdx.x & 31;
      for (int u = wg; u < 2 * G; u += gthreads >> 5) {
        const int i = u >> 1, spin = u & 1;
        const TieProposal& q = q_s[i];
        if (q.none || max_iter <= 0 || q.move != MV_INSERT) continue;
        const TieWork w = tie_work(chains[gl[i]], spin);
        double v = 0.0;
        for (int k = lane; k < nn_s[i]; k += 32) v += w.r[k];
        v = warp_sum(v);
        if (lane == 0) w.st[4] = v;
      }
    }
    grid.sync();
    for (int i = gtid; i < G; i += gthreads) {
      const Chain<float>& c = chains[gl[i]];
      Dyn& d = *c.dyn;
      const TieProposal& q = q_s[i];
      if (!(q.none || (max_iter > 0 && conv_s[i][0] && conv_s[i][1]))) continue;
      double ratio[2] = {0.0, 0.0};
      if (!q.none) {
        for (int spin = 0; spin < 2; ++spin) {
          const TieWork w = tie_work(c, spin);
          double gpp, lam;
          if (q.move == MV_INSERT) {
            gpp = g0_eval(c, spin, q.tau_new, q.site_new, q.tau_new, q.site_new) + w.st[4];
            lam = c.ev[spin][q.s_new + 2] - 1.0;
          } else {
            const int k = c.s[d.buf][q.p] + 2;
            gpp = (w.x[q.p] * c.ev[spin][k] - 1.0) * c.inv_em1[spin][k];
            lam = c.ev[spin][q.s_new - c.s[d.buf][q.p] + 2] - 1.0;
          }
          ratio[spin] = 1.0 + lam * (1.0 - gpp);
        }
      }
      set_forced(c, d, q, ratio);
    }
    if (threadIdx.x == 0)
      for (int i = 0; i < G; ++i)
        if (!(q_s[i].none || (max_iter > 0 && conv_s[i][0] && conv_s[i][1]))) fail_s = 1;
    grid.sync();
  }
  if (!fail_s) return;
  // fallback for the chains still pending: from-scratch FP64 refresh keeping
  // the FP64 N (N64), its stats, then the decision from N64
  refresh_body<float, double>(chains, n_chains, -1, 1);
  grid.sync();
  for (int ci = gtid; ci < n_chains; ci += gthreads) refresh_finish_one(chains[ci], 1);
  grid.sync();
  for (int ci = blockIdx.x; ci < n_chains; ci += gridDim.x) tie_eval_chain(chains[ci]);
}

cudaError_t launch_tie_refine(Chain<float>* dchains, const LaunchShape& ls, cudaStream_t st) {
  int nch = ls.n_chains;
  int max_iter = ls.tie_iters;
  void* args[] = {&dchains, &nch, &max_iter};
  return cudaLaunchCooperativeKernel((const void*)k_tie_refine, dim3(ls.tie_grid), dim3(256), args,
                                     0, st);
}

}  // namespace ctaux
