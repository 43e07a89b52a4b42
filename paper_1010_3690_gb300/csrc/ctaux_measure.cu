// G(tau) measurement (Sec. IV D) after a flush, on every chain.
//
// Estimator for external points a = (x_a, tau_a), b = (x_b, tau_b) (both s=0):
//   G(a, b) = G0(a, b) + sum_{l,m} G0(a, l) [(e^V - 1) N]_{lm} G0(m, b),
// the row of an s=0 vertex of N_ext (Sec. IV A) contracted with G = N G0.
// Anchors b = (site 0, j beta / n_anchors); a = (x_a, tau_b + tau_c) with
// tau_c the centre of a bin on (0, beta), folded into [0, beta) with the
// antiperiodic sign.  G_sigma(class(x_a), bin) is the average over anchors
// and over the sites of a class.
//
// Steps: gather g_b[m] = G0(m, b) (k_meas_gather), v_b = N g_b (batched GEMM,
// split over K), evaluate every point (k_meas_eval), reduce per class in a
// fixed order and accumulate sums and squares (k_meas_accumulate).
#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"

namespace ctaux {

template <typename T>
__global__ void __launch_bounds__(256) k_meas_gather(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.z];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const int spin = blockIdx.y, n = d.n, buf = d.buf, A = c.n_anchors;
  if (blockIdx.x == 0 && spin == 0 && threadIdx.x == 0) {
    // counters of this measurement (read by the accumulation kernel that follows)
    d.measurements += 1;
    d.order_sum += n;
    d.sign_sum += (double)d.sign;
    // both spins: v_b = N g_b (2 n^2 per anchor) and the contraction with
    // G0(a, l) (2 flops per point, vertex and anchor)
    const double nd = (double)n;
    d.work_meas += 2.0 * (2.0 * nd * nd * A + 2.0 * A * (double)c.n_c * c.n_bins * nd);
  }
  // the spins of the measured configuration: the next block's proposals may
  // change them while the rest of the measurement runs
  if (spin == 0)
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
      c.s_meas[v] = c.s[buf][v];
  const long total = (long)n * A;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int m = (int)(e % n), b = (int)(e / n);
    const double tb = (double)b * c.beta / (double)A;
    c.Mg[spin][(long)b * c.ld + m] = (T)g0_eval(c, spin, c.tau[buf][m], c.site[buf][m], tb, 0);
  }
}

// Evaluation of the estimator, persistent over the (chain, spin, point block,
// vertex chunk) items of all chains; partial sums over a chunk of meas_chunk(n)
// vertices go to Mpts[spin][chunk][(anchor * N_c + site) * B + bin].
//
// When the number of bins B is a multiple of the number of anchors A, every
// evaluation time tau_b + tau_c (folded into [0, beta)) is one of the B points
// tau_p = (p + 1/2) beta / B, shifted by B/A points per anchor.  A thread then
// owns a (site, tau_p) point, interpolates G0(a, l) once per vertex l and
// accumulates it for all A anchors (anchor b reads bin (p - b B/A) mod B, with
// the antiperiodic sign when the fold wrapped).  Otherwise a thread owns one
// (anchor, site, bin) point.
constexpr int kMaxSharedAnchors = 16;

template <typename T>
__device__ __forceinline__ bool meas_shared(const Chain<T>& c) {
  return c.n_anchors <= kMaxSharedAnchors && (c.n_bins % c.n_anchors) == 0;
}

template <typename T>
__device__ __forceinline__ int meas_points(const Chain<T>& c) {
  return (meas_shared(c) ? 1 : c.n_anchors) * c.n_c * c.n_bins;
}

template <typename T>
__device__ __forceinline__ int meas_items(const Chain<T>& c, const Dyn& d) {
  if (d.status) return 0;
  return 2 * ((meas_points(c) + 255) / 256) * max(1, (d.n + meas_chunk(d.n) - 1) / meas_chunk(d.n));
}

// Per-chunk vertex data staged in shared memory by every CTA of an item:
// tau_q, site_q and w_b(q) = (e^{V_q} - 1) v_b(q) for the anchors.
template <typename A>
struct MeasStage {
  double tau[kMeasChunkMax];
  int site[kMeasChunkMax];
  A w[kMaxSharedAnchors][kMeasChunkMax];
};

// Shared-anchor evaluation of one (site, tau_p) point over the staged chunk,
// NA anchors known at compile time.
template <int NA, typename T>
__device__ __forceinline__ void meas_point_shared(const Chain<T>& c, int spin, int xa, double tp,
                                                  int nq, const MeasStage<T>& st, double* acc) {
  if (sizeof(T) == 8) {
    double a[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) a[b] = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double g = g0_eval(c, spin, tp, xa, st.tau[q], st.site[q]);
#pragma unroll
      for (int b = 0; b < NA; ++b) a[b] = fma(g, (double)st.w[b][q], a[b]);
    }
#pragma unroll
    for (int b = 0; b < NA; ++b) acc[b] = a[b];
  } else {  // mixed form: float32 interpolation and products
    float a[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) a[b] = 0.f;
    const float tpf = (float)tp;
    for (int q = 0; q < nq; ++q) {
      const float g = g0_eval_f(c, spin, tpf, xa, (float)st.tau[q], st.site[q]);
#pragma unroll
      for (int b = 0; b < NA; ++b) a[b] = fmaf(g, (float)st.w[b][q], a[b]);
    }
#pragma unroll
    for (int b = 0; b < NA; ++b) acc[b] = (double)a[b];
  }
}

template <typename T>
__device__ __forceinline__ void meas_point_shared_n(int na, const Chain<T>& c, int spin, int xa,
                                                    double tp, int nq, const MeasStage<T>& st,
                                                    double* acc) {
  switch (na) {
    case 1: meas_point_shared<1>(c, spin, xa, tp, nq, st, acc); break;
    case 2: meas_point_shared<2>(c, spin, xa, tp, nq, st, acc); break;
    case 3: meas_point_shared<3>(c, spin, xa, tp, nq, st, acc); break;
    case 4: meas_point_shared<4>(c, spin, xa, tp, nq, st, acc); break;
    case 5: case 6: meas_point_shared<6>(c, spin, xa, tp, nq, st, acc); break;
    case 7: case 8: meas_point_shared<8>(c, spin, xa, tp, nq, st, acc); break;
    default: meas_point_shared<kMaxSharedAnchors>(c, spin, xa, tp, nq, st, acc); break;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_meas_eval(Chain<T>* chains, int n_chains) {
  __shared__ int off[kMaxChains + 1];
  __shared__ MeasStage<T> st;
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x)
    off[ci] = meas_items(chains[ci], *chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int ci = find_chain(off, n_chains, w);
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    const int n = d.n, buf = d.buf, A = c.n_anchors, B = c.n_bins;
    const int npts_out = A * c.n_c * B;
    const int npts = meas_points(c);
    const int chl = meas_chunk(n);
    const int pblocks = (npts + 255) / 256, nchunks = max(1, (n + chl - 1) / chl);
    const int l = w - off[ci];
    const int spin = l / (pblocks * nchunks), r0 = l % (pblocks * nchunks);
    const int chunk = r0 / pblocks;
    const int l0 = chunk * chl, l1 = min(n, l0 + chl);
    const int nq = max(0, l1 - l0);
    const int pt = (r0 % pblocks) * blockDim.x + threadIdx.x;
    const bool shared = meas_shared(c);
    __syncthreads();  // the previous item's readers are done with the stage
    if (shared) {
      for (int e = threadIdx.x; e < nq * (A + 1); e += blockDim.x) {
        const int q = e % nq, b = e / nq, v = l0 + q;
        if (b == A) {
          st.tau[q] = c.tau[buf][v];
          st.site[q] = c.site[buf][v];
        } else {
          const double em1 = c.ev[spin][c.s_meas[v] + 2] - 1.0;
          st.w[b][q] = (T)(em1 * (double)c.Mv[spin][(long)b * c.ld + v]);
        }
      }
    }
    __syncthreads();
    if (pt >= npts) continue;
    double* out = c.Mpts[spin] + (size_t)chunk * npts_out;
    if (shared) {
      const int p = pt % B, xa = pt / B, shift = B / A;
      const double tp = ((double)p + 0.5) * c.beta / (double)B;
      double acc[kMaxSharedAnchors];
      meas_point_shared_n(A, c, spin, xa, tp, nq, st, acc);
      for (int b = 0; b < A; ++b) {
        const int i = (p - b * shift + B) % B;
        const double sg = (p < b * shift) ? -1.0 : 1.0;
        double val = acc[b];
        if (chunk == 0) val += g0_eval(c, spin, tp, xa, (double)b * c.beta / (double)A, 0);
        out[((size_t)b * c.n_c + xa) * B + i] = sg * val;
      }
      continue;
    }
    const double* tau = c.tau[buf];
    const int* site = c.site[buf];
    const int8_t* s = c.s_meas;
    const int bin = pt % B, xa = (pt / B) % c.n_c, b = pt / (B * c.n_c);
    const double tb = (double)b * c.beta / (double)A;
    const double tc = ((double)bin + 0.5) * c.beta / (double)B;
    double ta = tb + tc, sg = 1.0;
    if (ta >= c.beta) {
      ta -= c.beta;
      sg = -1.0;
    }
    double val = (chunk == 0) ? g0_eval(c, spin, ta, xa, tb, 0) : 0.0;
    const T* V = c.Mv[spin] + (long)b * c.ld;  // v_b = N g_b
    if (sizeof(T) == 8) {
      for (int q = l0; q < l1; ++q) {
        const double vl = (c.ev[spin][s[q] + 2] - 1.0) * (double)V[q];
        val += g0_eval(c, spin, ta, xa, tau[q], site[q]) * vl;
      }
    } else {  // mixed form: float32 interpolation and products
      float accf = 0.f;
      const float taf = (float)ta;
      for (int q = l0; q < l1; ++q) {
        const float vl = ((float)c.ev[spin][s[q] + 2] - 1.f) * (float)V[q];
        accf += g0_eval_f(c, spin, taf, xa, (float)tau[q], site[q]) * vl;
      }
      val += (double)accf;
    }
    out[pt] = sg * val;
  }
}

// Per (chain, spin, class, bin), one warp: the partial sums over vertex
// chunks, anchors and the sites of the class are split over the lanes in a
// fixed pattern and combined by a fixed shuffle tree (deterministic).  Besides
// the running sums, consecutive measurements are grouped in bins of
// Chain::bin_size; each completed bin adds its mean and the mean's square to
// the bin accumulators (error bars of correlated Markov-chain samples).
template <typename T>
__global__ void k_meas_accumulate(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.z];
  Dyn& d = *c.dyn;
  if (d.status) return;
  const bool closes_bin = (d.measurements % c.bin_size) == 0;  // counted by k_meas_gather
  const int spin = blockIdx.y, A = c.n_anchors, B = c.n_bins, nc = c.n_c;
  const int npts = A * nc * B;
  const int nchunks = max(1, (d.n + meas_chunk(d.n) - 1) / meas_chunk(d.n));
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // output of this warp
  if (e < c.n_classes * B) {
    const int cls = e / B, bin = e % B;
    const double* Mp = c.Mpts[spin];
    double acc = 0.0;
    // only the sites of this class (a warp-uniform test), lanes over the chunks
    for (int xa = 0; xa < nc; ++xa) {
      if (c.dx_class[xa * nc] != cls) continue;
      for (int b = 0; b < A; ++b) {
        const double* src = Mp + (size_t)(b * nc + xa) * B + bin;
        for (int q = lane; q < nchunks; q += 32) acc += src[(size_t)q * npts];
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      acc *= c.class_weight[cls];
      const long o = ((long)spin * c.n_classes + cls) * B + bin;
      c.Gmeas[o] = acc;
      c.Gsum[o] += acc;
      c.Gsq[o] += acc * acc;
      const double open = c.Gbin[o] + acc;
      if (closes_bin) {
        const double mean = open / (double)c.bin_size;
        c.Gbsum[o] += mean;
        c.Gbsq[o] += mean * mean;
        c.Gbin[o] = 0.0;
      } else {
        c.Gbin[o] = open;
      }
    }
  }
  if (closes_bin && blockIdx.x == 0 && threadIdx.x == 0 && spin == 0) d.meas_bins += 1;
}

template <typename T>
__global__ void k_meas_reset(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 2 * c.n_classes * c.n_bins) {
    c.Gsum[e] = 0.0;
    c.Gsq[e] = 0.0;
    c.Gmeas[e] = 0.0;
    c.Gbin[e] = 0.0;
    c.Gbsum[e] = 0.0;
    c.Gbsq[e] = 0.0;
  }
  const long nw = (long)4 * c.n_c * c.n_c * c.n_freq;
  for (long q = e; q < nw; q += (long)gridDim.x * blockDim.x) {
    c.Gw_sum[q] = 0.0;
    c.Gw_sq[q] = 0.0;
  }
  if (e == 0) {
    c.dyn->measurements = 0;
    c.dyn->meas_bins = 0;
    c.dyn->order_sum = 0;
    c.dyn->sign_sum = 0.0;
  }
}

template <typename T>
int launch_measure_head(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st) {
  k_meas_gather<T><<<dim3(ls.gather_slices, 2, ls.n_chains), 256, 0, st>>>(dchains);
  return 1;
}

template <typename T>
int launch_measure_tail(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st) {
  const int nch = ls.n_chains;
  const int ng = launch_gemm<T>(dchains, ls, PH_MEAS, st);
  k_meas_eval<T><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
  k_meas_accumulate<T><<<dim3(ls.meas_acc_blocks, 2, nch), 256, 0, st>>>(dchains);
  if (ls.mats) launch_matsubara<T>(dchains, ls, st);
  return 2 + ng + (ls.mats ? 5 : 0);
}

template <typename T>
void launch_measure(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st, PhaseTimer* pt) {
  pt->begin(5, st);
  const int nk = launch_measure_head<T>(dchains, ls, st);
  pt->end(5, st, nk + launch_measure_tail<T>(dchains, ls, st));
}

template <typename T>
void launch_reset_measure(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st) {
  k_meas_reset<T><<<dim3(ls.meas_cb_blocks * 2, ls.n_chains), 256, 0, st>>>(dchains);
}

template void launch_measure<double>(Chain<double>*, const LaunchShape&, cudaStream_t, PhaseTimer*);
template int launch_measure_head<double>(Chain<double>*, const LaunchShape&, cudaStream_t);
template int launch_measure_head<float>(Chain<float>*, const LaunchShape&, cudaStream_t);
template int launch_measure_tail<double>(Chain<double>*, const LaunchShape&, cudaStream_t);
template int launch_measure_tail<float>(Chain<float>*, const LaunchShape&, cudaStream_t);
template void launch_measure<float>(Chain<float>*, const LaunchShape&, cudaStream_t, PhaseTimer*);
template void launch_reset_measure<double>(Chain<double>*, const LaunchShape&, cudaStream_t);
template void launch_reset_measure<float>(Chain<float>*, const LaunchShape&, cudaStream_t);

}  // namespace ctaux
