// Measurement directly in Matsubara frequencies (Sec. IV D: for large
// clusters G is measured directly in cluster momenta and Matsubara
// frequencies), after a flush, on every chain.
//
// The estimator is the Fourier transform (1/beta) int int dtau dtau'
// e^{i w (tau - tau')} of the G(tau) estimator G(a,b) = G0(a,b) +
// sum_lm G0(a,l) M_lm G0(m,b), M = (e^V - 1) N (the row of an s=0 vertex of
// the extended N of Sec. IV A contracted with G0).  G0(x - x_l, tau - tau_l)
// transforms to G0_{x x_l}(iw) e^{i w tau_l}, so
//   G_xy(iw) = G0_xy(iw) + (1/beta) sum_zw G0_xz(iw) S_zw(iw) G0_wy(iw),
//   S_zw(iw) = sum_{l on site z, m on site w} e^{i w tau_l} M_lm e^{-i w tau_m},
// w = (2f + 1) pi / beta.  G0(iw) is the transform of the same linearly
// interpolated table the weights use, integrated exactly.  Cluster momenta
// follow by G(K) = (1/N_c) sum_xy e^{-iK.(r_x - r_y)} G_xy.
//
// Steps per measurement: vertices grouped by site (k_mats_order), phase
// factors per vertex and frequency (k_mats_phase), S_zw for every site pair
// and frequency (k_mats_S, O(n^2 F): the dominant part), then the two N_c x
// N_c complex products and the accumulation (k_mats_G).
#include <math.h>

#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"

namespace ctaux {

template <typename T>
struct CplxOf;
template <>
struct CplxOf<double> {
  using type = double2;
};
template <>
struct CplxOf<float> {
  using type = float2;
};

__device__ __forceinline__ double mats_w(int f, double beta) {
  return (2.0 * f + 1.0) * 3.14159265358979323846 / beta;
}

// G0_sigma,class(i w_f) = int_0^beta e^{i w tau} g(tau) dtau of the linear
// interpolant g of the table row, integrated by parts (e^{i w beta} = -1):
//   -(g(beta-) + g(0+)) / (i w) + sum_j s_j (e^{i w t_{j+1}} - e^{i w t_j}) / w^2,
// s_j the slope of interval j.  One thread per (spin, class, f).
__global__ void k_g0_matsubara(const double* table, int n_classes, int n_tau, double beta,
                               int n_freq, double2* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * n_classes * n_freq) return;
  const int f = e % n_freq, row = e / n_freq;  // row = spin * n_classes + class
  const double* g = table + (size_t)row * n_tau;
  const double w = mats_w(f, beta), h = beta / (double)(n_tau - 1);
  double re = 0.0, im = 0.0;
  double c0 = 1.0, s0 = 0.0;
  for (int j = 0; j + 1 < n_tau; ++j) {
    double s1, c1;
    sincos(w * (double)(j + 1) * h, &s1, &c1);
    const double slope = (g[j + 1] - g[j]) / h;
    re += slope * (c1 - c0);
    im += slope * (s1 - s0);
    c0 = c1;
    s0 = s1;
  }
  const double iw2 = 1.0 / (w * w);
  re *= iw2;
  im *= iw2;
  // -(g(beta-) + g(0+)) / (i w) = i (g(beta-) + g(0+)) / w
  im += (g[n_tau - 1] + g[0]) / w;
  out[e] = make_double2(re, im);
}

// Vertex slots grouped by site (within a site in slot order): warp-level
// ballots over the configuration, one CTA per chain.
template <typename T>
__global__ void __launch_bounds__(1024) k_mats_order(Chain<T>* chains) {
  const Chain<T>& c = chains[blockIdx.x];
  const Dyn& d = *c.dyn;
  if (d.status || c.n_freq == 0) return;
  const int n = d.n, nc = c.n_c;
  const int* site = c.site[d.buf];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int cnt[kMaxMatsSites + 1];
  for (int z = warp; z < nc; z += nw) {
    int k = 0;
    for (int l0 = 0; l0 < n; l0 += 32) {
      const int l = l0 + lane;
      k += __popc(__ballot_sync(0xffffffffu, l < n && __ldg(site + l) == z));
    }
    if (lane == 0) cnt[z] = k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int z = 0; z < nc; ++z) {
      const int v = cnt[z];
      cnt[z] = run;
      c.site_off[z] = run;
      run += v;
    }
    cnt[nc] = run;
    c.site_off[nc] = run;
  }
  __syncthreads();
  for (int z = warp; z < nc; z += nw) {
    int pos = cnt[z];
    for (int l0 = 0; l0 < n; l0 += 32) {
      const int l = l0 + lane;
      const bool mine = l < n && __ldg(site + l) == z;
      const unsigned b = __ballot_sync(0xffffffffu, mine);
      if (mine) c.vorder[pos + __popc(b & ((1u << lane) - 1u))] = l;
      pos += __popc(b);
    }
  }
}

// Phase factors in site order p: PhR[p][f] = e^{-i w_f tau}, and per spin
// PhL[spin][p][f] = (e^{V_sigma} - 1) e^{+i w_f tau} (the row scaling of M).
// Evaluated in float64 and stored in the form's type.
template <typename T>
__global__ void __launch_bounds__(256) k_mats_phase(Chain<T>* chains) {
  using C2 = typename CplxOf<T>::type;
  const Chain<T>& c = chains[blockIdx.y];
  const Dyn& d = *c.dyn;
  if (d.status || c.n_freq == 0) return;
  const int n = d.n, F = c.n_freq, buf = d.buf;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)n * F;
       e += (long)gridDim.x * blockDim.x) {
    const int p = (int)(e / F), f = (int)(e % F);
    const int l = c.vorder[p];
    double sn, cs;
    sincos(mats_w(f, c.beta) * c.tau[buf][l], &sn, &cs);
    const int si = c.s_meas[l] + 2;
    static_cast<C2*>(c.PhR)[e] = C2{(T)cs, (T)(-sn)};
    const double e0 = c.ev[0][si] - 1.0, e1 = c.ev[1][si] - 1.0;
    static_cast<C2*>(c.PhL[0])[e] = C2{(T)(e0 * cs), (T)(e0 * sn)};
    static_cast<C2*>(c.PhL[1])[e] = C2{(T)(e1 * cs), (T)(e1 * sn)};
  }
}

// S_zw(f) for every (chain, spin, z, w): persistent over the items of all
// chains.  A thread owns one (vertex row l of site z, frequency f) pair of an
// l-chunk of min(64, 256/F) rows; the columns m of site w stream through
// shared memory in chunks of at most kMatsMc (the block N[l][m] and the phases
// e^{-i w tau_m}, at most kMatsPh of them):
//   acc(l, f) = sum_m N[l][m] e^{-i w_f tau_m},  s(f) += PhL[l][f] acc(l, f),
// then the rows' partial sums are added in a fixed order (deterministic).
constexpr int kMatsMc = 32, kMatsRows = 64, kMatsPh = 512;

template <typename T>
__device__ __forceinline__ int mats_items(const Chain<T>& c, const Dyn& d) {
  if (d.status || c.n_freq == 0 || d.n == 0) return 0;
  return 2 * c.n_c * c.n_c;
}

template <typename T>
__global__ void __launch_bounds__(256) k_mats_S(Chain<T>* chains, int n_chains) {
  using C2 = typename CplxOf<T>::type;
  __shared__ int off[kMaxChains + 1];
  __shared__ T Ns[kMatsMc][kMatsRows + 1];  // [m][row in the l-chunk]
  __shared__ C2 Ph[kMatsPh];                // e^{-i w tau_m}, [m][f]
  __shared__ double2 red[256];
  __shared__ int rows_s[kMatsRows], cols_s[kMatsMc];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x)
    off[ci] = mats_items(chains[ci], *chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int ci = find_chain(off, n_chains, it);
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    const int nc = c.n_c, F = c.n_freq, ld = c.ld;
    const int l_item = it - off[ci];
    const int spin = l_item / (nc * nc), zw = l_item % (nc * nc), z = zw / nc, w = zw % nc;
    const int oz = c.site_off[z], nz = c.site_off[z + 1] - oz;
    const int ow = c.site_off[w], nw = c.site_off[w + 1] - ow;
    const T* Nb = c.N[d.buf][spin];
    const C2* PhL = static_cast<const C2*>(c.PhL[spin]);
    const C2* PhR = static_cast<const C2*>(c.PhR);
    const int LC = min(kMatsRows, 256 / F);  // rows per l-chunk
    const int MC = min(kMatsMc, kMatsPh / F);  // columns per m-chunk
    const int f = threadIdx.x % F, li = threadIdx.x / F;
    const bool active = li < LC;
    double sr = 0.0, si = 0.0;               // s(f) over this thread's rows
    for (int l0 = 0; l0 < nz; l0 += LC) {
      const int lc = min(LC, nz - l0);
      __syncthreads();
      if (threadIdx.x < lc) rows_s[threadIdx.x] = c.vorder[oz + l0 + threadIdx.x];
      T ar = (T)0, ai = (T)0;
      for (int m0 = 0; m0 < nw; m0 += MC) {
        const int mc = min(MC, nw - m0);
        __syncthreads();
        if (threadIdx.x < mc) cols_s[threadIdx.x] = c.vorder[ow + m0 + threadIdx.x];
        for (int e = threadIdx.x; e < mc * F; e += blockDim.x)
          Ph[e] = PhR[(size_t)(ow + m0) * F + e];
        __syncthreads();
        // N block: column m (contiguous rows of N), rows of site z (gathered)
        for (int e = threadIdx.x; e < mc * lc; e += blockDim.x) {
          const int mm = e / lc, rr = e % lc;
          Ns[mm][rr] = Nb[(size_t)cols_s[mm] * ld + rows_s[rr]];
        }
        __syncthreads();
        if (active && li < lc) {
          for (int mm = 0; mm < mc; ++mm) {
            const T nv = Ns[mm][li];
            const C2 ph = Ph[mm * F + f];
            ar += nv * ph.x;
            ai += nv * ph.y;
          }
        }
      }
      if (active && li < lc) {
        const C2 pl = PhL[(size_t)(oz + l0 + li) * F + f];
        const double a_r = (double)ar, a_i = (double)ai;
        sr += (double)pl.x * a_r - (double)pl.y * a_i;
        si += (double)pl.x * a_i + (double)pl.y * a_r;
      }
    }
    __syncthreads();
    red[threadIdx.x] = make_double2(active ? sr : 0.0, active ? si : 0.0);
    __syncthreads();
    if (threadIdx.x < F) {
      double r = 0.0, i = 0.0;
      for (int q = 0; q < LC; ++q) {
        r += red[q * F + threadIdx.x].x;
        i += red[q * F + threadIdx.x].y;
      }
      c.Sw[spin][((size_t)z * nc + w) * F + threadIdx.x] = make_double2(r, i);
    }
  }
}

// The two N_c x N_c complex products per (chain, spin, f), one output row per
// item, and the accumulation:
//   stage 0: Tw[z][y] = sum_w S_zw G0_wy
//   stage 1: G_xy = G0_xy + (1/beta) sum_z G0_xz Tw[z][y]; sums of Re, Im and
//            of their squares.
// G0_xy(f) = G0w[spin][class(x, y)][f].
template <typename T>
__device__ __forceinline__ int mats_g_items(const Chain<T>& c, const Dyn& d) {
  if (d.status || c.n_freq == 0) return 0;
  return 2 * c.n_freq * c.n_c;
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(256) k_mats_G(Chain<T>* chains, int n_chains) {
  __shared__ int off[kMaxChains + 1];
  for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x)
    off[ci] = mats_g_items(chains[ci], *chains[ci].dyn);
  __syncthreads();
  block_exclusive_scan(off, n_chains);
  const int total = off[n_chains];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int ci = find_chain(off, n_chains, it);
    const Chain<T>& c = chains[ci];
    const Dyn& d = *c.dyn;
    const int nc = c.n_c, F = c.n_freq;
    const int l_item = it - off[ci];
    const int spin = l_item / (F * nc), r = l_item % (F * nc), f = r / nc, row = r % nc;
    const double2* G0w = c.G0w + (size_t)spin * c.n_classes * F;
    const bool empty = d.n == 0;
    for (int y = threadIdx.x; y < nc; y += blockDim.x) {
      double re = 0.0, im = 0.0;
      if (!empty) {
        for (int k = 0; k < nc; ++k) {
          double2 a, b;
          if (STAGE == 0) {
            a = c.Sw[spin][((size_t)row * nc + k) * F + f];
            b = G0w[(size_t)__ldg(c.dx_class + k * nc + y) * F + f];
          } else {
            a = G0w[(size_t)__ldg(c.dx_class + row * nc + k) * F + f];
            b = c.Tw[spin][((size_t)k * nc + y) * F + f];
          }
          re += a.x * b.x - a.y * b.y;
          im += a.x * b.y + a.y * b.x;
        }
      }
      if (STAGE == 0) {
        c.Tw[spin][((size_t)row * nc + y) * F + f] = make_double2(re, im);
      } else {
        const double2 g0 = G0w[(size_t)__ldg(c.dx_class + row * nc + y) * F + f];
        const double gr = g0.x + re / c.beta, gi = g0.y + im / c.beta;
        const size_t o = ((((size_t)spin * nc + row) * nc + y) * F + f) * 2;
        c.Gw_sum[o] += gr;
        c.Gw_sum[o + 1] += gi;
        c.Gw_sq[o] += gr * gr;
        c.Gw_sq[o + 1] += gi * gi;
      }
    }
  }
  if (STAGE == 1 && blockIdx.x == 0) {
    // algorithmic flops, both spins: S (a real N times complex phases, 4 n^2 F,
    // and the row phases, 8 n F) and the two complex N_c x N_c products (16 N_c^3 F)
    for (int ci = threadIdx.x; ci < n_chains; ci += blockDim.x) {
      const Chain<T>& c = chains[ci];
      Dyn& d = *c.dyn;
      if (!d.status && c.n_freq > 0) {
        const double n = d.n, F = c.n_freq, nc = c.n_c;
        d.work_mats += 2.0 * (4.0 * n * n * F + 8.0 * n * F + 16.0 * nc * nc * nc * F);
      }
    }
  }
}

template <typename T>
void launch_matsubara(Chain<T>* dchains, const LaunchShape& ls, cudaStream_t st) {
  const int nch = ls.n_chains;
  k_mats_order<T><<<nch, 1024, 0, st>>>(dchains);
  k_mats_phase<T><<<dim3(ls.gather_slices, nch), 256, 0, st>>>(dchains);
  k_mats_S<T><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
  k_mats_G<T, 0><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
  k_mats_G<T, 1><<<ls.persist_ctas, 256, 0, st>>>(dchains, nch);
}

void launch_g0_matsubara(const double* table, int n_classes, int n_tau, double beta, int n_freq,
                         double2* out, cudaStream_t st) {
  const int total = 2 * n_classes * n_freq;
  k_g0_matsubara<<<(total + 127) / 128, 128, 0, st>>>(table, n_classes, n_tau, beta, n_freq, out);
}

template void launch_matsubara<double>(Chain<double>*, const LaunchShape&, cudaStream_t);
template void launch_matsubara<float>(Chain<float>*, const LaunchShape&, cudaStream_t);

}  // namespace ctaux
