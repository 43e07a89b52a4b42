// Device-side state and helpers of the CT-AUX submatrix-update path.
//
// Layout in HBM, per chain (all allocated once at init):
//   N[buf][spin]   ld x ld, column-major, T = double (FP64 form) or float (mixed)
//                  double-buffered: a flush reads buffer `buf` and writes the
//                  compacted result into buffer 1-buf.
//   tau/site/s/birth[buf]  configuration, slot order = birth order (Sec. IV)
//   s0             auxiliary spin of each slot at block start
//   Cpan[spin]     k_max x ld row-major   C = G0(new, old) (e^{V_old} - 1)
//   Bpan[spin]     ld x k_max col-major   B = G0(old, new)
//   Gcol[spin]     ld x k_max col-major   columns of G = N_ext G0 for the new vertices
//   Ginv[spin]     k_max x (k_max+1) row-major  Gamma^{-1} (Sec. III D)
//   lam[spin], P   the touched slots of the block and their cumulative lambda
//   S              surviving slots of a flush (compaction list)
//   Y[spin]        ld x k_max col-major   (G - 1)_{S,P} Gamma^{-1}
// The extended matrix of Sec. IV A, N_ext = [[N, 0], [R~, 1]], is stored in
// place: rows/cols [n, m) of N hold R~ and the identity block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ctaux {

constexpr int kMaxK = 256;

enum { MV_INSERT = 0, MV_REMOVE = 1, MV_FLIP = 2 };
enum { DS_CAPACITY = 1, DS_NUMERIC = 2, DS_SINGULAR = 4, DS_TIMEOUT = 8, DS_INDEX = 16 };

struct TraceRec {  // layout of ctaux_trace_rec
  int64_t t;
  int32_t move;
  int32_t n;
  int64_t birth;
  int32_t s_new;
  int32_t accept;
  double ratio[2];
  double R;
  double u;
};

// The block's proposals, drawn once by the plan kernel (Philox counter t0 + j).
struct BlockDraw {
  double u_acc;    // Metropolis uniform
  double u_idx;    // vertex choice of a removal or flip
  int32_t slot;    // insertion: slot of the pre-inserted vertex; else -1
  int8_t move;     // MV_*
  int8_t s_new;    // insertion: proposed auxiliary spin (+1 / -1)
  int16_t pad;
};

struct Dyn {
  int n;        // interacting vertices (slots [0, n) after a flush)
  int m;        // n + k_ins during a block
  int k_ins;    // pre-inserted vertices of the block
  int k_acc;    // |P| at the end of the proposals
  int n_new;    // survivors of the flush
  int buf;      // current N / configuration buffer
  int status;   // DS_* bits
  int sign;     // walker sign
  int64_t t;    // next proposal counter
  int64_t proposals[3], accepted[3];
  int64_t sweeps, measurements, order_sum;
  int64_t meas_bins;       // completed bins of Chain::bin_size measurements
  double sign_sum;
  int64_t numeric_rejects;
  int64_t near_ties;      // mixed form: accept decisions within the guard band
  int64_t refreshes;
  double drift_max, drift_fro;
  double drift_rel;       // drift_max / max |N_fresh| at the last refresh
  int drift_exceeded;     // a refresh saw drift_rel above Chain::drift_limit (not yet reported)
  double logdet[2];
  int64_t trace_written;  // total records written
  int64_t trace_read;     // records handed to the host
  double work_prep;       // algorithmic flops of the prep products (both spins)
  double work_flush;      // algorithmic flops of the flush products
  double bytes_flush;     // algorithmic bytes of the flush (N read + N' written)
  double work_gamma;      // algorithmic flops of the Gamma growth (both spins)
  double work_meas;       // algorithmic flops of the G(tau) estimator (both spins)
  double work_refresh;    // algorithmic flops of the FP64 refreshes (2 m^3 per spin)
  double work_mats;       // algorithmic flops of the Matsubara-frequency measurement
  int flush_noop;         // block left N unchanged (nothing accepted, survivors = [0, n))
  int tie_pending;        // mixed form: 1 = proposal d.t awaits an FP64 decision
  int tie_jj;             // index in the block of the near-tie proposal
  int forced_accept;      // FP64 decision of proposal forced_t
  int64_t forced_t;       // proposal whose decision was taken in FP64 (-1: none)
  int64_t tie_refreshes;  // near ties decided through a from-scratch refresh (refinement failed)
  double forced_ratio[2];
  double forced_R;
  double tie_R32;         // mixed form: float32 R of the pending near tie
  double tie_err_max;     // largest |R_float32 - R_FP64| / |R_FP64| seen at near ties
  double guard_eff;       // the chain's guard band: max(tie_guard, min(0.05, 16 tie_err_max))
};

template <typename T>
struct Chain {
  double beta, K, gamma, dtau, inv_dtau;
  double ev[2][5];           // e^{gamma sigma d}, d = -2..2  (index d + 2)
  double inv_em1[2][5];      // 1 / (e^{gamma sigma d} - 1), d != 0
  T glam[2][5];              // (1 + lambda) / lambda in T, lambda = e^{gamma sigma d} - 1, d != 0
  double p_insert, p_remove;
  int n_c, n_classes, n_tau, k_max, cap_m, ld;
  uint64_t seed;
  uint32_t chain_id;
  int trace_cap;
  int n_bins, n_anchors;
  int kp;                    // mixed form: k_max rounded up to 32 (split operand row length)
  double tie_guard;          // mixed form: relative guard band of the FP64 re-evaluation (0 = off)
  double* N64[2];            // mixed form: FP64 N of a tie refresh [spin], ld x ld
  const double* g0;          // [2][n_classes][n_tau]
  const int* dx_class;       // [n_c][n_c]
  const double* class_weight;  // [n_classes] 1/(n_anchors * #sites of the class)
  T* N[2][2];                // [buf][spin]
  float* NT[2][2];           // mixed form with the tensor-core prep: N^T [buf][spin], ld x ld
  double* tau[2];
  int* site[2];
  int8_t* s[2];
  int64_t* birth[2];
  int8_t* s0;
  T* Cpan[2];
  T* Bpan[2];
  T* Gcol[2];
  T* Ginv[2];                // Gamma^{-1}, row-major, row stride k_max + 1 (inverse form)
  T* Glu[2];                 // L (strictly lower) and U (upper) of Gamma, same layout (LU form)
  int gamma_lu;              // 1: Gamma kept as L U
  double* lam[2];
  int* P;
  int* S;
  BlockDraw* draws;          // [k_max] proposals of the current block
  T* Y[2];
  T* Mg[2];                  // measurement: g_b columns, ld x n_anchors
  T* Mv[2];                  // measurement: v_b = N g_b, ld x n_anchors
  double* Mpts[2];           // measurement: value per (anchor, site, bin)
  float* Yh[2];              // mixed form: split K-major flush operands, rows x kp
  float* Yl[2];
  float* Xh[2];
  float* Xl[2];
  const int8_t* tile_var;    // tile-variant table of the products (tile_table_index)
  T* kpart[2];               // split-K partial tiles
  int* ticket[2];            // split-K arrival counters per output tile
  T* kpart_meas[2];          // the same for the measurement product, which may run beside a block
  int* ticket_meas[2];
  int8_t* s_meas;            // spins of the measured configuration, copied when a measurement starts
  double* work;              // refresh: per spin X (ld x ld), two panels, pivot rows (float64)
  int* perm;                 // refresh pivot rows [spin][ld]
  int8_t* used;              // refresh pivot flags [spin][ld]
  int* pcol;                 // refresh: column at which a row was pivoted, -1 if not [spin][ld]
  unsigned long long* pkeys; // refresh pivot keys [spin][ld]
  double* work_drift;        // refresh: max, sum of squares of the drift, max |N_fresh|
  double drift_limit;        // relative drift that a refresh reports as CTAUX_EDRIFT (0 = off)
  double* work_logdet;       // refresh: [spin]
  double* Gsum;              // [2][n_classes][n_bins] running sums
  double* Gsq;
  double* Gbin;              // sum over the measurements of the open bin
  double* Gbsum;             // sums of completed bin means and of their squares
  double* Gbsq;
  int bin_size;              // measurements per bin of the binned error
  int n_freq;                // Matsubara frequencies of the G(iw) measurement (0 = off)
  double2* G0w;              // [2][n_classes][n_freq] G0(i w_f) of the interpolated table
  int* vorder;               // [ld] vertex slots grouped by site
  int* site_off;             // [n_c + 1] start of each site's group in vorder
  void* PhR;                 // [ld][n_freq] e^{-i w tau} in site order (complex of T)
  void* PhL[2];              // [spin][ld][n_freq] (e^{V} - 1) e^{+i w tau}
  double2* Sw[2];            // [spin][n_c][n_c][n_freq] S_zw
  double2* Tw[2];            // [spin][n_c][n_c][n_freq] S G0
  double* Gw_sum;            // [2][n_c][n_c][n_freq][2] sums of Re, Im of G_xy(i w)
  double* Gw_sq;             // and of their squares
  double* Gmeas;             // last measurement
  TraceRec* trace;
  Dyn* dyn;
};

// ----------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32 -> 64-bit
// products; counter (t_lo, t_hi, chain, purpose), key = seed.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return (double)((((uint64_t)a) << 21) + (uint64_t)(b >> 11)) * 0x1.0p-53;
}

__device__ __forceinline__ void philox_pair(uint64_t seed, uint32_t chain, int64_t t,
                                            uint32_t purpose, double& u0, double& u1) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)((uint64_t)t & 0xffffffffu),
                                           (uint32_t)((uint64_t)t >> 32), chain, purpose),
                                make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)));
  u0 = u53(w.x, w.y);
  u1 = u53(w.z, w.w);
}

struct Draws {
  double u_move, u_acc, u_tau, u_site, u_spin, u_idx;
};

__device__ __forceinline__ Draws draw(uint64_t seed, uint32_t chain, int64_t t) {
  Draws d;
  philox_pair(seed, chain, t, 0u, d.u_move, d.u_acc);
  philox_pair(seed, chain, t, 1u, d.u_tau, d.u_site);
  philox_pair(seed, chain, t, 2u, d.u_spin, d.u_idx);
  return d;
}

__device__ __forceinline__ int move_of(double u_move, double p_insert, double p_remove) {
  if (u_move < p_insert) return MV_INSERT;
  if (u_move < p_insert + p_remove) return MV_REMOVE;
  return MV_FLIP;
}

// ------------------------------------------------------- G0 interpolation
// Linear interpolation of a table row at 0 <= x <= beta; explicit _rn
// operations keep the arithmetic free of FMA contraction.
__device__ __forceinline__ double interp_row(const double* row, int n_tau, double inv_dtau, double x) {
  const double pos = x * inv_dtau;
  const int idx = min(max((int)floor(pos), 0), n_tau - 2);
  const double f = pos - (double)idx;
  const double g0 = __ldg(row + idx), g1 = __ldg(row + idx + 1);
  return fma(f, g1 - g0, g0);
}

// G0_sigma(x_i - x_j, tau_i - tau_j): antiperiodic in tau; equal times take
// G0(0-) = -G0(beta-) (the density convention of Eq. Nmatrix's diagonal).
// Branch-free in the sign of tau_i - tau_j (neighbouring threads of the
// measurement and refresh see both signs).
template <typename T>
__device__ __forceinline__ double g0_eval(const Chain<T>& c, int spin, double ti, int xi, double tj,
                                          int xj) {
  const double dt = ti - tj;
  const int cls = __ldg(c.dx_class + xi * c.n_c + xj);
  const double* row = c.g0 + ((size_t)spin * c.n_classes + cls) * c.n_tau;
  const bool neg = dt < 0.0;
  const double v = interp_row(row, c.n_tau, c.inv_dtau, neg ? dt + c.beta : dt);
  if (dt == 0.0) return -__ldg(row + c.n_tau - 1);
  return neg ? -v : v;
}

// Same interpolation in float32 (the mixed form's measurement): table entries
// rounded to float, position and weights in float.
__device__ __forceinline__ float interp_row_f(const double* row, int n_tau, float inv_dtau, float x) {
  const float pos = x * inv_dtau;
  const int idx = min(max((int)floorf(pos), 0), n_tau - 2);
  const float f = pos - (float)idx;
  const float g0 = (float)__ldg(row + idx), g1 = (float)__ldg(row + idx + 1);
  return fmaf(f, g1 - g0, g0);
}

template <typename T>
__device__ __forceinline__ float g0_eval_f(const Chain<T>& c, int spin, float ti, int xi, float tj,
                                           int xj) {
  const float dt = ti - tj;
  const int cls = __ldg(c.dx_class + xi * c.n_c + xj);
  const double* row = c.g0 + ((size_t)spin * c.n_classes + cls) * c.n_tau;
  const bool neg = dt < 0.f;
  const float v = interp_row_f(row, c.n_tau, (float)c.inv_dtau, neg ? dt + (float)c.beta : dt);
  if (dt == 0.f) return -(float)__ldg(row + c.n_tau - 1);
  return neg ? -v : v;
}

// ------------------------------------------------------------ work lists
// Batched kernels loop over (chain, item) pairs: every CTA computes each
// chain's item count from its device-side sizes, an exclusive prefix sum in
// shared memory (off[0..n_chains], off[n_chains] = total), and finds the chain
// of a linear item index by binary search.
constexpr int kMaxChains = 2048;

__device__ __forceinline__ void block_exclusive_scan(int* a, int n) {
  // a[0..n] in shared memory; on return a[i] = sum_{k<i} a_k, a[n] = total
  __shared__ int part[1024];
  const int nt = blockDim.x, t = threadIdx.x;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += a[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < nt; ++i) {
      const int v = part[i];
      part[i] = run;
      run += v;
    }
    a[n] = run;
  }
  __syncthreads();
  int run = part[t];
  for (int i = lo; i < hi; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
  __syncthreads();
}

__device__ __forceinline__ int find_chain(const int* off, int n, int w) {
  int lo = 0, hi = n;  // off[lo] <= w < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ctaux
