/*
 * ctaux.h -- C ABI of the GB300 submatrix-update CT-AUX hot path.
 *
 * What the library computes (Gull et al., "Submatrix updates for the
 * Continuous-Time Auxiliary Field algorithm"):
 *   - Markov chains over auxiliary-spin configurations {(tau_i, x_i, s_i)} with
 *     weight prod_sigma det N_sigma^{-1}, N_sigma^{-1} = e^{V_sigma} - G0_sigma
 *     (e^{V_sigma} - 1)  (Sec. II A, Eqs. Zn_div_Z0 and Nmatrix);
 *   - insertion/removal/spin-flip proposals accepted with min(1, |R|)
 *     (Sec. II B, Eq. insprob);
 *   - executed as the submatrix update of Secs. III-IV: k_max s=0 vertices are
 *     pre-inserted (Sec. IV A), each proposal grows a k x k Gamma^{-1} per spin
 *     by partitioning (Sec. III D, Eq. ratS), and after k_max proposals N is
 *     updated by the Woodbury formula (Eq. Nshermanmorrison) and the s=0 rows
 *     and columns are removed (Sec. IV C);
 *   - plus a periodic from-scratch FP64 recomputation of N and the G(tau)
 *     measurement of Sec. IV D.
 *
 * Conventions shared by every entry point:
 *   - All pointers are HOST pointers unless a name says otherwise.  Input
 *     arrays are copied before the call returns; the caller keeps ownership.
 *     Output arrays are caller-owned and written synchronously.
 *   - The library allocates all device memory it needs in ctaux_init
 *     (cudaMalloc) and frees it in ctaux_destroy.
 *   - Errors are returned as ctaux_status; nothing aborts or traps.  A device
 *     side fault flag (capacity exceeded, non-finite ratio) is reported by the
 *     next synchronous call; ctaux_last_error() gives a text for the last
 *     failure of a context.
 *   - One context must be used from one host thread at a time.
 *   - Spin index: 0 = up (sigma = +1), 1 = down (sigma = -1).  Matrices are
 *     column-major.
 */
#ifndef CTAUX_H
#define CTAUX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctaux_ctx ctaux_ctx;

typedef enum {
  CTAUX_OK = 0,
  CTAUX_EINVAL = 1,     /* bad argument */
  CTAUX_ENOMEM = 2,     /* device allocation failed */
  CTAUX_ECUDA = 3,      /* CUDA runtime error (text in ctaux_last_error) */
  CTAUX_ECAPACITY = 4,  /* expansion order + k_max exceeded the capacity */
  CTAUX_ESINGULAR = 5,  /* zero pivot in the from-scratch recomputation */
  CTAUX_EDRIFT = 6,     /* drift above the threshold at a recomputation */
  CTAUX_ETIMEOUT = 7,   /* a bounded device-side wait gave up */
  CTAUX_ENUMERIC = 8    /* non-finite determinant ratio (proposal rejected) */
} ctaux_status;

/* Precision forms. */
enum {
  CTAUX_FP64 = 0,       /* N, Gamma^{-1}, all products in float64 */
  CTAUX_MIXED = 1       /* N, Gamma^{-1} in float32; FP64 refresh and near-tie accepts */
};

/* How a block keeps Gamma (Sec. III D). */
enum {
  CTAUX_GAMMA_INVERSE = 0,  /* Gamma^{-1} grown by partitioning (Eq. ratS) */
  CTAUX_GAMMA_LU = 1        /* Gamma = L U grown by bordering (triangular solves per proposal,
                               Eqs. lineq1-detrat); a slot changed twice re-factorises by
                               Bennett's rank-one update; the flush takes Gamma^{-1}
                               formed from L U after the block's proposals */
};

/* Move types (trace records). */
enum { CTAUX_INSERT = 0, CTAUX_REMOVE = 1, CTAUX_FLIP = 2 };

/* One Markov chain's model and run parameters. */
typedef struct {
  int n_c;                  /* cluster sites N_c (1 = single impurity) */
  int n_classes;            /* displacement classes = rows of the table per spin */
  int n_tau;                /* table points on [0, beta], both ends included, >= 2 */
  const double *g0_table;   /* [2][n_classes][n_tau]: G0_sigma(class, j*beta/(n_tau-1)),
                               sign G0 = -<T d d^dagger>; j=0 holds G0(0+), j=n_tau-1 G0(beta-) */
  const int *dx_class;      /* [n_c][n_c]: class of the displacement x_i - x_j */
  double beta;              /* inverse temperature */
  double U;                 /* Hubbard interaction, > 0 (at U = 0 every lambda vanishes and
                               the ratio formulas of Eq. ratS divide by zero) */
  double K;                 /* expansion constant (Eq. gamma), > 0 */
  int k_max;                /* proposals per submatrix block, 1..256 */
  int capacity;             /* largest expansion order n the chain may reach */
  uint64_t seed;            /* Philox-4x32-10 key */
  uint32_t chain_id;        /* third Philox counter word */
} ctaux_chain_params;

typedef struct {
  int n_chains;                       /* 1..2048 independent chains */
  const ctaux_chain_params *chains;   /* [n_chains] */
  int precision;                      /* CTAUX_FP64 or CTAUX_MIXED */
  int refresh_every;                  /* from-scratch N every this many blocks; 0 = never */
  double p_insert;                    /* move mix: insert / flip; remove = 1 - both */
  double p_flip;
  int n_tau_bins;                     /* G(tau) measurement bins on (0, beta) */
  int n_anchors;                      /* anchor times of the G(tau) estimator */
  int trace_capacity;                 /* per-chain trace ring size; 0 = no trace */
  int device;                         /* CUDA device ordinal */
  int mixed_flush_tc;                 /* mixed form: 1 = flush on the tensor cores (tcgen05,
                                         split 3xTF32), 0 = float32 CUDA-core product */
  double tie_guard;                   /* mixed form: the decision u < |R| of a proposal with
                                         |u - |R|| below tie_guard * max(u, |R|), i.e. one that
                                         a relative error of |R| below tie_guard could change,
                                         is taken in FP64 (the block stops there; FP64
                                         iterative refinement of the first-touch ratio, or a
                                         from-scratch FP64 refresh where it does not converge).
                                         Each chain widens its band to 16x the largest float32
                                         ratio error that its FP64 near-tie decisions have
                                         shown (at most 0.05; ctaux_stats.tie_guard_eff);
                                         0 = off; must be < 1 */
  int tie_refine_iters;               /* mixed form: most refinement iterations per near tie;
                                         0 = 12; -1 = none, so that every near tie takes the
                                         from-scratch fallback (for tests) */
  int use_graph;                      /* 1 = each block (with its near-tie launch) and each
                                         measurement is launched as one CUDA graph, captured
                                         on a private stream at first use; direct launches
                                         while profiling is on, or if capture fails */
  int refresh_df64;                   /* mixed form: 1 = the periodic from-scratch recomputation
                                         eliminates in double-float arithmetic (two float32,
                                         about 48 significand bits) on the float32 pipe, which
                                         GB300 runs 64x faster than float64; 0 = float64.  The
                                         matrix N^{-1} is built in float64 either way, and the
                                         near-tie fallback always eliminates in float64 */
  int meas_bin_size;                  /* measurements per bin of the binned error of
                                         ctaux_measure_G; 0 = 16 */
  int n_matsubara;                    /* 0 = off; 1..64: every measurement also evaluates
                                         G_xy(i w_n) at the first n_matsubara fermionic
                                         Matsubara frequencies (ctaux_measure_G_matsubara);
                                         needs n_c <= 1024 */
  double drift_limit;                 /* > 0: a from-scratch recomputation whose drift
                                         max |N_run - N_fresh| / max |N_fresh| exceeds it makes
                                         the next synchronous call return CTAUX_EDRIFT once (the
                                         chain continues from the fresh N); 0 = off */
  int mixed_prep_tc;                  /* mixed form with mixed_flush_tc: 1 = the two large prep
                                         products (rows of the extended N and G columns of the
                                         new vertices over the old ones, Sec. IV A) on the tensor
                                         cores, split 3xTF32; the flush step and the refresh then
                                         also keep N^T; 0 = float32 CUDA-core products.  Needs
                                         capacity + k_max > 96 */
  int tc_wait_limit;                  /* mixed form, tensor-core flush: most polls of one
                                         pipeline wait before the kernel stops with
                                         CTAUX_ETIMEOUT; 0 = 2^24 (seconds).  A negative value
                                         is a test of that path: the MMA issuer first waits
                                         -tc_wait_limit polls on a barrier that nothing
                                         completes, so every flush reports CTAUX_ETIMEOUT */
  int gamma_form;                     /* CTAUX_GAMMA_INVERSE (0) or CTAUX_GAMMA_LU (1); the
                                         same Markov chain either way (ratios equal up to
                                         rounding) */
} ctaux_params;

typedef struct {
  int64_t n;                 /* current expansion order */
  int64_t t;                 /* next proposal counter */
  int64_t proposals[3];      /* by move type */
  int64_t accepted[3];
  int64_t sweeps;            /* completed blocks (prep + k_max proposals + flush) */
  int64_t measurements;
  int64_t order_sum;         /* sum of n over measurements */
  double sign_sum;           /* sum of the walker sign over measurements */
  int64_t numeric_rejects;   /* proposals rejected for a non-finite ratio */
  int64_t near_ties;         /* mixed form: decisions within the guard band (tie_guard, or 1e-4
                                when the FP64 re-evaluation is off) */
  int64_t tie_refreshes;     /* near ties decided through a from-scratch FP64 refresh because
                                the iterative refinement did not converge */
  int64_t refreshes;
  double last_drift_max;     /* max |N_run - N_fresh| at the last refresh (both spins) */
  double last_drift_fro;     /* Frobenius norm of the same difference */
  double last_drift_rel;     /* last_drift_max / max |N_fresh| */
  double logdet[2];          /* log|det N_sigma^{-1}| at the last refresh */
  int sign;                  /* current walker sign */
  int status;                /* device fault bits (0 = none) */
  double tie_err_max;        /* mixed form: largest relative error of a float32 R against its
                                FP64 value, over the near ties decided in FP64 */
  double tie_guard_eff;      /* mixed form: the chain's guard band now, max(tie_guard,
                                min(0.05, 16 tie_err_max)): it widens when a near tie shows a
                                float32 ratio error above 1/16 of it */
} ctaux_stats;

typedef struct {
  int64_t t;                 /* proposal counter */
  int32_t move;              /* CTAUX_INSERT / REMOVE / FLIP */
  int32_t n;                 /* order before the proposal */
  int64_t birth;             /* birth stamp (insertion counter) of the vertex; -1 if none */
  int32_t s_new;             /* proposed auxiliary spin */
  int32_t accept;            /* bit 0: accepted; bit 1: decided in FP64 (mixed form near tie) */
  double ratio[2];           /* det N'^{-1}_sigma / det N^{-1}_sigma per spin */
  double R;                  /* full Metropolis ratio */
  double u;                  /* accept uniform */
} ctaux_trace_rec;

/* Create a context: copies the tables, allocates device state for every
 * chain (N double-buffered at (capacity + k_max)^2 per spin), starts every
 * chain from the empty configuration at counter 0.  *out is NULL on error. */
ctaux_status ctaux_init(const ctaux_params *params, ctaux_ctx **out);

/* Run n_sweeps blocks on every chain, asynchronously on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  One block = pre-insertion
 * of the block's insertion candidates (s = 0), the G0 gather and prep
 * products (Sec. IV A), k_max proposals with Gamma growth (Secs. III D, IV B),
 * the Woodbury flush with compaction (Sec. IV C), then, if `measure` is
 * non-zero, one G(tau) measurement (Sec. IV D), and every refresh_every
 * blocks a from-scratch FP64 recomputation of N.  With use_graph, a block's
 * measurement runs on a second stream beside the next block, and the last
 * block's measurement is launched by the next call that reads or changes the
 * context (another ctaux_sweep, ctaux_synchronize, ctaux_measure_G, ...), on
 * the stream of this call; the results equal the serial order bit for bit. */
ctaux_status ctaux_sweep(ctaux_ctx *ctx, int n_sweeps, int measure, void *cuda_stream);

/* G(tau) measurement of one chain (Sec. IV D; the estimator is the row of an
 * s=0 vertex of the extended N of Sec. IV A contracted with G0, averaged over
 * anchor times and the sites of each displacement class).  Mean of
 * G_sigma(class, tau bin) over the measurements since the last reset, arrays
 * [2][n_classes][n_tau_bins], and its standard error: the spread of the means of
 * completed bins of meas_bin_size consecutive measurements once two bins are
 * complete (Markov-chain samples are correlated), before that the naive error
 * of single measurements.  err_out and n_meas_out may be NULL.  Synchronises the
 * context's stream. */
ctaux_status ctaux_measure_G(ctaux_ctx *ctx, int chain, double *G_out, double *err_out,
                             int64_t *n_meas_out);

/* Measurement directly in Matsubara frequencies (Sec. IV D: for large clusters
 * the Green's function is measured directly in cluster momenta and Matsubara
 * frequencies).  The estimator is the Fourier transform of the G(tau)
 * estimator,
 *   G_xy(i w_n) = G0_xy(i w_n) + (1/beta) sum_{z,w} G0_xz(i w_n) S_zw G0_wy(i w_n),
 *   S_zw = sum_{l on site z, m on site w} e^{i w_n tau_l} [(e^V - 1) N]_lm e^{-i w_n tau_m},
 * w_n = (2n + 1) pi / beta, n = 0 .. n_matsubara - 1, with G0(i w_n) the exact
 * transform of the linearly interpolated table; cluster momenta follow by
 * G(K) = (1/N_c) sum_xy e^{-iK.(r_x - r_y)} G_xy.  Mean over the measurements
 * since the last reset, G_out[2][n_c][n_c][n_matsubara][2] (real, imaginary;
 * host, caller-owned) and the naive standard error of each part (err_out, may
 * be NULL).  CTAUX_EINVAL if the context was created with n_matsubara = 0.
 * Synchronises the context's stream. */
ctaux_status ctaux_measure_G_matsubara(ctaux_ctx *ctx, int chain, double *G_out, double *err_out,
                                       int64_t *n_meas_out);

/* Raw measurement accumulators of one chain, for merging chains or ranks:
 * running sums of the per-measurement G estimates and of their squares, sums of
 * the completed bin means and of their squares (arrays [2][n_classes][n_tau_bins],
 * host, caller-owned, any may be NULL) and counts_out[3] = {measurements,
 * completed bins, bin size} (may be NULL).  Pooled over chains or ranks by plain
 * sums, the mean is sum/measurements and the binned error follows from the bin
 * sums as in ctaux_measure_G.  Synchronises the context's stream. */
ctaux_status ctaux_get_accumulators(ctaux_ctx *ctx, int chain, double *sum_out, double *sumsq_out,
                                    double *bin_sum_out, double *bin_sumsq_out,
                                    int64_t *counts_out);

/* Zero every chain's measurement accumulators (asynchronous). */
ctaux_status ctaux_reset_measurements(ctaux_ctx *ctx);

/* FP64 from-scratch recomputation of N for every chain (build N^{-1} from the
 * configuration, Gauss-Jordan inversion with partial pivoting); returns the
 * largest max-abs drift |N_run - N_fresh| over chains and spins.  Synchronous. */
ctaux_status ctaux_recompute(ctaux_ctx *ctx, double *drift_max_out);

/* Counters of one chain (synchronous). */
ctaux_status ctaux_get_stats(ctaux_ctx *ctx, int chain, ctaux_stats *out);

/* The trace records written since the previous call (oldest first, at most
 * trace_capacity are kept); *n_out records are written to buf[0..cap). */
ctaux_status ctaux_get_trace(ctaux_ctx *ctx, int chain, ctaux_trace_rec *buf, int cap,
                             int *n_out);

/* Configuration checkpoint of one chain in birth order: tau, site, spin,
 * birth stamp (arrays of at least `cap` entries), order and next counter. */
ctaux_status ctaux_get_config(ctaux_ctx *ctx, int chain, double *tau, int *site, int *s,
                              int64_t *birth, int cap, int *n_out, int64_t *t_out);

/* Replace one chain's configuration (sorted by birth stamp inside) and
 * counter, then rebuild its N from scratch in FP64.  s must be +-1. */
ctaux_status ctaux_set_config(ctaux_ctx *ctx, int chain, const double *tau, const int *site,
                              const int *s, const int64_t *birth, int n, int64_t t);

/* Copy N_sigma of one chain (m x m, m = current order) into out[j*ld_out + i],
 * converted to float64; *m_out = m. */
ctaux_status ctaux_get_N(ctaux_ctx *ctx, int chain, int spin, double *out, int ld_out,
                         int *m_out);

/* Per-phase device time, accumulated with CUDA events recorded on the sweep
 * stream while profiling is on, and the number of kernels launched per phase
 * (always counted).  Phases: 0 plan + G0 gather, 1 prep products,
 * 2 proposals (Gamma growth), 3 flush product, 4 flush support (survivor
 * list, Y = (G-1) Gamma^{-1}, end of block), 5 measurement, 6 FP64 refresh
 * (periodic, and the fallback of a near-tie decision), 7 near-tie FP64
 * refinement (mixed form).  ms_out[8], kernels_out[8]; either may be NULL. */
ctaux_status ctaux_set_profiling(ctaux_ctx *ctx, int on);
ctaux_status ctaux_get_phase_times(ctaux_ctx *ctx, double *ms_out, int64_t *kernels_out);

/* Algorithmic work of the blocks run so far, summed over chains (for
 * rooflines): flop counts of the prep products, the flush products and the
 * Gamma growth (both spins), bytes of N read and written by the flush, flops
 * of the G(tau) estimator (the products v_b = N g_b and the contraction with
 * G0(a, l); the table interpolations are not counted) and of the FP64
 * refreshes (2 m^3 per spin and refresh), and of the Matsubara-frequency
 * measurement (4 n^2 F for S, 16 N_c^3 F for the two cluster products, per
 * spin).  Any output may be NULL. */
ctaux_status ctaux_get_work(ctaux_ctx *ctx, double *prep_flop, double *flush_flop,
                            double *flush_bytes, double *gamma_flop, double *meas_flop,
                            double *refresh_flop, double *mats_flop);

/* Change the submatrix size of one chain between sweeps: 1 <= k_max <= the
 * chain's k_max at ctaux_init (its buffers are sized for that).  The Markov
 * chain does not depend on k_max (every draw is keyed by the proposal
 * counter), so this changes only the speed.  Synchronizes the last stream. */
ctaux_status ctaux_set_kmax(ctaux_ctx *ctx, int chain, int k_max);

/* Autotune the submatrix size k_max per chain (the paper finds the optimum
 * k = 64-128 empirically, Sec. V A, and has no tuner).
 * Chains are grouped by (cluster size, octave of the current order).  Each
 * trial sets the k of every group, runs one untimed block and then n_blocks
 * timed blocks (CUDA events, no measurement, no refresh), and scores
 * proposals per second of the whole context.  First the best common k among
 * candidates[n_candidates] is taken, then each group's k is varied in turn
 * (most populated group first), and a change is kept only if it gains more than 2 %.
 * A candidate above a chain's k_max at init is capped to it.  The trials are
 * real Markov-chain steps (the chains advance); a from-scratch refresh ends
 * the tuning.  k_out[n_chains] (may be NULL) receives the chosen k per chain,
 * *rate_out (may be NULL) the best score.  Synchronous. */
ctaux_status ctaux_autotune_k(ctaux_ctx *ctx, const int *candidates, int n_candidates,
                              int n_blocks, int *k_out, double *rate_out);

/* Tile shapes of the CUDA-core products (the prep products, the flush of the
 * FP64 form, the measurement product).  Each product has CTAUX_TILE_VARIANTS
 * compiled output-tile shapes; a table of one byte per (product, octave of the
 * chain's current order n, octave of its k_max),
 *   index = (product * 16 + min(floor(log2 n), 15)) * 9 + min(floor(log2 k_max), 8),
 * products 0 R~, 1 G_{old,new}, 2 G_{new,new}, 3 flush, 4 measurement, picks the
 * shape each chain uses (the table is read on the device for every chain's
 * current order, so chains of different sizes in one launch use different
 * shapes).  A new context starts with all zeros (the default shapes).
 * ctaux_autotune_tiles times the variants on the context's own chains: per
 * product first one variant for every table slot, then the slots holding at
 * least a tenth of the chains (at most four, most populated first) one by one,
 * keeping a change only if it makes the product's time per algorithmic flop
 * more than 2 % lower; each trial is one untimed and n_blocks timed blocks
 * (CUDA events, direct launches, no refresh), real Markov-chain steps; a
 * from-scratch refresh ends it.  table_out (may be NULL) receives the table,
 * *gain_out (may be NULL) the summed time per flop of the default shapes over
 * that of the chosen ones.  ctaux_get_tile_table / ctaux_set_tile_table move a
 * table between contexts (a cache of tuned shapes).  Synchronous. */
#define CTAUX_TILE_VARIANTS 3
#define CTAUX_TILE_TABLE_SIZE 720
ctaux_status ctaux_autotune_tiles(ctaux_ctx *ctx, int n_blocks, int8_t *table_out, double *gain_out);
ctaux_status ctaux_get_tile_table(ctaux_ctx *ctx, int8_t *table_out);
ctaux_status ctaux_set_tile_table(ctaux_ctx *ctx, const int8_t *table);

/* Philox-4x32-10 on the device: for counters (t0 + i, chain, purpose), i <
 * count, write the two 53-bit uniforms of each draw to out[2*i], out[2*i+1].
 * A check of the device generator; allocates and frees a small buffer. */
ctaux_status ctaux_philox_uniforms(uint64_t seed, uint32_t chain, int64_t t0, int count,
                                   int purpose, double *out);

/* Block until all work queued on the context finishes; reports device faults. */
ctaux_status ctaux_synchronize(ctaux_ctx *ctx);

/* ---- Inversion without device allocation --------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: a host program whose device memory belongs to
 * another allocator (for example a framework's caching allocator that has
 * already reserved the GPU), or a steady-state loop that must not call
 * cudaMalloc because the call can block on, or synchronise, the whole device.
 *
 * Inverts the m x m float64 matrix d_a (column-major, leading dimension lda,
 * device memory) by Gauss-Jordan elimination with partial pivoting -- the
 * arithmetic of the FP64 recomputation that ctaux_recompute runs -- and
 * writes the inverse to d_inv (leading dimension ld_inv, device memory) and
 * log|det d_a| to *d_logdet (device memory, may be NULL).  Asynchronous on
 * cuda_stream (NULL = legacy default stream).  A singular input gives -inf in
 * *d_logdet and non-finite entries in d_inv.  The caller owns d_a, d_inv and
 * d_logdet; no context is needed.
 *
 * Scratch: one static device array of CTAUX_NOALLOC_SCRATCH_BYTES, held by
 * every GPU that loads the library until the process exits.  m is limited to
 * CTAUX_NOALLOC_MAX_M; a larger m returns CTAUX_ECAPACITY, bad pointers or
 * leading dimensions CTAUX_EINVAL, a failed launch CTAUX_ECUDA.  The first
 * call on a device looks up the array's device address and the launch size,
 * with that device current; make that first call before any stream capture.
 * Every call uses the same array and clears what must start at zero; calls
 * that overlap on the GPU (other streams, or other host threads without
 * ordering) race on it and corrupt each other's results. */
#define CTAUX_NOALLOC_MAX_M 512
#define CTAUX_NOALLOC_SCRATCH_BYTES 4202752
ctaux_status ctaux_invert_noalloc(const double *d_a, int lda, double *d_inv, int ld_inv, int m,
                                  double *d_logdet, void *cuda_stream);

void ctaux_destroy(ctaux_ctx *ctx);

/* Text of the last error of a context (never NULL). */
const char *ctaux_last_error(const ctaux_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CTAUX_H */
