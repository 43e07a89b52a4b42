// C ABI of the CT-AUX submatrix-update library (declared in include/ctaux.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/ctaux.h"
#include "ctaux_dev.cuh"
#include "ctaux_kernels.h"

using namespace ctaux;

struct ctaux_ctx {
  ctaux_params params{};
  std::vector<ctaux_chain_params> chains;
  int device = 0;
  int sm_count = 0;
  LaunchShape ls{};
  void* chains_dev = nullptr;        // Chain<double>[] or Chain<float>[]
  TcMaps* tc_maps_dev = nullptr;     // mixed form: TMA descriptors [chain][spin]
  std::vector<Chain<double>> hc64;   // host copies of the descriptors
  std::vector<Chain<float>> hc32;
  std::vector<void*> allocations;
  cudaStream_t last_stream = nullptr;
  PhaseTimer* timer = nullptr;
  bool profiling = false;
  int blocks_since_refresh = 0;
  std::string err;
  int max_ld = 0;
  // CUDA graphs of one block (with its near-tie launch), of one measurement,
  // and of one block with the previous block's measurement beside it (on the
  // side stream), captured on first use on a private stream, with their
  // kernel counts per phase
  cudaStream_t capture_stream = nullptr;
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};
  long long graph_kernels[3][PhaseTimer::kPhases] = {};
  bool graph_failed = false;
  // graph mode: the measurement of the last block swept, not yet launched (it
  // runs beside the next block, or alone before any other call reads or
  // changes the state)
  bool meas_pending = false;
  // tile-variant table of the products (the autotuner's cache), host copy
  std::vector<int8_t> tile_table = std::vector<int8_t>(kTileTable, 0);
  int8_t* tile_table_dev = nullptr;
};

namespace {

ctaux_status set_err(ctaux_ctx* ctx, ctaux_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

#define CUDA_TRY(ctx, expr)                                                                  \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      return set_err(ctx, CTAUX_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e));             \
  } while (0)

template <typename X>
X* dalloc(ctaux_ctx* ctx, size_t count, cudaError_t* err) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(X));
  if (e != cudaSuccess) {
    *err = e;
    return nullptr;
  }
  e = cudaMemset(p, 0, count * sizeof(X));
  if (e != cudaSuccess) *err = e;
  ctx->allocations.push_back(p);
  return reinterpret_cast<X*>(p);
}

int round_up(int v, int q) { return (v + q - 1) / q * q; }

bool is_mixed(const ctaux_ctx* ctx) { return ctx->params.precision == CTAUX_MIXED; }

template <typename T>
std::vector<Chain<T>>& host_chains(ctaux_ctx* ctx);
template <>
std::vector<Chain<double>>& host_chains<double>(ctaux_ctx* ctx) { return ctx->hc64; }
template <>
std::vector<Chain<float>>& host_chains<float>(ctaux_ctx* ctx) { return ctx->hc32; }

template <typename T>
ctaux_status build_chains(ctaux_ctx* ctx) {
  const ctaux_params& P = ctx->params;
  auto& hc = host_chains<T>(ctx);
  hc.resize(ctx->chains.size());
  cudaError_t err = cudaSuccess;
  int max_ld = 0, max_k = 1, max_cls_bins = 1;
  // launch shape first (tile bounds and k splits from the capacities)
  const int items = 2 * (int)ctx->chains.size();
  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    const ctaux_chain_params& cp = ctx->chains[ci];
    const int cap_m = cp.capacity + cp.k_max;
    const int ld = round_up(cap_m, 32);
    max_ld = std::max(max_ld, ld);
    max_k = std::max(max_k, cp.k_max);
    max_cls_bins = std::max(max_cls_bins, cp.n_classes * P.n_tau_bins);
  }
  LaunchShape& ls = ctx->ls;
  ls.n_chains = (int)ctx->chains.size();
  // fixed slice width of the inner dimension: narrow for FP64 (the FP64 pipe
  // is the bottleneck, so more CTAs), wider for FP32
  ls.kchunk = (sizeof(T) == 8) ? 32 : 128;
  // split-K partial tiles per (chain, spin): the most any product of the chain
  // can use at its capacity, at most kMaxPartials (device rule in gemm_items)
  std::vector<size_t> kpart_of(ctx->chains.size(), 1), kpart_meas_of(ctx->chains.size(), 1);
  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    const ctaux_chain_params& cp = ctx->chains[ci];
    const long cap_m = cp.capacity + cp.k_max, k = cp.k_max;
    // output rows and columns of each product at capacity (setup_gemm)
    const long rows[PH_COUNT] = {k, cap_m, k, cap_m, cap_m};
    const long cols[PH_COUNT] = {cap_m, k, k, cap_m, P.n_anchors};
    size_t need = 1;  // elements
    for (int ph = 0; ph < PH_COUNT; ++ph)
      for (int v = 0; v < kTileVariants; ++v) {
        const GemmTile tl = tile_variant(sizeof(T) == 8, ph, v);
        const long tiles = ((rows[ph] + tl.bm - 1) / tl.bm) * ((cols[ph] + tl.bn - 1) / tl.bn);
        const long k_inner = ph == PH_FLUSH ? k : cap_m;
        const long ks = std::max<long>(1, (k_inner + ls.kchunk - 1) / ls.kchunk);
        if (ks > 1) {
          const size_t el = (size_t)std::min<long>(kMaxPartials, tiles * ks) * tl.bm * tl.bn;
          need = std::max(need, el);
          if (ph == PH_MEAS) kpart_meas_of[ci] = std::max(kpart_meas_of[ci], el);
        }
      }
    kpart_of[ci] = need;
  }
  ls.persist_ctas = 8 * ctx->sm_count;   // 256-thread CTAs: up to 8 resident per SM
  for (int ph = 0; ph < PH_COUNT; ++ph) ls.tile_mask[ph] = 1;   // variant 0 until tuned
  {
    void* tt = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&tt, kTileTable));
    ctx->allocations.push_back(tt);
    CUDA_TRY(ctx, cudaMemset(tt, 0, kTileTable));
    ctx->tile_table_dev = reinterpret_cast<int8_t*>(tt);
  }
  ls.gather_slices = std::max(1, std::min(64, (2 * ctx->sm_count + items - 1) / items));
  ls.meas_lchunks = (max_ld + kMeasChunk - 1) / kMeasChunk;
  ls.meas_cb_blocks = (max_cls_bins + 255) / 256;
  ls.meas_acc_blocks = (max_cls_bins + 7) / 8;
  ctx->max_ld = max_ld;
  // proposal kernel shared memory
  size_t fixed = ((sizeof(T) * 8 * max_k + 15) & ~size_t(15)) + sizeof(double) * 2 * max_k + sizeof(int) * max_k +
                 sizeof(short) * ((max_ld + 7) & ~7) + sizeof(uint32_t) * ((max_ld + 31) / 32) +
                 sizeof(double) * 2 * max_k + sizeof(double) * 2 * max_k + ((max_ld + 15) & ~15) + 64;
  size_t gam = ((sizeof(T) * 2 * (size_t)max_k * (max_k + 1)) + 15) & ~size_t(15);
  ls.gamma_in_smem = (fixed + gam <= 200 * 1024) ? 1 : 0;
  ls.prop_smem = (int)(fixed + (ls.gamma_in_smem ? gam : 0));
  ls.gamma_lu = P.gamma_form == CTAUX_GAMMA_LU ? 1 : 0;
  ls.max_k = max_k;
  CUDA_TRY(ctx, configure_block_kernels<T>(ls));
  const bool mixed_tc = (sizeof(T) == 4) && P.mixed_flush_tc != 0;
  ls.use_tc = mixed_tc ? 1 : 0;
  int max_rows = 128;
  for (const auto& cp : ctx->chains) max_rows = std::max(max_rows, round_up(cp.capacity + cp.k_max, 128));
  ls.tc_ctas = ctx->sm_count;
  ls.split_x_blocks = std::max(1, std::min(256, (max_rows + 7) / 8));
  ls.mats = P.n_matsubara > 0 ? 1 : 0;
  ls.tc_wait_limit = P.tc_wait_limit;

  if (mixed_tc) CUDA_TRY(ctx, configure_flush_tc());
  // prep products on the tensor cores: the flush keeps N^T for them; every
  // chain's N must hold one 128-row TMA box
  bool prep_tc = mixed_tc && P.mixed_prep_tc != 0;
  for (const auto& cp : ctx->chains) prep_tc = prep_tc && round_up(cp.capacity + cp.k_max, 32) >= 128;
  ls.prep_tc = prep_tc ? 1 : 0;
  if (prep_tc) CUDA_TRY(ctx, configure_prep_tc());
  if (sizeof(T) == 4 && P.tie_guard > 0.0) {
    // one CTA per SM: the refinement is a chain of short grid-wide steps, so
    // barrier latency (which grows with the number of CTAs) dominates
    ls.tie_grid = ctx->sm_count;
    ls.tie_iters = P.tie_refine_iters == 0 ? 12 : std::max(0, P.tie_refine_iters);
  }
  std::vector<TcMaps> host_maps(mixed_tc ? 2 * ctx->chains.size() : 0);
  ls.refresh_df64 = (sizeof(T) == 4 && P.refresh_df64) ? 1 : 0;
  // refresh grid: every resident CTA, except when even a refresh of every chain
  // at its capacity is small (at most 4096 trailing-update tiles of 32 x 32 per
  // panel): then its ~35 grid barriers per panel, not its work, set its time,
  // and one CTA per SM makes each barrier shorter (measured: 0.081 -> 0.059 ms
  // per block for one 2x2x2 chain at n ~ 400; 22 % slower at n ~ 2100)
  int nb = refresh_blocks_per_sm<T>(ls.refresh_df64 != 0);
  long long cap_tiles = 0;
  for (const auto& cp : ctx->chains) {
    const long long tb = (cp.capacity + cp.k_max + 31) / 32;
    cap_tiles += 2 * tb * tb;
  }
  ls.refresh_grid = (cap_tiles <= 4096 ? 1 : std::max(1, nb)) * ctx->sm_count;

  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    const ctaux_chain_params& cp = ctx->chains[ci];
    Chain<T>& c = hc[ci];
    std::memset(&c, 0, sizeof(c));
    c.beta = cp.beta;
    c.K = cp.K;
    c.gamma = std::acosh(1.0 + cp.beta * cp.U * (double)cp.n_c / (2.0 * cp.K));
    c.dtau = cp.beta / (double)(cp.n_tau - 1);
    c.inv_dtau = (double)(cp.n_tau - 1) / cp.beta;
    for (int spin = 0; spin < 2; ++spin) {
      const double sig = spin == 0 ? 1.0 : -1.0;
      for (int dd = -2; dd <= 2; ++dd) {
        c.ev[spin][dd + 2] = (dd == 0) ? 1.0 : std::exp(c.gamma * sig * dd);
        c.inv_em1[spin][dd + 2] = (dd == 0) ? 0.0 : 1.0 / (c.ev[spin][dd + 2] - 1.0);
        const T lam = (T)(c.ev[spin][dd + 2] - 1.0);
        c.glam[spin][dd + 2] = (dd == 0) ? (T)0 : ((T)1 + lam) / lam;
      }
    }
    c.p_insert = P.p_insert;
    c.p_remove = 1.0 - P.p_insert - P.p_flip;
    c.n_c = cp.n_c;
    c.n_classes = cp.n_classes;
    c.n_tau = cp.n_tau;
    c.k_max = cp.k_max;
    c.cap_m = cp.capacity + cp.k_max;
    c.ld = round_up(c.cap_m, 32);
    c.seed = cp.seed;
    c.chain_id = cp.chain_id;
    c.tile_var = ctx->tile_table_dev;
    c.trace_cap = P.trace_capacity;
    c.n_bins = P.n_tau_bins;
    c.n_anchors = P.n_anchors;
    const size_t ld = c.ld, K = cp.k_max;
    const size_t tab = (size_t)2 * cp.n_classes * cp.n_tau;
    double* g0 = dalloc<double>(ctx, tab, &err);
    int* dxc = dalloc<int>(ctx, (size_t)cp.n_c * cp.n_c, &err);
    double* cw = dalloc<double>(ctx, cp.n_classes, &err);
    if (err != cudaSuccess) return set_err(ctx, CTAUX_ENOMEM, "device allocation failed: %s", cudaGetErrorString(err));
    CUDA_TRY(ctx, cudaMemcpy(g0, cp.g0_table, tab * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, cudaMemcpy(dxc, cp.dx_class, (size_t)cp.n_c * cp.n_c * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<double> w(cp.n_classes, 0.0);
    for (int x = 0; x < cp.n_c; ++x) w[cp.dx_class[x * cp.n_c + 0]] += 1.0;
    for (int k = 0; k < cp.n_classes; ++k) w[k] = w[k] > 0 ? 1.0 / (w[k] * P.n_anchors) : 0.0;
    CUDA_TRY(ctx, cudaMemcpy(cw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    c.g0 = g0;
    c.dx_class = dxc;
    c.class_weight = cw;
    for (int b = 0; b < 2; ++b) {
      for (int spin = 0; spin < 2; ++spin) c.N[b][spin] = dalloc<T>(ctx, ld * ld, &err);
      c.tau[b] = dalloc<double>(ctx, ld, &err);
      c.site[b] = dalloc<int>(ctx, ld, &err);
      c.s[b] = dalloc<int8_t>(ctx, ld, &err);
      c.birth[b] = dalloc<int64_t>(ctx, ld, &err);
    }
    c.s0 = dalloc<int8_t>(ctx, ld, &err);
    c.s_meas = dalloc<int8_t>(ctx, ld, &err);
    // panel rows: k_max, or whole 128-row TMA boxes for the tensor-core prep
    const size_t KR = prep_tc ? (size_t)round_up(std::max(cp.k_max, 128), 128) : K;
    for (int spin = 0; spin < 2; ++spin) {
      c.Cpan[spin] = dalloc<T>(ctx, KR * ld, &err);
      c.Bpan[spin] = dalloc<T>(ctx, ld * KR, &err);
      c.Gcol[spin] = dalloc<T>(ctx, ld * KR, &err);
      c.Ginv[spin] = dalloc<T>(ctx, K * (K + 1), &err);
      if (P.gamma_form == CTAUX_GAMMA_LU) c.Glu[spin] = dalloc<T>(ctx, K * (K + 1), &err);
      c.lam[spin] = dalloc<double>(ctx, K, &err);
      c.Y[spin] = dalloc<T>(ctx, ld * K, &err);
      c.Mg[spin] = dalloc<T>(ctx, ld * P.n_anchors, &err);
      c.Mv[spin] = dalloc<T>(ctx, ld * P.n_anchors, &err);
      c.Mpts[spin] = dalloc<double>(ctx, (size_t)ls.meas_lchunks * P.n_anchors * cp.n_c * P.n_tau_bins, &err);
      c.kpart[spin] = dalloc<T>(ctx, kpart_of[ci], &err);
      c.ticket[spin] = dalloc<int>(ctx, kMaxPartials, &err);
      c.kpart_meas[spin] = dalloc<T>(ctx, kpart_meas_of[ci], &err);
      c.ticket_meas[spin] = dalloc<int>(ctx, kMaxPartials, &err);
    }
    c.gamma_lu = P.gamma_form == CTAUX_GAMMA_LU ? 1 : 0;
    c.kp = round_up(cp.k_max, 32);
    c.tie_guard = (sizeof(T) == 4) ? P.tie_guard : 0.0;
    if (c.tie_guard > 0.0)
      for (int spin = 0; spin < 2; ++spin) c.N64[spin] = dalloc<double>(ctx, ld * ld, &err);
    if (mixed_tc) {
      const int rows = round_up(c.cap_m, 128);
      for (int spin = 0; spin < 2; ++spin) {
        c.Yh[spin] = reinterpret_cast<float*>(dalloc<T>(ctx, (size_t)rows * c.kp, &err));
        c.Yl[spin] = reinterpret_cast<float*>(dalloc<T>(ctx, (size_t)rows * c.kp, &err));
        c.Xh[spin] = reinterpret_cast<float*>(dalloc<T>(ctx, (size_t)rows * c.kp, &err));
        c.Xl[spin] = reinterpret_cast<float*>(dalloc<T>(ctx, (size_t)rows * c.kp, &err));
        if (err != cudaSuccess)
          return set_err(ctx, CTAUX_ENOMEM, "device allocation failed: %s", cudaGetErrorString(err));
        cudaError_t me = encode_tc_maps(&host_maps[2 * ci + spin], c.Yh[spin], c.Yl[spin], c.Xh[spin],
                                        c.Xl[spin], rows, c.kp, reinterpret_cast<float*>(c.N[0][spin]),
                                        reinterpret_cast<float*>(c.N[1][spin]), c.ld);
        if (me != cudaSuccess)
          return set_err(ctx, CTAUX_ECUDA, "tensor map encoding failed (%s)", cudaGetErrorString(me));
        if (prep_tc) {
          for (int b = 0; b < 2; ++b) c.NT[b][spin] = dalloc<float>(ctx, ld * ld, &err);
          if (err != cudaSuccess)
            return set_err(ctx, CTAUX_ENOMEM, "device allocation failed: %s", cudaGetErrorString(err));
          me = encode_prep_maps(&host_maps[2 * ci + spin], reinterpret_cast<float*>(c.Cpan[spin]),
                                reinterpret_cast<float*>(c.Bpan[spin]), (int)KR, reinterpret_cast<float*>(c.N[0][spin]),
                                reinterpret_cast<float*>(c.N[1][spin]), c.NT[0][spin], c.NT[1][spin], c.ld);
          if (me != cudaSuccess)
            return set_err(ctx, CTAUX_ECUDA, "prep tensor map encoding failed (%s)", cudaGetErrorString(me));
        }
      }
    }
    c.P = dalloc<int>(ctx, K, &err);
    c.draws = dalloc<BlockDraw>(ctx, K, &err);
    c.S = dalloc<int>(ctx, ld, &err);
    c.work = dalloc<double>(ctx, refresh_work_doubles((int)ld), &err);
    c.perm = dalloc<int>(ctx, 2 * ld, &err);
    c.used = dalloc<int8_t>(ctx, 2 * ld, &err);
    c.pcol = dalloc<int>(ctx, 2 * ld, &err);
    if (c.pcol) CUDA_TRY(ctx, cudaMemset(c.pcol, 0xFF, 2 * ld * sizeof(int)));
    c.pkeys = dalloc<unsigned long long>(ctx, 2 * ld, &err);
    c.work_drift = dalloc<double>(ctx, 3, &err);
    c.drift_limit = P.drift_limit;
    c.work_logdet = dalloc<double>(ctx, 2, &err);
    const size_t gb = (size_t)2 * cp.n_classes * P.n_tau_bins;
    c.Gsum = dalloc<double>(ctx, gb, &err);
    c.Gsq = dalloc<double>(ctx, gb, &err);
    c.Gbin = dalloc<double>(ctx, gb, &err);
    c.Gbsum = dalloc<double>(ctx, gb, &err);
    c.Gbsq = dalloc<double>(ctx, gb, &err);
    c.bin_size = P.meas_bin_size > 0 ? P.meas_bin_size : 16;
    c.n_freq = P.n_matsubara;
    if (c.n_freq > 0) {
      const size_t F = c.n_freq, nc = cp.n_c;
      c.G0w = dalloc<double2>(ctx, (size_t)2 * cp.n_classes * F, &err);
      c.vorder = dalloc<int>(ctx, ld, &err);
      c.site_off = dalloc<int>(ctx, nc + 1, &err);
      c.PhR = dalloc<unsigned char>(ctx, ld * F * 2 * sizeof(T), &err);
      for (int spin = 0; spin < 2; ++spin) {
        c.PhL[spin] = dalloc<unsigned char>(ctx, ld * F * 2 * sizeof(T), &err);
        c.Sw[spin] = dalloc<double2>(ctx, nc * nc * F, &err);
        c.Tw[spin] = dalloc<double2>(ctx, nc * nc * F, &err);
      }
      c.Gw_sum = dalloc<double>(ctx, 4 * nc * nc * F, &err);
      c.Gw_sq = dalloc<double>(ctx, 4 * nc * nc * F, &err);
      if (err != cudaSuccess)
        return set_err(ctx, CTAUX_ENOMEM, "device allocation failed: %s", cudaGetErrorString(err));
      launch_g0_matsubara(g0, cp.n_classes, cp.n_tau, cp.beta, c.n_freq, c.G0w, nullptr);
      CUDA_TRY(ctx, cudaDeviceSynchronize());
    }
    c.Gmeas = dalloc<double>(ctx, gb, &err);
    c.trace = dalloc<TraceRec>(ctx, std::max(1, P.trace_capacity), &err);
    c.dyn = dalloc<Dyn>(ctx, 1, &err);
    if (err != cudaSuccess)
      return set_err(ctx, CTAUX_ENOMEM, "device allocation failed: %s", cudaGetErrorString(err));
    Dyn d0;
    std::memset(&d0, 0, sizeof(d0));
    d0.sign = 1;
    d0.forced_t = -1;
    d0.guard_eff = c.tie_guard;
    CUDA_TRY(ctx, cudaMemcpy(c.dyn, &d0, sizeof(Dyn), cudaMemcpyHostToDevice));
  }
  if (mixed_tc) {
    void* dm = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&dm, host_maps.size() * sizeof(TcMaps)));
    ctx->allocations.push_back(dm);
    CUDA_TRY(ctx, cudaMemcpy(dm, host_maps.data(), host_maps.size() * sizeof(TcMaps),
                             cudaMemcpyHostToDevice));
    ctx->tc_maps_dev = reinterpret_cast<TcMaps*>(dm);
  }
  void* dc = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&dc, hc.size() * sizeof(Chain<T>)));
  ctx->allocations.push_back(dc);
  CUDA_TRY(ctx, cudaMemcpy(dc, hc.data(), hc.size() * sizeof(Chain<T>), cudaMemcpyHostToDevice));
  ctx->chains_dev = dc;
  return CTAUX_OK;
}

ctaux_status check_device_status(ctaux_ctx* ctx) {
  const bool mixed = is_mixed(ctx);
  int drift_chain = -1;
  double drift_rel = 0.0;
  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    Dyn* dp = mixed ? ctx->hc32[ci].dyn : ctx->hc64[ci].dyn;
    int st = 0;
    CUDA_TRY(ctx, cudaMemcpy(&st, &dp->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & DS_CAPACITY)
      return set_err(ctx, CTAUX_ECAPACITY, "chain %zu: expansion order + k_max exceeded the capacity", ci);
    if (st & DS_SINGULAR)
      return set_err(ctx, CTAUX_ESINGULAR, "chain %zu: zero pivot in the FP64 recomputation", ci);
    if (st & DS_INDEX) return set_err(ctx, CTAUX_EINVAL, "chain %zu: vertex selection out of range", ci);
    if (st & DS_TIMEOUT)
      return set_err(ctx, CTAUX_ETIMEOUT, "chain %zu: a bounded wait of the tensor-core flush gave up", ci);
    if (st) return set_err(ctx, CTAUX_ENUMERIC, "chain %zu: device status %d", ci, st);
    int ex = 0;
    CUDA_TRY(ctx, cudaMemcpy(&ex, &dp->drift_exceeded, sizeof(int), cudaMemcpyDeviceToHost));
    if (ex && drift_chain < 0) {
      drift_chain = (int)ci;
      CUDA_TRY(ctx, cudaMemcpy(&drift_rel, &dp->drift_rel, sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (ex) {
      const int zero = 0;   // reported once
      CUDA_TRY(ctx, cudaMemcpy(&dp->drift_exceeded, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  if (drift_chain >= 0)
    return set_err(ctx, CTAUX_EDRIFT, "chain %d: relative drift %.3e at a refresh above the limit %.3e",
                   drift_chain, drift_rel, ctx->params.drift_limit);
  return CTAUX_OK;
}

Dyn* dyn_of(ctaux_ctx* ctx, int chain) {
  return is_mixed(ctx) ? ctx->hc32[chain].dyn : ctx->hc64[chain].dyn;
}

ctaux_status read_dyn(ctaux_ctx* ctx, int chain, Dyn* out) {
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  CUDA_TRY(ctx, cudaMemcpy(out, dyn_of(ctx, chain), sizeof(Dyn), cudaMemcpyDeviceToHost));
  return CTAUX_OK;
}

template <typename T>
ctaux_status do_refresh(ctaux_ctx* ctx, int only_chain, cudaStream_t st) {
  cudaError_t e = launch_refresh<T>(reinterpret_cast<Chain<T>*>(ctx->chains_dev), ctx->ls, only_chain,
                                    st, ctx->timer);
  if (e != cudaSuccess) return set_err(ctx, CTAUX_ECUDA, "refresh launch: %s", cudaGetErrorString(e));
  return CTAUX_OK;
}

template <typename T>
ctaux_status do_sweeps(ctaux_ctx* ctx, int n_sweeps, int measure, cudaStream_t st) {
  Chain<T>* dc = reinterpret_cast<Chain<T>*>(ctx->chains_dev);
  PhaseTimer* pt = ctx->timer;
  const bool ties = (sizeof(T) == 4) && ctx->params.tie_guard > 0.0;
  // one block: plan, gather, prep, proposals, flush, and the near-tie decisions
  // in FP64 (iterative refinement against the float32 N, with a from-scratch
  // FP64 refresh in the same launch where it does not converge; the launch
  // exits at once without a pending tie)
  auto block = [&](cudaStream_t s, PhaseTimer* p) -> cudaError_t {
    launch_block<T>(dc, ctx->ls, s, p, ctx->tc_maps_dev);
    if (!ties) return cudaSuccess;
    p->begin(7, s);
    cudaError_t e = launch_tie_refine(reinterpret_cast<Chain<float>*>(dc), ctx->ls, s);
    p->end(7, s, 1);
    return e;
  };
  auto meas = [&](cudaStream_t s, PhaseTimer* p) -> cudaError_t {
    launch_measure<T>(dc, ctx->ls, s, p);
    return cudaSuccess;
  };
  // a block with the previous block's measurement beside it: the measurement's
  // head first, its tail on the side stream from the block's proposals to its end
  struct Tail {
    Chain<T>* dc;
    const LaunchShape* ls;
    int kernels;
  } tail{dc, &ctx->ls, 0};
  auto block_meas = [&](cudaStream_t s, PhaseTimer* p) -> cudaError_t {
    int nk = launch_measure_head<T>(dc, ctx->ls, s);
    BlockFork fk{ctx->side_stream, ctx->ev_fork, ctx->ev_join,
                 [](void* a, cudaStream_t side) {
                   Tail* t = static_cast<Tail*>(a);
                   t->kernels = launch_measure_tail<T>(t->dc, *t->ls, side);
                 },
                 &tail};
    launch_block<T>(dc, ctx->ls, s, p, ctx->tc_maps_dev, &fk);
    p->kernels[5] += nk + tail.kernels;
    if (!ties) return cudaSuccess;
    p->begin(7, s);
    cudaError_t e = launch_tie_refine(reinterpret_cast<Chain<float>*>(dc), ctx->ls, s);
    p->end(7, s, 1);
    return e;
  };
  // graph mode (not while profiling: the phase events would be frozen into the graph)
  const bool graphs = ctx->params.use_graph && !pt->on && !ctx->graph_failed;
  auto run = [&](int which, auto&& body) -> cudaError_t {
    if (graphs && !ctx->graph_exec[which]) {
      PhaseTimer counter;  // counts the captured kernels; records no events
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t eb = body(ctx->capture_stream, &counter);
        e = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (e == cudaSuccess) e = eb;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec[which], g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        // capture not possible here: direct launches from now on
        cudaGetLastError();
        ctx->graph_failed = true;
        ctx->graph_exec[which] = nullptr;
      } else {
        for (int ph = 0; ph < PhaseTimer::kPhases; ++ph) ctx->graph_kernels[which][ph] = counter.kernels[ph];
      }
    }
    if (graphs && ctx->graph_exec[which]) {
      for (int ph = 0; ph < PhaseTimer::kPhases; ++ph) pt->kernels[ph] += ctx->graph_kernels[which][ph];
      return cudaGraphLaunch(ctx->graph_exec[which], st);
    }
    return body(st, pt);
  };
  // with graphs, the measurement of block s (after its refresh, if one is due)
  // runs beside block s + 1, also across calls; it is left pending after the
  // last block, and launched alone (n_sweeps = 0) before any other entry point
  // reads or changes the state
  const bool can_fold = graphs && ctx->side_stream != nullptr;
  bool pend = ctx->meas_pending;
  ctx->meas_pending = false;
  if (pend && (n_sweeps == 0 || !can_fold)) {
    cudaError_t e = run(1, meas);
    if (e != cudaSuccess) return set_err(ctx, CTAUX_ECUDA, "measurement launch: %s", cudaGetErrorString(e));
    pend = false;
  }
  for (int s = 0; s < n_sweeps; ++s) {
    cudaError_t e = pend ? run(2, block_meas) : run(0, block);
    pend = false;
    if (e != cudaSuccess) return set_err(ctx, CTAUX_ECUDA, "block launch: %s", cudaGetErrorString(e));
    ctx->blocks_since_refresh += 1;
    if (ctx->params.refresh_every > 0 && ctx->blocks_since_refresh >= ctx->params.refresh_every) {
      ctaux_status r = do_refresh<T>(ctx, -1, st);
      if (r != CTAUX_OK) return r;
      ctx->blocks_since_refresh = 0;
    }
    if (measure) {
      if (can_fold) {
        pend = true;
      } else {
        e = run(1, meas);
        if (e != cudaSuccess) return set_err(ctx, CTAUX_ECUDA, "measurement launch: %s", cudaGetErrorString(e));
      }
    }
  }
  ctx->meas_pending = pend;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(ctx, CTAUX_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
  return CTAUX_OK;
}

// Launch the pending measurement (graph mode) on the sweeps' stream.
ctaux_status flush_pending(ctaux_ctx* ctx) {
  if (!ctx->meas_pending) return CTAUX_OK;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return is_mixed(ctx) ? do_sweeps<float>(ctx, 0, 0, ctx->last_stream)
                       : do_sweeps<double>(ctx, 0, 0, ctx->last_stream);
}

#define FLUSH_PENDING(ctx)                          \
  do {                                              \
    const ctaux_status _fp = flush_pending(ctx);    \
    if (_fp != CTAUX_OK) return _fp;                \
  } while (0)

}  // namespace

extern "C" {

ctaux_status ctaux_init(const ctaux_params* params, ctaux_ctx** out) {
  if (!out) return CTAUX_EINVAL;
  *out = nullptr;
  if (!params || params->n_chains < 1 || params->n_chains > 2048 || !params->chains)
    return CTAUX_EINVAL;
  if (params->precision != CTAUX_FP64 && params->precision != CTAUX_MIXED) return CTAUX_EINVAL;
  if (params->p_insert < 0 || params->p_flip < 0 || params->p_insert + params->p_flip > 1.0)
    return CTAUX_EINVAL;
  if (!(params->tie_guard >= 0.0) || params->tie_guard >= 1.0) return CTAUX_EINVAL;
  if (params->gamma_form != CTAUX_GAMMA_INVERSE && params->gamma_form != CTAUX_GAMMA_LU)
    return CTAUX_EINVAL;
  if (params->n_tau_bins < 1 || params->n_anchors < 1 || params->n_anchors > 64 ||
      params->trace_capacity < 0 || params->refresh_every < 0 || params->meas_bin_size < 0 ||
      params->n_matsubara < 0 || params->n_matsubara > kMaxMatsFreq ||
      !(params->drift_limit >= 0.0))
    return CTAUX_EINVAL;
  for (int i = 0; i < params->n_chains; ++i) {
    const ctaux_chain_params& c = params->chains[i];
    if (c.n_c < 1 || c.n_classes < 1 || c.n_tau < 2 || !c.g0_table || !c.dx_class) return CTAUX_EINVAL;
    if (!(c.beta > 0) || !(c.K > 0) || !(c.U > 0) || c.k_max < 1 || c.k_max > kMaxK || c.capacity < 1)
      return CTAUX_EINVAL;
    if (c.capacity + c.k_max > 30000) return CTAUX_EINVAL;
    if (params->n_matsubara > 0 && c.n_c > kMaxMatsSites) return CTAUX_EINVAL;
    for (int k = 0; k < c.n_c * c.n_c; ++k)
      if (c.dx_class[k] < 0 || c.dx_class[k] >= c.n_classes) return CTAUX_EINVAL;
  }
  ctaux_ctx* ctx = new ctaux_ctx();
  ctx->params = *params;
  ctx->chains.assign(params->chains, params->chains + params->n_chains);
  ctx->params.chains = nullptr;
  ctx->device = params->device;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) {
    set_err(ctx, CTAUX_ECUDA, "device %d: %s", ctx->device, cudaGetErrorString(e));
    ctaux_destroy(ctx);
    return CTAUX_ECUDA;
  }
  ctaux_status st = is_mixed(ctx) ? build_chains<float>(ctx) : build_chains<double>(ctx);
  if (st != CTAUX_OK) {
    ctaux_destroy(ctx);
    return st;
  }
  ctx->timer = new PhaseTimer();
  for (int i = 0; i < PhaseTimer::kPool; ++i) cudaEventCreate(&ctx->timer->ev[i]);
  ctx->timer->created = true;
  if (ctx->params.use_graph) {
    cudaError_t ge = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
    if (ge != cudaSuccess) {
      cudaGetLastError();
      ctx->graph_failed = true;
    } else if (cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ctx->side_stream = nullptr;   // measurements then run after their blocks
    }
  }
  *out = ctx;
  return CTAUX_OK;
}

ctaux_status ctaux_sweep(ctaux_ctx* ctx, int n_sweeps, int measure, void* cuda_stream) {
  if (!ctx || n_sweeps < 0) return CTAUX_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  ctx->last_stream = st;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // algorithmic work estimate from the current orders is accumulated at stats time
  return is_mixed(ctx) ? do_sweeps<float>(ctx, n_sweeps, measure, st)
                       : do_sweeps<double>(ctx, n_sweeps, measure, st);
}

ctaux_status ctaux_synchronize(ctaux_ctx* ctx) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return check_device_status(ctx);
}

ctaux_status ctaux_get_accumulators(ctaux_ctx* ctx, int chain, double* sum_out, double* sumsq_out,
                                    double* bin_sum_out, double* bin_sumsq_out, int64_t* counts_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size()) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  const ctaux_chain_params& cp = ctx->chains[chain];
  const size_t nb = (size_t)2 * cp.n_classes * ctx->params.n_tau_bins;
  const bool mx = is_mixed(ctx);
  const double* src[4] = {mx ? ctx->hc32[chain].Gsum : ctx->hc64[chain].Gsum,
                          mx ? ctx->hc32[chain].Gsq : ctx->hc64[chain].Gsq,
                          mx ? ctx->hc32[chain].Gbsum : ctx->hc64[chain].Gbsum,
                          mx ? ctx->hc32[chain].Gbsq : ctx->hc64[chain].Gbsq};
  double* dst[4] = {sum_out, sumsq_out, bin_sum_out, bin_sumsq_out};
  for (int k = 0; k < 4; ++k)
    if (dst[k]) CUDA_TRY(ctx, cudaMemcpy(dst[k], src[k], nb * sizeof(double), cudaMemcpyDeviceToHost));
  if (counts_out) {
    Dyn d;
    ctaux_status r = read_dyn(ctx, chain, &d);
    if (r != CTAUX_OK) return r;
    counts_out[0] = d.measurements;
    counts_out[1] = d.meas_bins;
    counts_out[2] = mx ? ctx->hc32[chain].bin_size : ctx->hc64[chain].bin_size;
  }
  return CTAUX_OK;
}

ctaux_status ctaux_measure_G(ctaux_ctx* ctx, int chain, double* G_out, double* err_out,
                             int64_t* n_meas_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || !G_out) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  const ctaux_chain_params& cp = ctx->chains[chain];
  const size_t nb = (size_t)2 * cp.n_classes * ctx->params.n_tau_bins;
  std::vector<double> sum(nb), sq(nb), bs(nb), bq(nb);
  int64_t cnt[3];
  ctaux_status r = ctaux_get_accumulators(ctx, chain, sum.data(), sq.data(), bs.data(), bq.data(), cnt);
  if (r != CTAUX_OK) return r;
  const double nm = (double)cnt[0], nbins = (double)cnt[1];
  for (size_t i = 0; i < nb; ++i) {
    const double mean = nm > 0 ? sum[i] / nm : 0.0;
    G_out[i] = mean;
    if (err_out) {
      if (nbins >= 2) {
        // spread of the completed bin means (binning analysis)
        const double bm = bs[i] / nbins;
        const double var = std::max(0.0, bq[i] / nbins - bm * bm) * nbins / (nbins - 1.0);
        err_out[i] = std::sqrt(var / nbins);
      } else {
        const double var = nm > 1 ? std::max(0.0, sq[i] / nm - mean * mean) * nm / (nm - 1.0) : 0.0;
        err_out[i] = nm > 1 ? std::sqrt(var / nm) : 0.0;
      }
    }
  }
  if (n_meas_out) *n_meas_out = cnt[0];
  return CTAUX_OK;
}

ctaux_status ctaux_measure_G_matsubara(ctaux_ctx* ctx, int chain, double* G_out, double* err_out,
                                       int64_t* n_meas_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || !G_out) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  if (ctx->params.n_matsubara <= 0)
    return set_err(ctx, CTAUX_EINVAL, "the context measures no Matsubara frequencies (n_matsubara = 0)");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  const ctaux_chain_params& cp = ctx->chains[chain];
  const size_t nb = (size_t)4 * cp.n_c * cp.n_c * ctx->params.n_matsubara;
  std::vector<double> sum(nb), sq(nb);
  const bool mx = is_mixed(ctx);
  CUDA_TRY(ctx, cudaMemcpy(sum.data(), mx ? ctx->hc32[chain].Gw_sum : ctx->hc64[chain].Gw_sum,
                           nb * sizeof(double), cudaMemcpyDeviceToHost));
  CUDA_TRY(ctx, cudaMemcpy(sq.data(), mx ? ctx->hc32[chain].Gw_sq : ctx->hc64[chain].Gw_sq,
                           nb * sizeof(double), cudaMemcpyDeviceToHost));
  Dyn d;
  ctaux_status r = read_dyn(ctx, chain, &d);
  if (r != CTAUX_OK) return r;
  const double nm = (double)d.measurements;
  for (size_t i = 0; i < nb; ++i) {
    const double mean = nm > 0 ? sum[i] / nm : 0.0;
    G_out[i] = mean;
    if (err_out) {
      const double var = nm > 1 ? std::max(0.0, sq[i] / nm - mean * mean) * nm / (nm - 1.0) : 0.0;
      err_out[i] = nm > 1 ? std::sqrt(var / nm) : 0.0;
    }
  }
  if (n_meas_out) *n_meas_out = d.measurements;
  return CTAUX_OK;
}

ctaux_status ctaux_reset_measurements(ctaux_ctx* ctx) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  if (is_mixed(ctx))
    launch_reset_measure<float>(reinterpret_cast<Chain<float>*>(ctx->chains_dev), ctx->ls, ctx->last_stream);
  else
    launch_reset_measure<double>(reinterpret_cast<Chain<double>*>(ctx->chains_dev), ctx->ls, ctx->last_stream);
  CUDA_TRY(ctx, cudaGetLastError());
  return CTAUX_OK;
}

ctaux_status ctaux_recompute(ctaux_ctx* ctx, double* drift_max_out) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  ctaux_status r = is_mixed(ctx) ? do_refresh<float>(ctx, -1, ctx->last_stream)
                                 : do_refresh<double>(ctx, -1, ctx->last_stream);
  if (r != CTAUX_OK) return r;
  ctx->blocks_since_refresh = 0;
  r = ctaux_synchronize(ctx);
  if (r != CTAUX_OK) return r;
  double mx = 0.0;
  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    Dyn d;
    r = read_dyn(ctx, (int)ci, &d);
    if (r != CTAUX_OK) return r;
    mx = std::max(mx, d.drift_max);
  }
  if (drift_max_out) *drift_max_out = mx;
  return CTAUX_OK;
}

ctaux_status ctaux_get_stats(ctaux_ctx* ctx, int chain, ctaux_stats* out) {
  if (!ctx || !out || chain < 0 || chain >= (int)ctx->chains.size()) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  Dyn d;
  ctaux_status r = read_dyn(ctx, chain, &d);
  if (r != CTAUX_OK) return r;
  std::memset(out, 0, sizeof(*out));
  out->n = d.n;
  out->t = d.t;
  for (int q = 0; q < 3; ++q) {
    out->proposals[q] = d.proposals[q];
    out->accepted[q] = d.accepted[q];
  }
  out->sweeps = d.sweeps;
  out->measurements = d.measurements;
  out->order_sum = d.order_sum;
  out->sign_sum = d.sign_sum;
  out->numeric_rejects = d.numeric_rejects;
  out->near_ties = d.near_ties;
  out->tie_refreshes = d.tie_refreshes;
  out->refreshes = d.refreshes;
  out->last_drift_max = d.drift_max;
  out->last_drift_fro = d.drift_fro;
  out->last_drift_rel = d.drift_rel;
  out->tie_err_max = d.tie_err_max;
  out->tie_guard_eff = d.guard_eff;
  out->logdet[0] = d.logdet[0];
  out->logdet[1] = d.logdet[1];
  out->sign = d.sign;
  out->status = d.status;
  return CTAUX_OK;
}

ctaux_status ctaux_get_trace(ctaux_ctx* ctx, int chain, ctaux_trace_rec* buf, int cap, int* n_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || (!buf && cap > 0) || !n_out)
    return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  *n_out = 0;
  const int tc = ctx->params.trace_capacity;
  if (tc <= 0) return CTAUX_OK;
  Dyn d;
  ctaux_status r = read_dyn(ctx, chain, &d);
  if (r != CTAUX_OK) return r;
  int64_t from = std::max(d.trace_read, d.trace_written - (int64_t)tc);
  int64_t count = std::min<int64_t>(d.trace_written - from, cap);
  const TraceRec* dt = is_mixed(ctx) ? ctx->hc32[chain].trace : ctx->hc64[chain].trace;
  static_assert(sizeof(TraceRec) == sizeof(ctaux_trace_rec), "trace record layout");
  for (int64_t i = 0; i < count; ++i) {
    const int64_t slot = (from + i) % tc;
    CUDA_TRY(ctx, cudaMemcpy(buf + i, dt + slot, sizeof(TraceRec), cudaMemcpyDeviceToHost));
  }
  const int64_t new_read = from + count;
  CUDA_TRY(ctx, cudaMemcpy(&dyn_of(ctx, chain)->trace_read, &new_read, sizeof(int64_t),
                           cudaMemcpyHostToDevice));
  *n_out = (int)count;
  return CTAUX_OK;
}

ctaux_status ctaux_get_config(ctaux_ctx* ctx, int chain, double* tau, int* site, int* s,
                              int64_t* birth, int cap, int* n_out, int64_t* t_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || !n_out) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  Dyn d;
  ctaux_status r = read_dyn(ctx, chain, &d);
  if (r != CTAUX_OK) return r;
  *n_out = d.n;
  if (t_out) *t_out = d.t;
  if (d.n > cap) return set_err(ctx, CTAUX_EINVAL, "buffer of %d entries for %d vertices", cap, d.n);
  const int b = d.buf;
  const double* dtau = is_mixed(ctx) ? ctx->hc32[chain].tau[b] : ctx->hc64[chain].tau[b];
  const int* dsite = is_mixed(ctx) ? ctx->hc32[chain].site[b] : ctx->hc64[chain].site[b];
  const int8_t* ds = is_mixed(ctx) ? ctx->hc32[chain].s[b] : ctx->hc64[chain].s[b];
  const int64_t* db = is_mixed(ctx) ? ctx->hc32[chain].birth[b] : ctx->hc64[chain].birth[b];
  std::vector<int8_t> s8(d.n);
  if (d.n > 0) {
    if (tau) CUDA_TRY(ctx, cudaMemcpy(tau, dtau, d.n * sizeof(double), cudaMemcpyDeviceToHost));
    if (site) CUDA_TRY(ctx, cudaMemcpy(site, dsite, d.n * sizeof(int), cudaMemcpyDeviceToHost));
    if (birth) CUDA_TRY(ctx, cudaMemcpy(birth, db, d.n * sizeof(int64_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(ctx, cudaMemcpy(s8.data(), ds, d.n, cudaMemcpyDeviceToHost));
    if (s)
      for (int i = 0; i < d.n; ++i) s[i] = s8[i];
  }
  return CTAUX_OK;
}

ctaux_status ctaux_set_config(ctaux_ctx* ctx, int chain, const double* tau, const int* site,
                              const int* s, const int64_t* birth, int n, int64_t t) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || n < 0 || t < 0) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  const ctaux_chain_params& cp = ctx->chains[chain];
  if (n > cp.capacity) return set_err(ctx, CTAUX_ECAPACITY, "order %d above capacity %d", n, cp.capacity);
  if (n > 0 && (!tau || !site || !s || !birth)) return CTAUX_EINVAL;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return birth[a] < birth[b]; });
  std::vector<double> tv(n);
  std::vector<int> sv(n);
  std::vector<int8_t> s8(n);
  std::vector<int64_t> bv(n);
  for (int i = 0; i < n; ++i) {
    const int k = order[i];
    if (!(tau[k] >= 0.0 && tau[k] < cp.beta) || site[k] < 0 || site[k] >= cp.n_c || (s[k] != 1 && s[k] != -1))
      return set_err(ctx, CTAUX_EINVAL, "vertex %d out of range", k);
    tv[i] = tau[k];
    sv[i] = site[k];
    s8[i] = (int8_t)s[k];
    bv[i] = birth[k];
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  Dyn d;
  CUDA_TRY(ctx, cudaMemcpy(&d, dyn_of(ctx, chain), sizeof(Dyn), cudaMemcpyDeviceToHost));
  const int b = d.buf;
  double* dtau = is_mixed(ctx) ? ctx->hc32[chain].tau[b] : ctx->hc64[chain].tau[b];
  int* dsite = is_mixed(ctx) ? ctx->hc32[chain].site[b] : ctx->hc64[chain].site[b];
  int8_t* ds = is_mixed(ctx) ? ctx->hc32[chain].s[b] : ctx->hc64[chain].s[b];
  int64_t* db = is_mixed(ctx) ? ctx->hc32[chain].birth[b] : ctx->hc64[chain].birth[b];
  if (n > 0) {
    CUDA_TRY(ctx, cudaMemcpy(dtau, tv.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, cudaMemcpy(dsite, sv.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, cudaMemcpy(ds, s8.data(), n, cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, cudaMemcpy(db, bv.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  d.n = n;
  d.t = t;
  d.status = 0;
  d.tie_pending = 0;
  d.forced_t = -1;
  int sg = 1;
  d.sign = sg;
  CUDA_TRY(ctx, cudaMemcpy(dyn_of(ctx, chain), &d, sizeof(Dyn), cudaMemcpyHostToDevice));
  ctaux_status r = is_mixed(ctx) ? do_refresh<float>(ctx, chain, ctx->last_stream)
                                 : do_refresh<double>(ctx, chain, ctx->last_stream);
  if (r != CTAUX_OK) return r;
  // the drift of this refresh compares N of the previous configuration with the
  // new one: it is not a drift of the chain
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  const int zero = 0;
  CUDA_TRY(ctx, cudaMemcpy(&dyn_of(ctx, chain)->drift_exceeded, &zero, sizeof(int), cudaMemcpyHostToDevice));
  return ctaux_synchronize(ctx);
}

ctaux_status ctaux_get_N(ctaux_ctx* ctx, int chain, int spin, double* out, int ld_out, int* m_out) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size() || spin < 0 || spin > 1 || !m_out)
    return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  Dyn d;
  ctaux_status r = read_dyn(ctx, chain, &d);
  if (r != CTAUX_OK) return r;
  *m_out = d.n;
  if (!out) return CTAUX_OK;
  if (ld_out < d.n) return CTAUX_EINVAL;
  const int b = d.buf;
  if (is_mixed(ctx)) {
    const Chain<float>& c = ctx->hc32[chain];
    std::vector<float> col(d.n);
    for (int j = 0; j < d.n; ++j) {
      CUDA_TRY(ctx, cudaMemcpy(col.data(), c.N[b][spin] + (size_t)j * c.ld, d.n * sizeof(float),
                               cudaMemcpyDeviceToHost));
      for (int i = 0; i < d.n; ++i) out[(size_t)j * ld_out + i] = col[i];
    }
  } else {
    const Chain<double>& c = ctx->hc64[chain];
    if (d.n > 0)
      CUDA_TRY(ctx, cudaMemcpy2D(out, (size_t)ld_out * sizeof(double), c.N[b][spin], (size_t)c.ld * sizeof(double),
                                 d.n * sizeof(double), d.n, cudaMemcpyDeviceToHost));
  }
  return CTAUX_OK;
}

ctaux_status ctaux_set_profiling(ctaux_ctx* ctx, int on) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  if (ctx->profiling && !on) ctx->timer->collect();
  ctx->profiling = on != 0;
  ctx->timer->on = ctx->profiling;
  return CTAUX_OK;
}

ctaux_status ctaux_get_phase_times(ctaux_ctx* ctx, double* ms_out, int64_t* kernels_out) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  ctx->timer->collect();
  for (int p = 0; p < PhaseTimer::kPhases; ++p) {
    if (ms_out) ms_out[p] = ctx->timer->ms[p];
    if (kernels_out) kernels_out[p] = ctx->timer->kernels[p];
  }
  return CTAUX_OK;
}

ctaux_status ctaux_get_work(ctaux_ctx* ctx, double* prep_flop, double* flush_flop, double* flush_bytes,
                            double* gamma_flop, double* meas_flop, double* refresh_flop,
                            double* mats_flop) {
  if (!ctx) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  double a = 0.0, b = 0.0, c = 0.0, g = 0.0, me = 0.0, rf = 0.0, mw = 0.0;
  for (size_t ci = 0; ci < ctx->chains.size(); ++ci) {
    Dyn d;
    ctaux_status r = read_dyn(ctx, (int)ci, &d);
    if (r != CTAUX_OK) return r;
    a += d.work_prep;
    b += d.work_flush;
    c += d.bytes_flush;
    g += d.work_gamma;
    me += d.work_meas;
    rf += d.work_refresh;
    mw += d.work_mats;
  }
  if (mats_flop) *mats_flop = mw;
  if (gamma_flop) *gamma_flop = g;
  if (meas_flop) *meas_flop = me;
  if (refresh_flop) *refresh_flop = rf;
  if (prep_flop) *prep_flop = a;
  if (flush_flop) *flush_flop = b;
  if (flush_bytes) *flush_bytes = c;
  return CTAUX_OK;
}

ctaux_status ctaux_set_kmax(ctaux_ctx* ctx, int chain, int k_max) {
  if (!ctx || chain < 0 || chain >= (int)ctx->chains.size()) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  if (k_max < 1 || k_max > ctx->chains[chain].k_max) return CTAUX_EINVAL;  // buffers sized at init
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  if (is_mixed(ctx)) {
    ctx->hc32[chain].k_max = k_max;
    Chain<float>* dc = reinterpret_cast<Chain<float>*>(ctx->chains_dev) + chain;
    CUDA_TRY(ctx, cudaMemcpy(&dc->k_max, &k_max, sizeof(int), cudaMemcpyHostToDevice));
  } else {
    ctx->hc64[chain].k_max = k_max;
    Chain<double>* dc = reinterpret_cast<Chain<double>*>(ctx->chains_dev) + chain;
    CUDA_TRY(ctx, cudaMemcpy(&dc->k_max, &k_max, sizeof(int), cudaMemcpyHostToDevice));
  }
  return CTAUX_OK;
}

namespace {
int current_kmax(ctaux_ctx* ctx, int chain) {
  return is_mixed(ctx) ? ctx->hc32[chain].k_max : ctx->hc64[chain].k_max;
}
}  // namespace

ctaux_status ctaux_autotune_k(ctaux_ctx* ctx, const int* candidates, int n_candidates, int n_blocks,
                              int* k_out, double* rate_out) {
  if (!ctx || !candidates || n_candidates < 1 || n_blocks < 1) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  for (int i = 0; i < n_candidates; ++i)
    if (candidates[i] < 1 || candidates[i] > kMaxK) return CTAUX_EINVAL;
  const int nch = (int)ctx->chains.size();
  cudaStream_t st = ctx->last_stream;
  // buckets: (cluster size, order octave) from the current orders
  std::vector<int> bucket(nch);
  std::vector<std::pair<int, int>> keys;
  std::vector<int> pop;
  for (int c = 0; c < nch; ++c) {
    Dyn d;
    ctaux_status r = read_dyn(ctx, c, &d);
    if (r != CTAUX_OK) return r;
    int oct = 0;
    while ((16 << oct) <= d.n && oct < 20) ++oct;
    const std::pair<int, int> key(ctx->chains[c].n_c, oct);
    int b = 0;
    while (b < (int)keys.size() && keys[b] != key) ++b;
    if (b == (int)keys.size()) {
      keys.push_back(key);
      pop.push_back(0);
    }
    bucket[c] = b;
    pop[b] += 1;
  }
  const int nb = (int)keys.size();
  const int saved_refresh = ctx->params.refresh_every;
  ctx->params.refresh_every = 0;  // no refresh inside the timed trials
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(ctx, cudaEventCreate(&e0));
  CUDA_TRY(ctx, cudaEventCreate(&e1));
  ctaux_status status = CTAUX_OK;
  // proposals per second of the whole context with bucket b at k[b] (capped by
  // each chain's allocation); one untimed block first
  auto evaluate = [&](const std::vector<int>& kb, double* rate) -> ctaux_status {
    for (int c = 0; c < nch; ++c) {
      const int k = std::min(kb[bucket[c]], ctx->chains[c].k_max);
      if (k != current_kmax(ctx, c)) {
        ctaux_status r = ctaux_set_kmax(ctx, c, k);
        if (r != CTAUX_OK) return r;
      }
    }
    ctaux_status r = ctaux_sweep(ctx, 1, 0, st);
    if (r != CTAUX_OK) return r;
    r = ctaux_synchronize(ctx);
    if (r != CTAUX_OK) return r;
    int64_t t0 = 0, t1 = 0;
    for (int c = 0; c < nch; ++c) {
      Dyn d;
      if ((r = read_dyn(ctx, c, &d)) != CTAUX_OK) return r;
      t0 += d.t;
    }
    CUDA_TRY(ctx, cudaEventRecord(e0, st));
    if ((r = ctaux_sweep(ctx, n_blocks, 0, st)) != CTAUX_OK) return r;
    CUDA_TRY(ctx, cudaEventRecord(e1, st));
    if ((r = ctaux_synchronize(ctx)) != CTAUX_OK) return r;
    float ms = 0.f;
    CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
    for (int c = 0; c < nch; ++c) {
      Dyn d;
      if ((r = read_dyn(ctx, c, &d)) != CTAUX_OK) return r;
      t1 += d.t;
    }
    *rate = (double)(t1 - t0) / (ms > 0.f ? ms * 1e-3 : 1e-9);
    return CTAUX_OK;
  };
  // 1) the best common k; 2) coordinate descent over buckets, most populated
  // first, keeping a change only if it gains more than 2 %
  std::vector<int> best_k(nb, candidates[0]);
  double best = -1.0;
  for (int i = 0; i < n_candidates && status == CTAUX_OK; ++i) {
    std::vector<int> kb(nb, candidates[i]);
    double rate = 0.0;
    status = evaluate(kb, &rate);
    if (status == CTAUX_OK && rate > best) {
      best = rate;
      best_k = kb;
    }
  }
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return pop[a] > pop[b]; });
  if (nb > 1) {
    for (int b : order) {
      for (int i = 0; i < n_candidates && status == CTAUX_OK; ++i) {
        if (candidates[i] == best_k[b]) continue;
        std::vector<int> kb = best_k;
        kb[b] = candidates[i];
        double rate = 0.0;
        status = evaluate(kb, &rate);
        if (status == CTAUX_OK && rate > 1.02 * best) {
          best = rate;
          best_k = kb;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->params.refresh_every = saved_refresh;
  if (status != CTAUX_OK) return status;
  for (int c = 0; c < nch; ++c) {
    const int k = std::min(best_k[bucket[c]], ctx->chains[c].k_max);
    ctaux_status r = ctaux_set_kmax(ctx, c, k);
    if (r != CTAUX_OK) return r;
    if (k_out) k_out[c] = k;
  }
  if (rate_out) *rate_out = best;
  // the trials ran without refreshes: start from a fresh N
  return ctaux_recompute(ctx, nullptr);
}

ctaux_status ctaux_set_tile_table(ctaux_ctx* ctx, const int8_t* table) {
  if (!ctx || !table) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  for (int i = 0; i < kTileTable; ++i)
    if (table[i] < 0 || table[i] >= kTileVariants) return CTAUX_EINVAL;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->last_stream));
  std::copy(table, table + kTileTable, ctx->tile_table.begin());
  CUDA_TRY(ctx, cudaMemcpy(ctx->tile_table_dev, table, kTileTable, cudaMemcpyHostToDevice));
  for (int ph = 0; ph < PH_COUNT; ++ph) {
    int mask = 0;
    for (int i = 0; i < kTileOct * kTileKOct; ++i) mask |= 1 << table[ph * kTileOct * kTileKOct + i];
    ctx->ls.tile_mask[ph] = mask;
  }
  // captured graphs hold the old set of launches
  for (int w = 0; w < 3; ++w)
    if (ctx->graph_exec[w]) {
      cudaGraphExecDestroy(ctx->graph_exec[w]);
      ctx->graph_exec[w] = nullptr;
    }
  return CTAUX_OK;
}

ctaux_status ctaux_get_tile_table(ctaux_ctx* ctx, int8_t* table_out) {
  if (!ctx || !table_out) return CTAUX_EINVAL;
  std::copy(ctx->tile_table.begin(), ctx->tile_table.end(), table_out);
  return CTAUX_OK;
}

ctaux_status ctaux_autotune_tiles(ctaux_ctx* ctx, int n_blocks, int8_t* table_out, double* gain_out) {
  if (!ctx || n_blocks < 1) return CTAUX_EINVAL;
  FLUSH_PENDING(ctx);
  const int nch = (int)ctx->chains.size();
  const bool mixed = is_mixed(ctx);
  // products this context launches on the CUDA cores, with the phase timer and
  // work counter that measure them (0 prep, 1 flush, 2 measurement)
  std::vector<std::pair<int, int>> prods;
  if (!(mixed && ctx->ls.prep_tc))
    for (int ph : {PH_RTILDE, PH_GCOL_OLD, PH_GCOL_NEW}) prods.push_back({ph, 0});
  if (!(mixed && ctx->ls.use_tc)) prods.push_back({PH_FLUSH, 1});
  prods.push_back({PH_MEAS, 2});
  const int timer_phase[3] = {1, 3, 5};
  // groups: (octave of the current order, octave of k_max) slots of the table
  std::vector<int> slot_pop(kTileOct * kTileKOct, 0);
  for (int c = 0; c < nch; ++c) {
    Dyn d;
    ctaux_status r = read_dyn(ctx, c, &d);
    if (r != CTAUX_OK) return r;
    const int kmax = mixed ? ctx->hc32[c].k_max : ctx->hc64[c].k_max;
    slot_pop[tile_table_index(0, d.n, kmax)] += 1;
  }
  std::vector<int> slots;
  for (int i = 0; i < (int)slot_pop.size(); ++i)
    if (slot_pop[i] * 10 >= nch) slots.push_back(i);
  std::sort(slots.begin(), slots.end(), [&](int a, int b) { return slot_pop[a] > slot_pop[b]; });
  if (slots.size() > 4) slots.resize(4);
  const int saved_refresh = ctx->params.refresh_every;
  const bool saved_prof = ctx->profiling;
  ctx->params.refresh_every = 0;  // no refresh inside the timed trials
  ctaux_set_profiling(ctx, 1);
  std::vector<int8_t> table = ctx->tile_table;
  double first_total = 0.0, best_total = 0.0;
  ctaux_status status = CTAUX_OK;
  // milliseconds per algorithmic flop of product p's phase over n_blocks blocks
  auto score = [&](int kind, double* out) -> ctaux_status {
    ctaux_status r = ctaux_set_tile_table(ctx, table.data());
    if (r != CTAUX_OK) return r;
    if ((r = ctaux_sweep(ctx, 1, kind == 2, ctx->last_stream)) != CTAUX_OK) return r;  // untimed
    if ((r = ctaux_synchronize(ctx)) != CTAUX_OK) return r;
    double ms0[PhaseTimer::kPhases], ms1[PhaseTimer::kPhases], w0[7], w1[7];
    ctaux_get_phase_times(ctx, ms0, nullptr);
    ctaux_get_work(ctx, &w0[0], &w0[1], &w0[2], &w0[3], &w0[4], &w0[5], &w0[6]);
    if ((r = ctaux_sweep(ctx, n_blocks, kind == 2, ctx->last_stream)) != CTAUX_OK) return r;
    if ((r = ctaux_synchronize(ctx)) != CTAUX_OK) return r;
    ctaux_get_phase_times(ctx, ms1, nullptr);
    ctaux_get_work(ctx, &w1[0], &w1[1], &w1[2], &w1[3], &w1[4], &w1[5], &w1[6]);
    const int wi = kind == 0 ? 0 : kind == 1 ? 1 : 4;
    const double work = w1[wi] - w0[wi];
    const double ms = ms1[timer_phase[kind]] - ms0[timer_phase[kind]];
    *out = work > 0.0 ? ms / work : ms;
    return CTAUX_OK;
  };
  for (const auto& pk : prods) {
    const int ph = pk.first, kind = pk.second;
    auto set_all = [&](int v) {
      for (int i = 0; i < kTileOct * kTileKOct; ++i) table[ph * kTileOct * kTileKOct + i] = (int8_t)v;
    };
    // 1) one variant for every slot; 2) per populated slot, keep a change
    // only if it gains more than 2 %
    double best = 0.0, s0 = 0.0;
    int best_v = 0;
    for (int v = 0; v < kTileVariants && status == CTAUX_OK; ++v) {
      set_all(v);
      double sc = 0.0;
      status = score(kind, &sc);
      if (v == 0) s0 = sc;
      if (status == CTAUX_OK && (v == 0 || sc < best)) {
        best = sc;
        best_v = v;
      }
    }
    if (status != CTAUX_OK) break;
    set_all(best_v);
    for (int slot : slots) {
      const int idx = ph * kTileOct * kTileKOct + slot;
      for (int v = 0; v < kTileVariants && status == CTAUX_OK; ++v) {
        if (v == table[idx]) continue;
        const int8_t keep = table[idx];
        table[idx] = (int8_t)v;
        double sc = 0.0;
        status = score(kind, &sc);
        if (status == CTAUX_OK && sc < 0.98 * best) best = sc;
        else table[idx] = keep;
      }
    }
    first_total += s0;
    best_total += best;
  }
  ctx->params.refresh_every = saved_refresh;
  ctaux_set_profiling(ctx, saved_prof ? 1 : 0);
  if (status != CTAUX_OK) return status;
  ctaux_status r = ctaux_set_tile_table(ctx, table.data());
  if (r != CTAUX_OK) return r;
  if (table_out) std::copy(table.begin(), table.end(), table_out);
  if (gain_out) *gain_out = best_total > 0.0 ? first_total / best_total : 1.0;
  // the trials ran without refreshes: start from a fresh N
  return ctaux_recompute(ctx, nullptr);
}

ctaux_status ctaux_philox_uniforms(uint64_t seed, uint32_t chain, int64_t t0, int count, int purpose,
                                   double* out) {
  if (count < 0 || !out || purpose < 0) return CTAUX_EINVAL;
  if (count == 0) return CTAUX_OK;
  double* d = nullptr;
  if (cudaMalloc(&d, (size_t)count * 2 * sizeof(double)) != cudaSuccess) return CTAUX_ENOMEM;
  launch_philox_test(seed, chain, t0, count, purpose, d, nullptr);
  cudaError_t e = cudaMemcpy(out, d, (size_t)count * 2 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? CTAUX_OK : CTAUX_ECUDA;
}

void ctaux_destroy(ctaux_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->last_stream);
  for (int w = 0; w < 3; ++w)
    if (ctx->graph_exec[w]) cudaGraphExecDestroy(ctx->graph_exec[w]);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (void* p : ctx->allocations) cudaFree(p);
  if (ctx->timer) {
    if (ctx->timer->created)
      for (int i = 0; i < PhaseTimer::kPool; ++i) cudaEventDestroy(ctx->timer->ev[i]);
    delete ctx->timer;
  }
  delete ctx;
}

const char* ctaux_last_error(const ctaux_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

}  // extern "C"
