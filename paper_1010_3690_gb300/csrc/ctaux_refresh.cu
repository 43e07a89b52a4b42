// From-scratch refresh kernels (bodies in ctaux_refresh.cuh): elimination in
// float64, or in double-float on the float32 pipe (mixed form, optional).
#include <type_traits>

#include "ctaux_refresh.cuh"

namespace ctaux {

template <typename T, typename E>
__global__ void __launch_bounds__(256) k_refresh(Chain<T>* chains, int n_chains, int only_chain,
                                                 int filter) {
  refresh_body<T, E>(chains, n_chains, only_chain, filter);
}

// Small follow-up kernel: the stats of every refreshed chain.
template <typename T>
__global__ void k_refresh_finish(Chain<T>* chains, int n_chains, int only_chain, int filter) {
  const int ci = (only_chain >= 0) ? only_chain : (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (ci >= n_chains) return;
  if (only_chain >= 0 && (blockIdx.x | threadIdx.x)) return;
  refresh_finish_one(chains[ci], filter);
}

template <typename T>
cudaError_t launch_refresh(Chain<T>* dchains, const LaunchShape& ls, int only_chain,
                           cudaStream_t st, PhaseTimer* pt, int filter) {
  pt->begin(6, st);
  int nch = ls.n_chains;
  cudaError_t e = cudaSuccess;
  void* args[] = {&dchains, &nch, &only_chain, &filter};
  // double-float elimination only for the float32 form's own refreshes; the
  // near-tie fallback (filter 1) keeps float64, whose N it also stores
  const void* fn = (const void*)k_refresh<T, double>;
  size_t dyn = 0;
  if constexpr (std::is_same<T, float>::value)
    if (ls.refresh_df64 && filter == 0) {
      fn = (const void*)k_refresh<T, df64>;
      dyn = refresh_dyn_smem<df64>();
    }
  e = cudaLaunchCooperativeKernel(fn, dim3(ls.refresh_grid), dim3(256), args, dyn, st);
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
int refresh_blocks_per_sm(bool df) {
  // with the double-float option the grid must be co-resident for either
  // element type (the near-tie fallback keeps float64)
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refresh<T, double>, 256, 0);
  if constexpr (std::is_same<T, float>::value) {
    if (df) {
      int nb2 = 0;
      cudaFuncSetAttribute(k_refresh<T, df64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           refresh_dyn_smem<df64>());
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_refresh<T, df64>, 256,
                                                    refresh_dyn_smem<df64>());
      nb = nb < nb2 ? nb : nb2;
    }
  }
  return nb;
}

template cudaError_t launch_refresh<double>(Chain<double>*, const LaunchShape&, int, cudaStream_t,
                                            PhaseTimer*, int);
template cudaError_t launch_refresh<float>(Chain<float>*, const LaunchShape&, int, cudaStream_t,
                                           PhaseTimer*, int);
size_t refresh_work_doubles(int ld) { return 2 * refresh_work_per_spin(ld); }

template int refresh_blocks_per_sm<double>(bool);
template int refresh_blocks_per_sm<float>(bool);

}  // namespace ctaux
