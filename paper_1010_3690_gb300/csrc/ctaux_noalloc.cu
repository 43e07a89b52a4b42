// ctaux_invert_noalloc: the FP64 Gauss-Jordan inversion of the from-scratch
// recomputation, for callers that cannot allocate device memory.  Its scratch
// (two ping-pong matrices, pivot keys, pivot flags, the pivot permutation and
// the log-determinant accumulator) lives in one file-scope static device
// array; nothing here calls cudaMalloc, cudaFree or an allocating library
// routine.  Declared in include/ctaux.h.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ctaux.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kM = CTAUX_NOALLOC_MAX_M;
constexpr size_t kWorkDoubles = (size_t)2 * kM * kM;
constexpr size_t kScratchBytes = kWorkDoubles * sizeof(double)  // ping-pong matrices
                                 + kM * sizeof(unsigned long long)  // pivot keys
                                 + kM * sizeof(int)                 // pivot rows
                                 + kM * sizeof(int)                 // pivot flags
                                 + 2 * sizeof(double);              // log|det|, spare
static_assert(kScratchBytes <= CTAUX_NOALLOC_SCRATCH_BYTES, "scratch size in the header");

// Shared by every call on a device; held by each device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CTAUX_NOALLOC_SCRATCH_BYTES];

// Pivot key: the upper 32 bits of |v|'s float64 pattern (sign 0, the whole
// exponent, 20 significand bits) order like |v| for every non-negative double,
// so any normal entry, however small, beats an exact zero; ties within 2^-20
// go to the lower row.
__device__ __forceinline__ unsigned long long na_pivot_key(double v, int row) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(v));
  return (bits & 0xffffffff00000000ull) | (unsigned long long)(0xffffffffu - (unsigned)row);
}
__device__ __forceinline__ int na_key_row(unsigned long long k) {
  return (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// Cooperative kernel: m Gauss-Jordan column steps with partial pivoting,
// ping-pong between the two scratch matrices, grid barriers between steps
// (the same arithmetic as the context's FP64 refresh).
__global__ void __launch_bounds__(256) k_invert_noalloc(const double* __restrict__ A, int lda,
                                                        double* __restrict__ Ainv, int ldi, int m,
                                                        unsigned char* scratch, double* logdet_out) {
  cg::grid_group grid = cg::this_grid();
  double* W0 = reinterpret_cast<double*>(scratch);
  double* W1 = W0 + (size_t)kM * kM;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(W0 + kWorkDoubles);
  int* perm = reinterpret_cast<int*>(keys + kM);
  int* used = perm + kM;
  double* acc = reinterpret_cast<double*>(used + kM);
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gthreads = (long)gridDim.x * blockDim.x;

  // the previous call's keys, flags and log-determinant must not leak in
  for (long e = gtid; e < kM; e += gthreads) {
    keys[e] = 0ull;
    used[e] = 0;
  }
  if (gtid == 0) acc[0] = 0.0;
  grid.sync();

  for (int j = blockIdx.x; j < m; j += gridDim.x)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[(size_t)j * lda + i];
      W0[(size_t)j * kM + i] = v;
      if (j == 0) atomicMax(keys, na_pivot_key(v, i));
    }
  grid.sync();

  for (int col = 0; col < m; ++col) {
    const double* X = (col & 1) ? W1 : W0;
    double* Y = (col & 1) ? W0 : W1;
    const int pr = na_key_row(keys[col]);
    const double piv = X[(size_t)col * kM + pr];
    if (gtid == 0) {
      perm[col] = pr;
      used[pr] = 1;
      acc[0] += log(fabs(piv));
    }
    const double ipiv = 1.0 / piv;
    for (int j = blockIdx.x; j < m; j += gridDim.x) {
      const double xpj = X[(size_t)j * kM + pr] * ipiv;
      const double* Xj = X + (size_t)j * kM;
      const double* Xc = X + (size_t)col * kM;
      double* Yj = Y + (size_t)j * kM;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double v;
        if (i == pr) v = (j == col) ? ipiv : xpj;
        else if (j == col) v = -Xc[i] * ipiv;
        else v = Xj[i] - Xc[i] * xpj;
        Yj[i] = v;
        if (j == col + 1 && i != pr && !used[i]) atomicMax(keys + col + 1, na_pivot_key(v, i));
      }
    }
    grid.sync();
  }

  const double* X = (m & 1) ? W1 : W0;
  for (int j = blockIdx.x; j < m; j += gridDim.x)
    for (int c = threadIdx.x; c < m; c += blockDim.x)
      Ainv[(size_t)perm[j] * ldi + c] = X[(size_t)j * kM + perm[c]];  // inv[c][perm[j]]
  if (gtid == 0 && logdet_out) *logdet_out = acc[0];
}

struct DeviceSetup {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int grid = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];

}  // namespace

extern "C" ctaux_status ctaux_invert_noalloc(const double* d_a, int lda, double* d_inv, int ld_inv,
                                             int m, double* d_logdet, void* cuda_stream) {
  if (!d_a || !d_inv || m < 1 || lda < m || ld_inv < m) return CTAUX_EINVAL;
  if (m > CTAUX_NOALLOC_MAX_M) return CTAUX_ECAPACITY;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CTAUX_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return CTAUX_EINVAL;
  DeviceSetup& s = g_setup[dev];
  // once per device, with that device current: the host-side name of the
  // array is only a stand-in, so resolve its device address here
  std::call_once(s.once, [&s, dev]() {
    s.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scratch), g_noalloc_scratch);
    int sms = 0, per_sm = 0;
    if (s.err == cudaSuccess) s.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (s.err == cudaSuccess)
      s.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_invert_noalloc, 256, 0);
    s.grid = (per_sm > 0 ? per_sm : 1) * sms;
  });
  if (s.err != cudaSuccess || !s.scratch || s.grid < 1) return CTAUX_ECUDA;
  unsigned char* scratch = s.scratch;
  void* args[] = {(void*)&d_a, &lda, (void*)&d_inv, &ld_inv, &m, &scratch, (void*)&d_logdet};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_invert_noalloc, dim3(s.grid),
                                                    dim3(256), args, 0,
                                                    reinterpret_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? CTAUX_OK : CTAUX_ECUDA;
}
