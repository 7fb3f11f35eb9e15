// Allocation-free variant of the free-DOF residual norm (the Newton
// convergence check's reduction).
//
// Some callers cannot call cudaMalloc at the point where they need this
// check: code that runs while a framework owns every device allocation (a
// host application's memory pool, a plugin handed only pre-allocated
// buffers), or a real-time loop that forbids allocation after start-up.  This
// entry point takes the caller's device buffers for its inputs and a host
// pointer for its output, and keeps its only scratch (one FP64 partial sum per
// thread block) in a file-scope device array.  It calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The array costs NOALLOC_MAX_BLOCKS * 8 bytes (64 KiB) of device memory on
// every GPU that loads the library, held until the process exits.  All calls
// share it, so calls whose work overlaps on the GPU race with each other; the
// caller must order them (one stream, or events).  Each call writes every
// slot it later reads, so nothing needs clearing between calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "mpm.h"

namespace {

constexpr int NOALLOC_TPB = 256;
constexpr int NOALLOC_MAX_BLOCKS = 8192;                  // 64 KiB of partial sums
constexpr long long NOALLOC_MAX_ROWS = (long long)NOALLOC_MAX_BLOCKS * NOALLOC_TPB;
constexpr int NOALLOC_MAX_DEVICES = 64;

// The scratch: one partial per block of stage 1, plus one slot for the total.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS + 32];

// Host-side device addresses of the scratch, one per device, set up once.
double* g_scratch_addr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;
thread_local std::string g_noalloc_err;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[NOALLOC_TPB / 32];
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < NOALLOC_TPB / 32) ? ws[threadIdx.x] : 0.0;
    t = wsum(t);
  }
  return t;   // valid in thread 0
}

// Stage 1: each block writes the sum of r^2 over the free DOFs of its rows.
__global__ void __launch_bounds__(NOALLOC_TPB) k_norm_partials(const double* __restrict__ r,
                                                               const int* __restrict__ rows, int nrow,
                                                               const uint8_t* __restrict__ fixed, int dim,
                                                               double* partial) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (row < nrow) {
    const long long i = rows[row];
    for (int a = 0; a < dim; ++a) {
      const double v = r[i * dim + a];
      if (!fixed[i * dim + a]) s += v * v;
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Stage 2: one block adds the partials (fixed order: deterministic).
__global__ void __launch_bounds__(NOALLOC_TPB) k_norm_total(double* partial, int nblk) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[NOALLOC_MAX_BLOCKS] = s;
}

// Device address of the scratch on the current device (set up on first use).
double* scratch_for_current_device(mpm_status* st) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    *st = MPM_ERR_CUDA;
    g_noalloc_err = std::string("no usable current device: ") + cudaGetErrorString(e);
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      *st = MPM_ERR_CUDA;
      g_noalloc_err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_scratch_addr[dev] = ptr;
  }
  *st = MPM_OK;
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" mpm_status mpm_residual_norm_noalloc(const double* r, const int* rows, int nrow,
                                                const unsigned char* fixed, int dim, double* out_norm,
                                                void* stream) {
  if ((long long)nrow > NOALLOC_MAX_ROWS) {
    g_noalloc_err = "nrow exceeds the allocation-free limit of " + std::to_string(NOALLOC_MAX_ROWS) +
                    " rows (8192 blocks of 256)";
    return MPM_ERR_INVALID_ARG;
  }
  if (!out_norm || (dim != 2 && dim != 3) || nrow < 0 || (nrow > 0 && (!r || !rows || !fixed))) {
    g_noalloc_err = "invalid argument (need device r, rows, fixed, a host out_norm, 2 or 3 values per node)";
    return MPM_ERR_INVALID_ARG;
  }
  mpm_status st;
  double* scratch = scratch_for_current_device(&st);
  if (!scratch) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (nrow + NOALLOC_TPB - 1) / NOALLOC_TPB;
  // An error left pending by earlier, unrelated work on this thread is
  // reported (and cleared) here, named as such, before anything is launched.
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_noalloc_err = std::string("CUDA error pending from earlier work on this thread: ") + cudaGetErrorString(e);
    return MPM_ERR_CUDA;
  }
  if (nblk > 0) {
    k_norm_partials<<<nblk, NOALLOC_TPB, 0, s>>>(r, rows, nrow, fixed, dim, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      g_noalloc_err = std::string("launch of k_norm_partials failed: ") + cudaGetErrorString(e);
      return MPM_ERR_CUDA;
    }
  }
  k_norm_total<<<1, NOALLOC_TPB, 0, s>>>(scratch, nblk);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_noalloc_err = std::string("launch of k_norm_total failed: ") + cudaGetErrorString(e);
    return MPM_ERR_CUDA;
  }
  double total = 0.0;
  e = cudaMemcpyAsync(&total, scratch + NOALLOC_MAX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    g_noalloc_err = std::string("CUDA error reading the norm back: ") + cudaGetErrorString(e);
    return MPM_ERR_CUDA;
  }
  *out_norm = sqrt(total);
  return MPM_OK;
}

extern "C" const char* mpm_noalloc_last_error(void) { return g_noalloc_err.c_str(); }
