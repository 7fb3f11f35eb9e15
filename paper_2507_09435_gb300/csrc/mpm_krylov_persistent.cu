// Persistent (cooperative) BiCGStab: the whole right-preconditioned
// BiCGStab solve of J d = -r runs as ONE kernel launch per Newton iteration.
// Its five phases per iteration are separated by a grid barrier instead of
// kernel boundaries, removing the per-kernel launch and drain latency that
// dominates the multi-kernel form on L2-resident 2D problems.
//
// Same-address atomics are what makes a naive grid-wide form slow (every
// barrier and every dot product serialises one atomic per block on one L2
// line), so:
//  * dot products are deterministic two-level sums: each block writes its
//    partial to its own slot; after the barrier every block adds all slots in
//    the same order, so every block holds bit-identical scalars (alpha, beta,
//    omega, the convergence test) without any further communication;
//  * the grid barrier is a two-level tree: blocks arrive on one of NGROUP
//    counters (each on its own 128-byte line), the last arrival of a group
//    arrives on the root, the last root arrival advances the generation word.
// Every spin is bounded (about a second): on timeout the block raises
// ERRF_BARRIER and returns; every other block then returns at its next
// barrier.  Launched with cudaLaunchCooperativeKernel (all blocks co-resident).
//
// Coherence: vectors written inside the kernel are read with ld.global.cg
// (L2, not the non-coherent L1); the matrix, the block-Jacobi inverse and
// rhat, constant during the solve, use the read-only path.
#include <algorithm>

#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int PTPB = 512;
constexpr int RSPLIT = 4;     // threads per row in the products
constexpr int NGROUP = 16;    // barrier tree fan-in groups
constexpr int LINE = 32;      // unsigned ints per 128-byte line

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values; the result is returned to every thread.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV]) {
  __shared__ double sh[NV][PTPB / 32];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = wsum(v[k]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = (lane < PTPB / 32) ? sh[k][lane] : 0.0;
    v[k] = wsum(t);
  }
  __syncthreads();
}

// Write this block's NV partials to part[k*stride + block].
template <int NV>
__device__ __forceinline__ void publish(double v[NV], double* part, int stride) {
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * stride + blockIdx.x] = v[k];
  }
}

// Every block: sum the NV partial arrays in a fixed order (bitwise identical
// in all blocks).
template <int NV>
__device__ __forceinline__ void gather(const double* part, int stride, int nb, double out[NV]) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  // thread t adds blocks t, t + PTPB, ... ; the block sum then fixes the order
  for (int b = threadIdx.x; b < nb; b += PTPB) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(&part[k * stride + b]);
  }
  block_sum<NV>(v);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = v[k];
}

// Returns false when a barrier timed out (the caller returns).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err) {
  __syncthreads();
  __shared__ int timed_out;
  if (threadIdx.x == 0) {
    timed_out = 0;
    volatile unsigned int* vgen = &bar[(NGROUP + 1) * LINE];
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int grp = blockIdx.x % NGROUP;
    const unsigned int gsize = (nblocks - grp + NGROUP - 1) / NGROUP;
    const unsigned int ngroups = nblocks < NGROUP ? nblocks : NGROUP;
    bool last = false;
    if (atomicAdd(&bar[grp * LINE], 1u) + 1u == gsize) {
      atomicExch(&bar[grp * LINE], 0u);
      if (atomicAdd(&bar[NGROUP * LINE], 1u) + 1u == ngroups) {
        atomicExch(&bar[NGROUP * LINE], 0u);
        __threadfence();
        atomicAdd((unsigned int*)vgen, 1u);
        last = true;
      }
    }
    if (!last) {
      unsigned int spins = 0;
      while (*vgen == g) {
        if (++spins > (1u << 25)) {
          atomicOr(err, ERRF_BARRIER);
          timed_out = 1;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !timed_out && !(*(volatile int*)err & ERRF_BARRIER);
}

// Partial product of one row over the slots sub, sub+RSPLIT, ...
template <int D, class T>
__device__ __forceinline__ void spmv_part(const DevMatrix<T>& K, int row, long long i, int sub, int nx1,
                                          int ny1, const T* x, T y[D]) {
  constexpr int S = (D == 2) ? 25 : 125;
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = (T)0;
  const long long cap = K.cap;
#pragma unroll 4
  for (int slot = sub; slot < S; slot += RSPLIT) {
    const int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
    const long long j = i + dx + (long long)nx1 * (dy + (long long)ny1 * dz);
    T xj[D];
#pragma unroll
    for (int b = 0; b < D; ++b) xj[b] = __ldcg(&x[j * D + b]);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) y[a] += __ldg(&K.val[((long long)(slot * D + a) * D + b) * cap + row]) * xj[b];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = RSPLIT / 2; o > 0; o >>= 1) y[a] += __shfl_xor_sync(0xffffffffu, y[a], o);
  }
}

// partial-slot arrays: index k * PSTRIDE + block
constexpr int P_RV = 0, P_TS = 1, P_TT = 2, P_RHO = 3, P_RR = 4;
}  // namespace

// S must hold what k_bicg_init leaves: acc_rr = (r,r), acc_rho = (rhat, r),
// tol2, maxit.  part holds 5 * PERSIST_MAX_BLOCKS doubles; bar the barrier
// words (zeroed by the launcher).
template <int D, class T>
__global__ void __launch_bounds__(PTPB) k_bicg_persistent(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v,
                                                          KrylovScalars* S, double* part, unsigned int* bar,
                                                          int* err) {
  constexpr int PS = PERSIST_MAX_BLOCKS;
  const unsigned int nb = gridDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const int nrow = *K.nrow;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const double tol2 = S->tol2;
  const int maxit = S->maxit;
  // scalars, identical in every block
  double rr = S->acc_rr, rho_new = S->acc_rho;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int status = 0;
  int it = 0;
  for (;; ++it) {
    // ---- P1: convergence test; p = r + beta (p - omega v); phat = M^-1 p
    const bool conv = rr <= tol2;
    const bool maxed = it >= maxit;
    const bool bad = (it > 0 && (rho == 0.0 || omega == 0.0)) || !(rr == rr);
    if (conv || maxed || bad) {
      status = conv ? 0 : (maxed ? 1 : 2);
      break;
    }
    {
      const double beta = (it == 0) ? 0.0 : (rho_new / rho) * (alpha / omega);
      const T tb = (T)beta, tw = (T)omega;
      for (long long row = gtid; row < nrow; row += gsz) {
        const long long i = K.rows[row];
        T p[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          p[a] = __ldcg(&v.r[d]) + tb * (__ldcg(&v.p[d]) - tw * __ldcg(&v.v[d]));
          v.p[d] = p[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          T z = (T)0;
#pragma unroll
          for (int b = 0; b < D; ++b) z += __ldg(&K.dinv[(long long)(a * D + b) * K.cap + row]) * p[b];
          v.phat[i * D + a] = z;
        }
      }
    }
    rho = rho_new;
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P2: v = J phat; (rhat, v)
    {
      double acc[1] = {0.0};
      const long long items = (long long)nrow * RSPLIT;
      const long long span = ((items + gsz - 1) / gsz) * gsz;   // same trip count in every lane
      for (long long w = gtid; w < span; w += gsz) {
        const bool live = w < items;
        const int row = live ? (int)(w / RSPLIT) : 0;
        const int sub = (int)(w % RSPLIT);
        const long long i = live ? K.rows[row] : 0;
        T y[D];
        spmv_part<D, T>(K, row, i, live ? sub : 1000, G.nx1, G.ny1, v.phat, y);
        if (live && sub == 0) {
#pragma unroll
          for (int a = 0; a < D; ++a) {
            v.v[i * D + a] = y[a];
            acc[0] += (double)__ldg(&v.rhat[i * D + a]) * (double)y[a];
          }
        }
      }
      publish<1>(acc, part + P_RV * PS, PS);
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P3: alpha = rho / (rhat, v); s = r - alpha v; shat = M^-1 s
    {
      double rv[1];
      gather<1>(part + P_RV * PS, PS, nb, rv);
      if (rv[0] == 0.0 || !(rv[0] == rv[0])) {
        status = 2;
        break;
      }
      alpha = rho / rv[0];
      const T ta = (T)alpha;
      for (long long row = gtid; row < nrow; row += gsz) {
        const long long i = K.rows[row];
        T s[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          s[a] = __ldcg(&v.r[d]) - ta * __ldcg(&v.v[d]);
          v.s[d] = s[a];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          T z = (T)0;
#pragma unroll
          for (int b = 0; b < D; ++b) z += __ldg(&K.dinv[(long long)(a * D + b) * K.cap + row]) * s[b];
          v.shat[i * D + a] = z;
        }
      }
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P4: t = J shat; (t, s), (t, t)
    {
      double acc[2] = {0.0, 0.0};
      const long long items = (long long)nrow * RSPLIT;
      const long long span = ((items + gsz - 1) / gsz) * gsz;
      for (long long w = gtid; w < span; w += gsz) {
        const bool live = w < items;
        const int row = live ? (int)(w / RSPLIT) : 0;
        const int sub = (int)(w % RSPLIT);
        const long long i = live ? K.rows[row] : 0;
        T y[D];
        spmv_part<D, T>(K, row, i, live ? sub : 1000, G.nx1, G.ny1, v.shat, y);
        if (live && sub == 0) {
#pragma unroll
          for (int a = 0; a < D; ++a) {
            v.t[i * D + a] = y[a];
            const double sv = (double)__ldcg(&v.s[i * D + a]);
            acc[0] += (double)y[a] * sv;
            acc[1] += (double)y[a] * (double)y[a];
          }
        }
      }
      publish<2>(acc, part + P_TS * PS, PS);
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P5: omega; x += alpha phat + omega shat; r = s - omega t; (rhat,r), (r,r)
    {
      double tsn[2];
      gather<2>(part + P_TS * PS, PS, nb, tsn);
      omega = (tsn[1] > 0.0) ? tsn[0] / tsn[1] : 0.0;
      const T ta = (T)alpha, tw = (T)omega;
      double acc[2] = {0.0, 0.0};
      for (long long row = gtid; row < nrow; row += gsz) {
        const long long i = K.rows[row];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          v.x[d] = __ldcg(&v.x[d]) + ta * __ldcg(&v.phat[d]) + tw * __ldcg(&v.shat[d]);
          const T rn = __ldcg(&v.s[d]) - tw * __ldcg(&v.t[d]);
          v.r[d] = rn;
          acc[0] += (double)__ldg(&v.rhat[d]) * (double)rn;
          acc[1] += (double)rn * (double)rn;
        }
      }
      publish<2>(acc, part + P_RHO * PS, PS);
    }
    if (!grid_barrier(bar, nb, err)) return;
    {
      double rr2[2];
      gather<2>(part + P_RHO * PS, PS, nb, rr2);
      rho_new = rr2[0];
      rr = rr2[1];
    }
  }
  if (lead) {
    S->done = 1;
    S->status = status;
    S->rr_last = rr;
    S->iter = it;
    S->rho = rho;
    S->alpha = alpha;
    S->omega = omega;
  }
}

template <int D, class T>
int persistent_blocks(int device) {
  int nsm = 0, per = 0, coop = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bicg_persistent<D, T>, PTPB, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) return 0;
  if (per < 1) return 0;
  return std::min(nsm, PERSIST_MAX_BLOCKS);   // one block per SM
}

template <int D, class T>
cudaError_t launch_bicgstab_persistent(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                       double* part, unsigned int* bar, int* err, int nblocks, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, PERSIST_BAR_WORDS * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  DevGrid g = G;
  void* args[] = {&g, &K, &v, &S, &part, &bar, &err};
  return cudaLaunchCooperativeKernel((void*)k_bicg_persistent<D, T>, dim3(nblocks), dim3(PTPB), args, 0, st);
}

#define MPM_PERSIST_INST(D, T)                                                                          \
  template int persistent_blocks<D, T>(int);                                                            \
  template cudaError_t launch_bicgstab_persistent<D, T>(const DevGrid&, DevMatrix<T>, KrylovVecs<D, T>, \
                                                        KrylovScalars*, double*, unsigned int*, int*,   \
                                                        int, cudaStream_t);
MPM_PERSIST_INST(2, float)
MPM_PERSIST_INST(2, double)
MPM_PERSIST_INST(3, float)
MPM_PERSIST_INST(3, double)

}  // namespace mpm
