// Persistent (cooperative) BiCGStab: the whole right-preconditioned
// BiCGStab solve of J d = -r runs as ONE kernel launch per Newton iteration.
// Its five phases per iteration are separated by a grid barrier instead of
// kernel boundaries, removing the per-kernel launch and drain latency that
// dominates the multi-kernel form on L2-resident 2D problems.
//
// Grid barrier: sense-counting on a global counter and generation word, with
// a bounded spin (about a second): on timeout the block raises ERRF_BARRIER,
// and every block returns at its next barrier.  The kernel is launched with
// cudaLaunchCooperativeKernel so that all blocks are co-resident.
//
// Coherence: vectors written inside the kernel are read with ld.global.cg
// (L2, not the non-coherent L1); the matrix, the block-Jacobi inverse and
// rhat, constant during the solve, use the read-only path.
#include <algorithm>

#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int PTPB = 256;
constexpr int RSPLIT = 4;   // threads per row in the products

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Returns false when the barrier timed out (every block then exits).
__device__ __forceinline__ bool grid_barrier(GridBarrier* b, unsigned int nblocks, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &b->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned int spins = 0;
      while (*vgen == g) {
        if (++spins > (1u << 25)) {
          atomicOr(err, ERRF_BARRIER);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0 || !(*(volatile int*)err & ERRF_BARRIER);
}

template <int NV>
__device__ __forceinline__ void block_add(double v[NV], double* const out[NV]) {
  __shared__ double sh[NV][PTPB / 32];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = wsum(v[k]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = (lane < PTPB / 32) ? sh[k][lane] : 0.0;
      t = wsum(t);
      if (lane == 0 && t != 0.0) atomicAdd(out[k], t);
    }
  }
  __syncthreads();
}

// Partial product of one row over the slots sub, sub+RSPLIT, ...: the caller
// reduces the RSPLIT partials with shuffles.
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
}

template <int D, class T>
__device__ __forceinline__ void reduce_split(T y[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = RSPLIT / 2; o > 0; o >>= 1) y[a] += __shfl_xor_sync(0xffffffffu, y[a], o);
  }
}
}  // namespace

// S must hold the state k_bicg_init leaves (accumulators of (r,r), (rhat,r),
// rho = alpha = omega = 1, iter = 0, tol2, maxit).
template <int D, class T>
__global__ void __launch_bounds__(PTPB) k_bicg_persistent(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v,
                                                          KrylovScalars* S, GridBarrier* bar, int* err) {
  const unsigned int nb = gridDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const int nrow = *K.nrow;
  volatile KrylovScalars* VS = S;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  for (;;) {
    // ---- P1: convergence test; p = r + beta (p - omega v); phat = M^-1 p
    const double rr = VS->acc_rr;
    const int it = VS->iter;
    const bool conv = rr <= VS->tol2;
    const bool maxed = it >= VS->maxit;
    const bool bad = (it > 0 && (VS->rho == 0.0 || VS->omega == 0.0)) || !(rr == rr);
    if (conv || maxed || bad) {
      if (lead) {
        S->done = 1;
        S->status = conv ? 0 : (maxed ? 1 : 2);
        S->rr_last = rr;
      }
      return;
    }
    {
      const double beta = (it == 0) ? 0.0 : (VS->acc_rho / VS->rho) * (VS->alpha / VS->omega);
      const T tb = (T)beta, tw = (T)VS->omega;
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
      if (lead) S->acc_rv = 0.0;
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P2: v = J phat; (rhat, v)
    {
      double acc[1] = {0.0};
      const long long items = (long long)nrow * RSPLIT;
      const long long span = ((items + gsz - 1) / gsz) * gsz;   // every lane runs the same trip count
      for (long long w = gtid; w < span; w += gsz) {
        const bool live = w < items;
        const int row = live ? (int)(w / RSPLIT) : 0;
        const int sub = (int)(w % RSPLIT);
        const long long i = live ? K.rows[row] : 0;
        T y[D];
        if (live) spmv_part<D, T>(K, row, i, sub, G.nx1, G.ny1, v.phat, y);
        else {
#pragma unroll
          for (int a = 0; a < D; ++a) y[a] = (T)0;
        }
        reduce_split<D, T>(y);
        if (live && sub == 0) {
#pragma unroll
          for (int a = 0; a < D; ++a) {
            v.v[i * D + a] = y[a];
            acc[0] += (double)__ldg(&v.rhat[i * D + a]) * (double)y[a];
          }
        }
      }
      double* outs[1] = {&S->acc_rv};
      block_add<1>(acc, outs);
      if (lead) {
        S->rho = VS->acc_rho;
        S->acc_ts = 0.0;
        S->acc_tt = 0.0;
      }
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P3: alpha = rho / (rhat, v); s = r - alpha v; shat = M^-1 s
    {
      const double rv = VS->acc_rv;
      if (rv == 0.0 || !(rv == rv)) {
        if (lead) { S->done = 1; S->status = 2; S->rr_last = VS->acc_rr; }
        return;
      }
      const double alpha = VS->rho / rv;
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
      if (lead) {
        S->alpha = alpha;
        S->acc_rho = 0.0;
        S->acc_rr = 0.0;
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
        if (live) spmv_part<D, T>(K, row, i, sub, G.nx1, G.ny1, v.shat, y);
        else {
#pragma unroll
          for (int a = 0; a < D; ++a) y[a] = (T)0;
        }
        reduce_split<D, T>(y);
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
      double* outs[2] = {&S->acc_ts, &S->acc_tt};
      block_add<2>(acc, outs);
    }
    if (!grid_barrier(bar, nb, err)) return;
    // ---- P5: omega; x += alpha phat + omega shat; r = s - omega t; (rhat,r), (r,r)
    {
      const double tt = VS->acc_tt;
      const double omega = (tt > 0.0) ? VS->acc_ts / tt : 0.0;
      const T ta = (T)VS->alpha, tw = (T)omega;
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
      double* outs[2] = {&S->acc_rho, &S->acc_rr};
      block_add<2>(acc, outs);
      if (lead) {
        S->omega = omega;
        S->iter = it + 1;
      }
    }
    if (!grid_barrier(bar, nb, err)) return;
  }
}

template <int D, class T>
int persistent_blocks(int device) {
  int nsm = 0, per = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bicg_persistent<D, T>, PTPB, 0) != cudaSuccess) return 0;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (!coop) return 0;
  return nsm * std::min(per, 2);
}

template <int D, class T>
cudaError_t launch_bicgstab_persistent(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                       GridBarrier* bar, int* err, int nblocks, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  DevGrid g = G;
  void* args[] = {&g, &K, &v, &S, &bar, &err};
  return cudaLaunchCooperativeKernel((void*)k_bicg_persistent<D, T>, dim3(nblocks), dim3(PTPB), args, 0, st);
}

#define MPM_PERSIST_INST(D, T)                                                                          \
  template int persistent_blocks<D, T>(int);                                                            \
  template cudaError_t launch_bicgstab_persistent<D, T>(const DevGrid&, DevMatrix<T>, KrylovVecs<D, T>, \
                                                        KrylovScalars*, GridBarrier*, int*, int, cudaStream_t);
MPM_PERSIST_INST(2, float)
MPM_PERSIST_INST(2, double)
MPM_PERSIST_INST(3, float)
MPM_PERSIST_INST(3, double)

}  // namespace mpm
