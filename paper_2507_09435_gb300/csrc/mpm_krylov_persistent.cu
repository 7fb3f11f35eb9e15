// Persistent (cooperative) BiCGStab: the whole right-preconditioned
// BiCGStab solve of J d = -r runs as ONE kernel launch per Newton iteration.
// Its five phases per iteration are separated by a grid barrier instead of
// kernel boundaries, removing the per-kernel launch and drain latency of the
// multi-kernel form.
//
//  * Grid barrier: a monotonic arrival counter (zeroed at launch); one
//    release-add per block, acquire-reads while waiting, no reset between
//    barriers.  Every spin is bounded (about a second): on timeout the block
//    raises ERRF_BARRIER and returns; every other block then returns at its
//    next barrier.  Launched with cudaLaunchCooperativeKernel, so all blocks
//    are co-resident.
//  * Memory ordering: vectors written inside the kernel are read with
//    ordinary (weak) loads after the barrier; the release-add / acquire-read
//    pair plus __syncthreads orders them after the writes of every block
//    (PTX memory model), so they may use L1.  The matrix, the block-Jacobi
//    inverse and rhat, constant over the kernel, use the read-only path.
//  * Dot products: block sums, then one atomic add per block into an
//    accumulator that is zeroed two barriers away from both its last read
//    and its next accumulation.  Every block reads the same accumulated
//    value after the barrier, so all blocks take identical decisions.
#include <algorithm>

#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int PTPB = 512;
constexpr int RSPLIT = 4;     // threads per row in the products

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Add the block's sums of NV values to out[k] (one atomic per block and value).
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
}

__device__ __forceinline__ unsigned int atom_add_release(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier number `epoch` completes when the counter reaches (epoch+1)*nblocks.
// Returns false when the wait timed out (the caller returns).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err,
                                             unsigned int& epoch) {
  __syncthreads();
  __shared__ int timed_out;
  if (threadIdx.x == 0) {
    timed_out = 0;
    atom_add_release(bar, 1u);
    const unsigned int target = (epoch + 1u) * nblocks;
    // each acquire read goes to L2 (a few hundred ns), so 2^22 reads bound
    // the wait at roughly one to two seconds
    unsigned int spins = 0;
    while (ld_acquire(bar) < target) {
      if (++spins > (1u << 22)) {
        atomicOr(err, ERRF_BARRIER);
        timed_out = 1;
        break;
      }
    }
  }
  ++epoch;
  __syncthreads();
  return !timed_out && !(*(volatile int*)err & ERRF_BARRIER);
}

// Partial product of one row over the slots sub, sub+RSPLIT, ...; s_off holds
// the node offset of every slot (shared memory, filled once per block).
template <int D, class T>
__device__ __forceinline__ void spmv_part(const DevMatrix<T>& K, int row, long long i, int sub,
                                          const int* s_off, const T* x, T y[D]) {
  constexpr int S = (D == 2) ? 25 : 125;
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = (T)0;
  const T* base = K.val + (long long)row * (D * D);
  const long long plane = (long long)K.cap * (D * D);
  unsigned pm[pmask_words(D)];
  load_pmask<D>(K.pmask, row, pm);
#pragma unroll 4
  for (int slot = sub; slot < S; slot += RSPLIT) {
    if (!((pm[slot >> 5] >> (slot & 31)) & 1u)) continue;
    T xj[D], kb[D * D];
    ld_node<D, T, true>(x, i + s_off[slot], xj);
    ld_block<D, T>(base + slot * plane, kb);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) y[a] += kb[a * D + b] * xj[b];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = RSPLIT / 2; o > 0; o >>= 1) y[a] += __shfl_xor_sync(0xffffffffu, y[a], o);
  }
}

template <int D, class T>
__device__ __forceinline__ void precond(const DevMatrix<T>& K, int row, const T v[D], T z[D]) {
  T m[D * D];
  ld_block<D, T>(&K.dinv[(long long)row * (D * D)], m);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T s = (T)0;
#pragma unroll
    for (int b = 0; b < D; ++b) s += m[a * D + b] * v[b];
    z[a] = s;
  }
}
}  // namespace

// S must hold what k_bicg_init leaves: rr_last = (r,r), rho = (rhat, r),
// tol2, maxit, and zero accumulators.  bar is zeroed by the launcher.
template <int D, class T>
__global__ void __launch_bounds__(PTPB) k_bicg_persistent(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v,
                                                          KrylovScalars* S, double* part, unsigned int* bar,
                                                          int* err) {
  (void)part;
  const unsigned int nb = gridDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const int nrow = *K.nrow;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  constexpr int NSLOT = (D == 2) ? 25 : 125;
  __shared__ int s_off[NSLOT];
  for (int slot = threadIdx.x; slot < NSLOT; slot += blockDim.x) {
    const int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
    s_off[slot] = dx + G.nx1 * (dy + G.ny1 * dz);
  }
  __syncthreads();
  volatile KrylovScalars* VS = S;
  const double tol2 = VS->tol2;
  const int maxit = VS->maxit;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int status = 0;
  int it = 0;
  unsigned int epoch = 0;
  double rr = VS->acc_rr;
  for (;; ++it) {
    // ---- P1: convergence test; p = r + beta (p - omega v); phat = M^-1 p
    // (the first iteration takes (rhat, r0) and (r0, r0) from the init kernel)
    const double rho_new = (it == 0) ? VS->rho : VS->acc_rho;
    rr = (it == 0) ? VS->rr_last : VS->acc_rr;
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
        T p[D], z[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          p[a] = v.r[d] + tb * (v.p[d] - tw * v.v[d]);
          v.p[d] = p[a];
        }
        precond<D, T>(K, (int)row, p, z);
#pragma unroll
        for (int a = 0; a < D; ++a) v.phat[i * D + a] = z[a];
      }
    }
    rho = rho_new;
    if (lead) S->acc_ts = 0.0, S->acc_tt = 0.0;   // last read in P5 of the previous iteration
    if (!grid_barrier(bar, nb, err, epoch)) return;
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
        spmv_part<D, T>(K, row, i, live ? sub : 1000, s_off, v.phat, y);
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
    }
    if (!grid_barrier(bar, nb, err, epoch)) return;
    // ---- P3: alpha = rho / (rhat, v); s = r - alpha v; shat = M^-1 s
    {
      const double rv = VS->acc_rv;
      if (rv == 0.0 || !(rv == rv)) {
        status = 2;
        break;
      }
      alpha = rho / rv;
      const T ta = (T)alpha;
      for (long long row = gtid; row < nrow; row += gsz) {
        const long long i = K.rows[row];
        T s[D], z[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          s[a] = v.r[d] - ta * v.v[d];
          v.s[d] = s[a];
        }
        precond<D, T>(K, (int)row, s, z);
#pragma unroll
        for (int a = 0; a < D; ++a) v.shat[i * D + a] = z[a];
      }
      if (lead) S->acc_rho = 0.0, S->acc_rr = 0.0;   // last read in P1
    }
    if (!grid_barrier(bar, nb, err, epoch)) return;
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
        spmv_part<D, T>(K, row, i, live ? sub : 1000, s_off, v.shat, y);
        if (live && sub == 0) {
#pragma unroll
          for (int a = 0; a < D; ++a) {
            v.t[i * D + a] = y[a];
            const double sv = (double)v.s[i * D + a];
            acc[0] += (double)y[a] * sv;
            acc[1] += (double)y[a] * (double)y[a];
          }
        }
      }
      double* outs[2] = {&S->acc_ts, &S->acc_tt};
      block_add<2>(acc, outs);
      if (lead) S->acc_rv = 0.0;   // last read in P3
    }
    if (!grid_barrier(bar, nb, err, epoch)) return;
    // ---- P5: omega; x += alpha phat + omega shat; r = s - omega t; (rhat,r), (r,r)
    {
      const double tt = VS->acc_tt;
      omega = (tt > 0.0) ? VS->acc_ts / tt : 0.0;
      const T ta = (T)alpha, tw = (T)omega;
      double acc[2] = {0.0, 0.0};
      for (long long row = gtid; row < nrow; row += gsz) {
        const long long i = K.rows[row];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const long long d = i * D + a;
          v.x[d] = v.x[d] + ta * v.phat[d] + tw * v.shat[d];
          const T rn = v.s[d] - tw * v.t[d];
          v.r[d] = rn;
          acc[0] += (double)__ldg(&v.rhat[d]) * (double)rn;
          acc[1] += (double)rn * (double)rn;
        }
      }
      double* outs[2] = {&S->acc_rho, &S->acc_rr};
      block_add<2>(acc, outs);
    }
    if (!grid_barrier(bar, nb, err, epoch)) return;
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
