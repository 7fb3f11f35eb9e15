// Krylov solver kernels for the Newton correction J d = -r (the paper solves
// this system with AMG/direct solvers on the CPU, Sec. 2.2 remark; here a
// block-Jacobi preconditioned BiCGStab and GMRES(m) run on the GPU).
//
// Vectors live on the dense node grid (nnode*D entries, padded on both sides
// by the stencil reach so that neighbour reads of boundary rows stay inside
// the allocation); only active rows are ever written.  The matrix is the
// stencil-BSR layout of mpm_internal.h: val[((slot*D + a)*D + b)*cap + row],
// one thread per row, fully coalesced value reads, no column indices.
//
// Scalars of the iteration stay on the device (KrylovScalars); every kernel
// returns at once when the solve is done, so the host can launch fixed-length
// CUDA-graph chunks of iterations and only poll the done flag between chunks.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int KTPB = 256;

template <int D>
__device__ __forceinline__ long long nbr(long long i, int dx, int dy, int dz, int nx1, int ny1) {
  return i + dx + (long long)nx1 * (dy + (long long)ny1 * dz);
}

// y = K x for one row (node i).
template <int D, class T>
__device__ __forceinline__ void spmv_row(const DevMatrix<T>& K, int row, long long i, int nx1, int ny1,
                                         const T* __restrict__ x, T y[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = (T)0;
  constexpr int ZR = (D == 3) ? 2 : 0;
  const long long cap = K.cap;
#pragma unroll
  for (int dz = -ZR; dz <= ZR; ++dz)
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
      for (int dx = -2; dx <= 2; ++dx) {
        const int slot = (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
        const long long j = nbr<D>(i, dx, dy, dz, nx1, ny1);
        T xj[D];
#pragma unroll
        for (int b = 0; b < D; ++b) xj[b] = __ldg(&x[j * D + b]);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b)
            y[a] += __ldg(&K.val[((long long)(slot * D + a) * D + b) * cap + row]) * xj[b];
      }
}

template <int D, class T>
__device__ __forceinline__ void precond_row(const DevMatrix<T>& K, int row, const T v[D], T z[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T s = (T)0;
#pragma unroll
    for (int b = 0; b < D; ++b) s += __ldg(&K.dinv[(long long)(a * D + b) * K.cap + row]) * v[b];
    z[a] = s;
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV partial sums and add them atomically to out[k].
template <int NV>
__device__ __forceinline__ void block_accumulate(double v[NV], double* const out[NV]) {
  __shared__ double sh[NV][KTPB / 32];
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
      double t = (lane < KTPB / 32) ? sh[k][lane] : 0.0;
      t = wsum(t);
      if (lane == 0 && t != 0.0) atomicAdd(out[k], t);
    }
  }
}

enum { KS_OK = 0, KS_MAXIT = 1, KS_BREAKDOWN = 2 };
}  // namespace

// ------------------------------------------------------------------ BiCGStab
// Right-preconditioned BiCGStab (van der Vorst 1992) on J d = b, d0 = 0.

template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_init(DevMatrix<T> K, const double* __restrict__ res,
                                                    const uint8_t* __restrict__ fixed, KrylovVecs<D, T> v,
                                                    KrylovScalars* S, double tol2, int maxit) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *K.nrow;
  double acc[2] = {0.0, 0.0};
  if (row < nrow) {
    const long long i = K.rows[row];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const long long d = i * D + a;
      T b = fixed[d] ? (T)0 : (T)(-res[d]);
      v.r[d] = b;
      v.rhat[d] = b;
      v.p[d] = (T)0;
      v.v[d] = (T)0;
      v.x[d] = (T)0;
      acc[0] += (double)b * (double)b;
    }
    acc[1] = acc[0];
  }
  double* outs[2] = {&S->acc_rr, &S->acc_rho};
  block_accumulate<2>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->rho = 1.0;
    S->alpha = 1.0;
    S->omega = 1.0;
    S->tol2 = tol2;
    S->maxit = maxit;
    S->iter = 0;
    S->done = 0;
    S->status = KS_OK;
  }
}

// K1: convergence test on ||r||^2, then p = r + beta (p - omega v), phat = M^-1 p.
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_1(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double rr = S->acc_rr;
  const int it = S->iter;
  const bool conv = rr <= S->tol2;
  const bool maxed = it >= S->maxit;
  const bool bad = it > 0 && (S->rho == 0.0 || S->omega == 0.0);
  if (conv || maxed || bad || !(rr == rr)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->done = 1;
      S->status = conv ? KS_OK : (maxed ? KS_MAXIT : KS_BREAKDOWN);
      S->rr_last = rr;
    }
    return;
  }
  const double beta = (it == 0) ? 0.0 : (S->acc_rho / S->rho) * (S->alpha / S->omega);
  const T tb = (T)beta, tw = (T)S->omega;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T p[D], z[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const long long d = i * D + a;
      p[a] = v.r[d] + tb * (v.p[d] - tw * v.v[d]);
      v.p[d] = p[a];
    }
    precond_row<D, T>(K, row, p, z);
#pragma unroll
    for (int a = 0; a < D; ++a) v.phat[i * D + a] = z[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) S->acc_rv = 0.0;
}

// K2: v = J phat; (rhat, v).
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_2(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[D];
    spmv_row<D, T>(K, row, i, G.nx1, G.ny1, v.phat, y);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v.v[i * D + a] = y[a];
      acc[0] += (double)v.rhat[i * D + a] * (double)y[a];
    }
  }
  double* outs[1] = {&S->acc_rv};
  block_accumulate<1>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->rho = S->acc_rho;   // rho_i = (rhat, r_i), consumed by K3 and the next K1
    S->acc_ts = 0.0;
    S->acc_tt = 0.0;
  }
}

// K3: alpha = rho / (rhat, v); s = r - alpha v; shat = M^-1 s.
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_3(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double rv = S->acc_rv;
  if (rv == 0.0 || !(rv == rv)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { S->done = 1; S->status = KS_BREAKDOWN; S->rr_last = S->acc_rr; }
    return;
  }
  const double alpha = S->rho / rv;
  const T ta = (T)alpha;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T s[D], z[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const long long d = i * D + a;
      s[a] = v.r[d] - ta * v.v[d];
      v.s[d] = s[a];
    }
    precond_row<D, T>(K, row, s, z);
#pragma unroll
    for (int a = 0; a < D; ++a) v.shat[i * D + a] = z[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = alpha;
    S->acc_rho = 0.0;
    S->acc_rr = 0.0;
  }
}

// K4: t = J shat; (t, s), (t, t).
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_4(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[D];
    spmv_row<D, T>(K, row, i, G.nx1, G.ny1, v.shat, y);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v.t[i * D + a] = y[a];
      acc[0] += (double)y[a] * (double)v.s[i * D + a];
      acc[1] += (double)y[a] * (double)y[a];
    }
  }
  double* outs[2] = {&S->acc_ts, &S->acc_tt};
  block_accumulate<2>(acc, outs);
}

// K5: omega = (t,s)/(t,t); x += alpha phat + omega shat; r = s - omega t;
// (rhat, r) and (r, r) for the next iteration.
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_bicg_5(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double tt = S->acc_tt;
  const double omega = (tt > 0.0) ? S->acc_ts / tt : 0.0;
  const T ta = (T)S->alpha, tw = (T)omega;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const long long d = i * D + a;
      v.x[d] += ta * v.phat[d] + tw * v.shat[d];
      T rn = v.s[d] - tw * v.t[d];
      v.r[d] = rn;
      acc[0] += (double)v.rhat[d] * (double)rn;
      acc[1] += (double)rn * (double)rn;
    }
  }
  double* outs[2] = {&S->acc_rho, &S->acc_rr};
  block_accumulate<2>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->omega = omega;
    S->iter = S->iter + 1;
  }
}

template <int D, class T>
cudaError_t launch_bicgstab_init(DevMatrix<T> K, const double* res, const uint8_t* fixed, KrylovVecs<D, T> v,
                                 KrylovScalars* S, double tol2, int maxit, int nblk, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(KrylovScalars), st);
  if (e != cudaSuccess) return e;
  k_bicg_init<D, T><<<nblk, KTPB, 0, st>>>(K, res, fixed, v, S, tol2, maxit);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_bicgstab_iter(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                 int nblk, cudaStream_t st) {
  k_bicg_1<D, T><<<nblk, KTPB, 0, st>>>(K, v, S);
  k_bicg_2<D, T><<<nblk, KTPB, 0, st>>>(G, K, v, S);
  k_bicg_3<D, T><<<nblk, KTPB, 0, st>>>(K, v, S);
  k_bicg_4<D, T><<<nblk, KTPB, 0, st>>>(G, K, v, S);
  k_bicg_5<D, T><<<nblk, KTPB, 0, st>>>(K, v, S);
  return cudaGetLastError();
}

// du = base + alpha d on the free DOFs (the halved step of a Newton iteration
// whose full step drove a return map out of its domain).
template <int D, class T>
__global__ void k_step_du(DevMatrix<T> K, const T* __restrict__ x, const uint8_t* __restrict__ fixed,
                          const double* __restrict__ base, double* du, double alpha) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const long long i = K.rows[row];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const long long d = i * D + a;
    if (!fixed[d]) du[d] = base[d] + alpha * (double)x[d];
  }
}
template <int D, class T>
cudaError_t launch_step_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, const double* base, double* du,
                           double alpha, int nblk, cudaStream_t st) {
  k_step_du<D, T><<<nblk, KTPB, 0, st>>>(K, x, fixed, base, du, alpha);
  return cudaGetLastError();
}

// Plain y = J x over the active rows (used to time the product in isolation).
template <int D, class T>
__global__ void __launch_bounds__(KTPB) k_spmv(DevGrid G, DevMatrix<T> K, const T* __restrict__ x, T* y) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const long long i = K.rows[row];
  T v[D];
  spmv_row<D, T>(K, row, i, G.nx1, G.ny1, x, v);
#pragma unroll
  for (int a = 0; a < D; ++a) y[i * D + a] = v[a];
}
template <int D, class T>
cudaError_t launch_spmv(const DevGrid& G, DevMatrix<T> K, const T* x, T* y, int nblk, cudaStream_t st) {
  k_spmv<D, T><<<nblk, KTPB, 0, st>>>(G, K, x, y);
  return cudaGetLastError();
}

// du += d on the free DOFs of active rows (FP64 accumulation of the update).
template <int D, class T>
__global__ void k_update_du(DevMatrix<T> K, const T* __restrict__ x, const uint8_t* __restrict__ fixed,
                            double* du) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const long long i = K.rows[row];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const long long d = i * D + a;
    if (!fixed[d]) du[d] += (double)x[d];
  }
}
template <int D, class T>
cudaError_t launch_update_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, double* du, int nblk,
                             cudaStream_t st) {
  k_update_du<D, T><<<nblk, KTPB, 0, st>>>(K, x, fixed, du);
  return cudaGetLastError();
}

#define MPM_KRYLOV_INST(D, T)                                                                          \
  template cudaError_t launch_bicgstab_init<D, T>(DevMatrix<T>, const double*, const uint8_t*,          \
                                                  KrylovVecs<D, T>, KrylovScalars*, double, int, int,   \
                                                  cudaStream_t);                                        \
  template cudaError_t launch_bicgstab_iter<D, T>(const DevGrid&, DevMatrix<T>, KrylovVecs<D, T>,       \
                                                  KrylovScalars*, int, cudaStream_t);                   \
  template cudaError_t launch_update_du<D, T>(DevMatrix<T>, const T*, const uint8_t*, double*, int,     \
                                              cudaStream_t);                                            \
  template cudaError_t launch_spmv<D, T>(const DevGrid&, DevMatrix<T>, const T*, T*, int, cudaStream_t);  \
  template cudaError_t launch_step_du<D, T>(DevMatrix<T>, const T*, const uint8_t*, const double*, double*, \
                                            double, int, cudaStream_t);
MPM_KRYLOV_INST(2, float)
MPM_KRYLOV_INST(2, double)
MPM_KRYLOV_INST(3, float)
MPM_KRYLOV_INST(3, double)

}  // namespace mpm
