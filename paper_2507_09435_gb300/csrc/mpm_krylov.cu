// Krylov solver kernels for the Newton correction J d = -r (the paper solves
// this system with AMG/direct solvers on the CPU, Sec. 2.2 remark; here a
// block-Jacobi preconditioned BiCGStab runs on the GPU).
//
// Vectors live on the dense node grid (nnode*B entries, B values per node:
// the D displacements, plus the pore pressure for u-p; padded on both sides
// by the stencil reach so that neighbour reads of boundary rows stay inside
// the allocation); only active rows are ever written.  The matrix is the
// stencil-BSR layout of mpm_internal.h: val[(slot*cap + row)*B*B + a*B + b],
// one thread per row, coalesced block reads, no column indices.
//
// Scalars of the iteration stay on the device (KrylovScalars); every kernel
// returns at once when the solve is done, so the host can launch fixed-length
// CUDA-graph chunks of iterations and only poll the done flag between chunks.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int KTPB = KRYLOV_TPB;

template <int D>
__device__ __forceinline__ long long nbr(long long i, int dx, int dy, int dz, int nx1, int ny1) {
  return i + dx + (long long)nx1 * (dy + (long long)ny1 * dz);
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
// Right-preconditioned BiCGStab (van der Vorst 1992) on J d = b, d0 = 0, in a
// merged-reduction form with four kernels per iteration:
//   B: v = J phat, (rhat, v)
//   C: alpha = rho/(rhat,v); s = r - alpha v; shat = M^-1 s; (s,s), (rhat,s)
//   D: t = J shat; (t,s), (t,t), (rhat,t)
//   A: omega = (t,s)/(t,t); x += alpha phat + omega shat; r = s - omega t;
//      rho' = (rhat,s) - omega (rhat,t); ||r||^2 = (s,s) - 2 omega (t,s) +
//      omega^2 (t,t); beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v);
//      phat = M^-1 p.
// The two dot products of the classical form's last step follow from the
// ones already reduced, so the update and the next search direction share one
// pass.  (FP32 products are exact in FP64 and summed in FP64, which keeps the
// cancellation in ||r||^2 harmless at the linear tolerances used.)
// A kernel's lead thread never writes a field that other blocks of the same
// kernel read: rho is read in C and written in A; C copies it to rho_old,
// which A reads; iter is read in B and advanced in D; each accumulator is
// zeroed in a kernel that neither produces nor consumes it.

// init: r = b, rhat = b, x = 0, p = r, phat = M^-1 r; rho = (rhat, r),
// rr_last = (r, r).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_init(DevMatrix<T> K, const double* __restrict__ res,
                                                    const uint8_t* __restrict__ fixed, KrylovVecs<D, T> v,
                                                    KrylovScalars* S, double tol2, int maxit) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *K.nrow;
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  double acc[2] = {0.0, 0.0};
  if (row < nrow) {
    const long long i = K.rows[row];
    T b[B], z[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      b[a] = fixed[d] ? (T)0 : (T)(-res[d]);
      v.r[d] = b[a];
      v.rhat[d] = b[a];
      v.p[d] = b[a];
      v.x[d] = (T)0;
      acc[0] += (double)b[a] * (double)b[a];
    }
    precond_apply<B, T>(K, row, b, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
    acc[1] = acc[0];
  }
  double acc3[3] = {acc[0], acc[1], acc[0]};
  double* outs[3] = {&S->rr_last, &S->rho, &S->rhat2};
  block_accumulate<3>(acc3, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = 1.0;
    S->omega = 1.0;
    S->tol2 = tol2;
    S->maxit = maxit;
    S->iter = 0;
    S->done = 0;
    S->status = KS_OK;
  }
}

// B: convergence / limit test, then v = J phat and (rhat, v).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_B(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double rr = S->rr_last;
  const int it = S->iter;
  const bool conv = rr <= S->tol2;
  const bool maxed = it >= S->maxit;
  const bool bad = !(rr == rr) || (it > 0 && (S->rho == 0.0 || S->omega == 0.0));
  if (conv || maxed || bad) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->done = 1;
      S->status = conv ? KS_OK : (maxed ? KS_MAXIT : KS_BREAKDOWN);
    }
    return;
  }
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, v.phat, y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      v.v[i * B + a] = y[a];
      acc[0] += (double)v.rhat[i * B + a] * (double)y[a];
      acc[1] += (double)y[a] * (double)y[a];
    }
  }
  double* outs[2] = {&S->acc_rv, &S->acc_vv};
  block_accumulate<2>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->acc_ss = 0.0;
    S->acc_rs = 0.0;
  }
}

// C: alpha = rho / (rhat, v); s = r - alpha v; shat = M^-1 s; (s,s), (rhat,s).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_C(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double rv = S->acc_rv;
  // (near) breakdown: rhat and v almost orthogonal, relative to FP32 vectors
  if (!(fabs(rv) > 1e-7 * sqrt(S->acc_vv * S->rhat2))) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { S->done = 1; S->status = KS_BREAKDOWN; }
    return;
  }
  const double rho = S->rho;
  const double alpha = rho / rv;
  const T ta = (T)alpha;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, row < *K.nrow);
  double acc[2] = {0.0, 0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T s[B], z[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      s[a] = v.r[d] - ta * v.v[d];
      v.s[d] = s[a];
      acc[0] += (double)s[a] * (double)s[a];
      acc[1] += (double)v.rhat[d] * (double)s[a];
    }
    precond_apply<B, T>(K, row, s, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.shat[i * B + a] = z[a];
  }
  double* outs[2] = {&S->acc_ss, &S->acc_rs};
  block_accumulate<2>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = alpha;
    S->rho_old = rho;
    S->acc_ts = 0.0;
    S->acc_tt = 0.0;
    S->acc_rt = 0.0;
  }
}

// D: t = J shat; (t,s), (t,t), (rhat,t).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_D(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[3] = {0.0, 0.0, 0.0};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, v.shat, y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      v.t[d] = y[a];
      acc[0] += (double)y[a] * (double)v.s[d];
      acc[1] += (double)y[a] * (double)y[a];
      acc[2] += (double)v.rhat[d] * (double)y[a];
    }
  }
  double* outs[3] = {&S->acc_ts, &S->acc_tt, &S->acc_rt};
  block_accumulate<3>(acc, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->acc_rv = 0.0;
    S->acc_vv = 0.0;
    S->iter = S->iter + 1;
  }
}

// A: omega; x and r updates; rho', ||r||^2 from the reduced products; the
// next search direction p and phat.
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_A(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (S->done) return;
  const double tt = S->acc_tt, ts = S->acc_ts;
  const double omega = (tt > 0.0) ? ts / tt : 0.0;
  const double alpha = S->alpha, rho_old = S->rho_old;
  const double rho_new = S->acc_rs - omega * S->acc_rt;
  const double rr = fmax(S->acc_ss - 2.0 * omega * ts + omega * omega * tt, 0.0);
  const double beta = (omega != 0.0 && rho_old != 0.0) ? (rho_new / rho_old) * (alpha / omega) : 0.0;
  const T ta = (T)alpha, tw = (T)omega, tb = (T)beta;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, row < *K.nrow);
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T p[B], z[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      v.x[d] += ta * v.phat[d] + tw * v.shat[d];
      const T rn = v.s[d] - tw * v.t[d];
      v.r[d] = rn;
      p[a] = rn + tb * (v.p[d] - tw * v.v[d]);
      v.p[d] = p[a];
    }
    precond_apply<B, T>(K, row, p, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->omega = omega;
    S->rho = rho_new;
    S->rr_last = rr;
  }
}

// restart from the current x: r = b - J x (the true residual), rhat = r,
// p = r, phat = M^-1 r; rho = (rhat, r), rr_last = (r, r), rhat2 = (r, r).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_restart(DevGrid G, DevMatrix<T> K, const double* __restrict__ res,
                                                       const uint8_t* __restrict__ fixed, KrylovVecs<D, T> v,
                                                       KrylovScalars* S, double tol2, int maxit) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, row < *K.nrow);
  double acc = 0.0;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B], r[B], z[B];
    stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, v.x, y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      const T b = fixed[d] ? (T)0 : (T)(-res[d]);
      r[a] = b - y[a];
      v.r[d] = r[a];
      v.rhat[d] = r[a];
      v.p[d] = r[a];
      acc += (double)r[a] * (double)r[a];
    }
    precond_apply<B, T>(K, row, r, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
  }
  double acc3[3] = {acc, acc, acc};
  double* outs[3] = {&S->rr_last, &S->rho, &S->rhat2};
  block_accumulate<3>(acc3, outs);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = 1.0;
    S->omega = 1.0;
    S->tol2 = tol2;
    S->maxit = maxit;
    S->iter = 0;
    S->done = 0;
    S->status = KS_OK;
  }
}

template <int D, class T, int B>
cudaError_t launch_bicgstab_restart(const DevGrid& G, DevMatrix<T> K, const double* res, const uint8_t* fixed,
                                    KrylovVecs<D, T> v, KrylovScalars* S, double tol2, int maxit, int nblk,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(KrylovScalars), st);
  if (e != cudaSuccess) return e;
  k_bicg_restart<D, T, B><<<nblk, KTPB, 0, st>>>(G, K, res, fixed, v, S, tol2, maxit);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_bicgstab_init(DevMatrix<T> K, const double* res, const uint8_t* fixed, KrylovVecs<D, T> v,
                                 KrylovScalars* S, double tol2, int maxit, int nblk, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(KrylovScalars), st);
  if (e != cudaSuccess) return e;
  k_bicg_init<D, T, B><<<nblk, KTPB, 0, st>>>(K, res, fixed, v, S, tol2, maxit);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_bicgstab_iter(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                 int nblk, cudaStream_t st, const MgApply<T>* mg) {
  k_bicg_B<D, T, B><<<nblk, KTPB, 0, st>>>(G, K, v, S);
  k_bicg_C<D, T, B><<<nblk, KTPB, 0, st>>>(K, v, S);
  // multigrid: C left the first smoothing sweep in shat; the V-cycle completes it
  if (mg) launch_mg_vcycle<D, T, B>(*mg, v.s, v.shat, &S->done, st);
  k_bicg_D<D, T, B><<<nblk, KTPB, 0, st>>>(G, K, v, S);
  k_bicg_A<D, T, B><<<nblk, KTPB, 0, st>>>(K, v, S);
  if (mg) launch_mg_vcycle<D, T, B>(*mg, v.p, v.phat, &S->done, st);
  return cudaGetLastError();
}
// max |d| over the free displacement DOFs of the active rows (the first D of
// the B values of a node), as the ordered bits of a non-negative double
// (atomicMax on the integer image preserves the order).
template <int D, class T, int B>
__global__ void k_absmax(DevMatrix<T> K, const T* __restrict__ x, const uint8_t* __restrict__ fixed,
                         unsigned long long* out) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      const double v = fabs((double)x[d]);
      if (!fixed[d]) m = (v <= 1.7976931348623157e308) ? ((a < D) ? fmax(m, v) : m) : INFINITY;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
template <int D, class T, int B>
cudaError_t launch_absmax(DevMatrix<T> K, const T* x, const uint8_t* fixed, unsigned long long* out, int nblk,
                          cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_absmax<D, T, B><<<nblk, KTPB, 0, st>>>(K, x, fixed, out);
  return cudaGetLastError();
}

// du = base + alpha * step * d on the free DOFs.  step is the Newton
// step-length limit read from the device: with xmax = max |d| over the free
// displacement DOFs (k_absmax), step = hlim / xmax when xmax > hlim, 0 when
// xmax is not finite, else 1 (absmax == nullptr: step = 1).  The halved steps
// of a Newton iteration whose full step drove a return map out of its domain
// pass alpha = 2^-k.
__device__ __forceinline__ double step_limit(const unsigned long long* absmax, double hlim) {
  if (!absmax) return 1.0;
  const double xmax = __longlong_as_double((long long)*absmax);
  if (!(xmax <= 1.7976931348623157e308)) return 0.0;
  return (xmax > hlim) ? hlim / xmax : 1.0;
}
template <int D, class T, int B>
__global__ void k_step_du(DevMatrix<T> K, const T* __restrict__ x, const uint8_t* __restrict__ fixed,
                          const double* __restrict__ base, double* du, double alpha,
                          const unsigned long long* absmax, double hlim) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const double a = alpha * step_limit(absmax, hlim);
  const long long i = K.rows[row];
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const long long d = i * B + c;
    if (!fixed[d]) du[d] = base[d] + a * (double)x[d];
  }
}
template <int D, class T, int B>
cudaError_t launch_step_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, const double* base, double* du,
                           double alpha, int nblk, cudaStream_t st, const unsigned long long* absmax,
                           double hlim) {
  k_step_du<D, T, B><<<nblk, KTPB, 0, st>>>(K, x, fixed, base, du, alpha, absmax, hlim);
  return cudaGetLastError();
}

// Plain y = J x over the active rows (used to time the product in isolation).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_spmv(DevGrid G, DevMatrix<T> K, const T* __restrict__ x, T* y) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const long long i = K.rows[row];
  T v[B];
  stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, x, v);
#pragma unroll
  for (int a = 0; a < B; ++a) y[i * B + a] = v[a];
}
template <int D, class T, int B>
cudaError_t launch_spmv(const DevGrid& G, DevMatrix<T> K, const T* x, T* y, int nblk, cudaStream_t st) {
  k_spmv<D, T, B><<<nblk, KTPB, 0, st>>>(G, K, x, y);
  return cudaGetLastError();
}

// du += d on the free DOFs of active rows (FP64 accumulation of the update).
template <int D, class T, int B>
__global__ void k_update_du(DevMatrix<T> K, const T* __restrict__ x, const uint8_t* __restrict__ fixed,
                            double* du) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *K.nrow) return;
  const long long i = K.rows[row];
#pragma unroll
  for (int a = 0; a < B; ++a) {
    const long long d = i * B + a;
    if (!fixed[d]) du[d] += (double)x[d];
  }
}
template <int D, class T, int B>
cudaError_t launch_update_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, double* du, int nblk,
                             cudaStream_t st) {
  k_update_du<D, T, B><<<nblk, KTPB, 0, st>>>(K, x, fixed, du);
  return cudaGetLastError();
}

#define MPM_KRYLOV_INST(D, T, B)                                                                          \
  template cudaError_t launch_bicgstab_init<D, T, B>(DevMatrix<T>, const double*, const uint8_t*,          \
                                                  KrylovVecs<D, T>, KrylovScalars*, double, int, int,   \
                                                  cudaStream_t);                                        \
  template cudaError_t launch_bicgstab_iter<D, T, B>(const DevGrid&, DevMatrix<T>, KrylovVecs<D, T>,       \
                                                  KrylovScalars*, int, cudaStream_t, const MgApply<T>*); \
  template cudaError_t launch_bicgstab_restart<D, T, B>(const DevGrid&, DevMatrix<T>, const double*,       \
                                                     const uint8_t*, KrylovVecs<D, T>, KrylovScalars*,  \
                                                     double, int, int, cudaStream_t);                   \
  template cudaError_t launch_update_du<D, T, B>(DevMatrix<T>, const T*, const uint8_t*, double*, int,     \
                                              cudaStream_t);                                            \
  template cudaError_t launch_spmv<D, T, B>(const DevGrid&, DevMatrix<T>, const T*, T*, int, cudaStream_t);  \
  template cudaError_t launch_absmax<D, T, B>(DevMatrix<T>, const T*, const uint8_t*, unsigned long long*, int, \
                                           cudaStream_t);                                                  \
  template cudaError_t launch_step_du<D, T, B>(DevMatrix<T>, const T*, const uint8_t*, const double*, double*, \
                                            double, int, cudaStream_t, const unsigned long long*, double);
MPM_KRYLOV_INST(2, float, 2)
MPM_KRYLOV_INST(2, double, 2)
MPM_KRYLOV_INST(3, float, 3)
MPM_KRYLOV_INST(3, double, 3)
MPM_KRYLOV_INST(2, float, 3)
MPM_KRYLOV_INST(2, double, 3)

}  // namespace mpm
