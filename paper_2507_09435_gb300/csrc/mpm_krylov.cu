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

// Accumulator of a dot product.  For FP64 vectors a double; for FP32
// vectors a double-float pair (hi + lo, about 48 significant bits): each
// product enters exactly (Dekker's product by a fused multiply-add) and each
// sum is Knuth's error-free two-sum, so the sums keep FP64-level accuracy
// while running on the FP32 pipe (the FP64 pipe has 1/64 of its rate here).
// The explicit _rn intrinsics keep the compiler from contracting or
// reassociating the error terms.
template <class T>
struct Acc;
template <>
struct Acc<double> {
  double v;
  __device__ static Acc zero() { return {0.0}; }
  __device__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ void add(const Acc& o) { v += o.v; }
  __device__ Acc shfl_xor(int o) const { return {__shfl_xor_sync(0xffffffffu, v, o)}; }
  __device__ double value() const { return v; }
  __device__ static Acc load_l2(const Acc* p) { return {__ldcg(&p->v)}; }
};
template <>
struct Acc<float> {
  float hi, lo;
  __device__ static Acc zero() { return {0.0f, 0.0f}; }
  // (hi, lo) += (x, xe)
  __device__ void add2(float x, float xe) {
    const float s = __fadd_rn(hi, x);
    const float bv = __fadd_rn(s, -hi);
    const float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bv)), __fadd_rn(x, -bv));
    const float t = __fadd_rn(e, __fadd_rn(lo, xe));
    hi = __fadd_rn(s, t);
    lo = __fadd_rn(t, -__fadd_rn(hi, -s));
  }
  __device__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    add2(p, __fmaf_rn(a, b, -p));
  }
  __device__ void add(const Acc& o) { add2(o.hi, o.lo); }
  __device__ Acc shfl_xor(int o) const {
    return {__shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o)};
  }
  __device__ double value() const { return (double)hi + (double)lo; }
  __device__ static Acc load_l2(const Acc* p) {
    const float2 u = __ldcg(reinterpret_cast<const float2*>(p));
    return {u.x, u.y};
  }
};
static_assert(sizeof(Acc<float>) == sizeof(double) && sizeof(Acc<double>) == sizeof(double),
              "one reduction slot per accumulator");

// Sums of NV per-thread accumulators over the whole grid, in an order fixed
// by the grid alone (the result does not depend on the order in which the
// blocks run): each block stores its NV block sums in red[k * gridDim.x +
// block] and takes a ticket; the block that takes the last ticket adds the
// stored sums in block order (strided over its threads, then a fixed tree)
// and resets the ticket for the next kernel.  Returns true in every thread
// of that last block, with the sums in out[] of its thread 0.  Every block
// of the grid calls this exactly once.
template <class T, int NV>
__device__ __forceinline__ bool grid_sum(Acc<T> v[NV], double* red_raw, unsigned int* ticket, double out[NV]) {
  constexpr int NW = KTPB / 32;
  constexpr int RU = 8;   // loads per sum in flight in the last block
  __shared__ Acc<T> sh[NV][NW];
  __shared__ int last;
  Acc<T>* red = reinterpret_cast<Acc<T>*>(red_raw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k].add(v[k].shfl_xor(o));
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  }
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      Acc<T> t = sh[k][0];
#pragma unroll
      for (int q = 1; q < NW; ++q) t.add(sh[k][q]);
      red[k * nb + blockIdx.x] = t;
    }
    __threadfence();
    last = (atomicAdd(ticket, 1u) == (unsigned)(nb - 1));
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // one sum at a time, RU of its block sums in flight (few registers: this
  // code shares the kernel's register allocation)
  Acc<T> t[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    t[k] = Acc<T>::zero();
    for (int q0 = threadIdx.x; q0 < nb; q0 += KTPB * RU) {
      Acc<T> l[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int q = q0 + u * KTPB;
        l[u] = (q < nb) ? Acc<T>::load_l2(&red[k * nb + q]) : Acc<T>::zero();
      }
#pragma unroll
      for (int u = 0; u < RU; ++u) t[k].add(l[u]);
    }
  }
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[k].add(t[k].shfl_xor(o));
  __syncthreads();   // sh is reused
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = t[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      Acc<T> u = sh[k][0];
#pragma unroll
      for (int q = 1; q < NW; ++q) u.add(sh[k][q]);
      out[k] = u.value();
    }
    *ticket = 0u;
  }
  return true;
}

enum { KS_OK = 0, KS_MAXIT = 1, KS_BREAKDOWN = 2 };

// Stop decision taken once per iteration from the reduced scalars (0: go
// on; else 1 + the status): converged, iteration limit, or breakdown (a
// non-finite residual norm, or a zero rho or omega).
__device__ __forceinline__ int stop_code(double rr, int it, int maxit, double tol2, bool bad) {
  if (rr <= tol2) return 1 + KS_OK;
  if (it >= maxit) return 1 + KS_MAXIT;
  if (!(rr == rr) || bad) return 1 + KS_BREAKDOWN;
  return 0;
}

// The working-precision copy of a scalar of the iteration.
template <class T>
__device__ __forceinline__ T scal(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}
}  // namespace

// ------------------------------------------------------------------ BiCGStab
// Right-preconditioned BiCGStab (van der Vorst 1992) on J d = b, d0 = 0, in a
// merged-reduction form with four kernels per iteration:
//   B: v = J phat, (rhat, v); then alpha = rho / (rhat, v)
//   C: s = r - alpha v; shat = M^-1 s; (s,s), (rhat,s)
//   D: t = J shat; (t,s), (t,t), (rhat,t); then omega = (t,s)/(t,t),
//      rho' = (rhat,s) - omega (rhat,t), ||r||^2 = (s,s) - 2 omega (t,s) +
//      omega^2 (t,t), beta = (rho'/rho)(alpha/omega)
//   A: x += alpha phat + omega shat; r = s - omega t;
//      p = r + beta (p - omega v); phat = M^-1 p.
// The two dot products of the classical form's last step follow from the
// ones already reduced, so the update and the next search direction share one
// pass.  The scalars ("then ...") are computed once, by the thread that
// finishes the kernel's grid sum, which also takes the stop decision for the
// next iteration; the row kernels only read their FP32 copies.  (The dot
// products keep FP64-level accuracy, see Acc, which keeps the cancellation in
// ||r||^2 harmless at the linear tolerances used.)
// Every field of the scalars is written in one kernel and read only in later
// kernels, except the stop fields (done, status), which block 0 sets when
// the whole grid returns at once.

// The start of an iteration's kernels: the solve is over (every kernel of a
// graph chunk then returns at once).
__device__ __forceinline__ bool bicg_over(KrylovScalars* S) { return S->done != 0; }

// init: r = b, rhat = b, x = 0, p = r, phat = M^-1 r; rho = (rhat, r),
// rr_last = (r, r).
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_init(DevMatrix<T> K, const double* __restrict__ res,
                                                    const uint8_t* __restrict__ fixed, KrylovVecs<D, T> v,
                                                    KrylovScalars* S, double tol2, int maxit) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *K.nrow;
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  Acc<T> acc[1] = {Acc<T>::zero()};
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
      acc[0].add_prod(b[a], b[a]);
    }
    precond_apply<B, T>(K, row, b, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
  }
  double out[1];
  const bool last = grid_sum<T, 1>(acc, v.red, &S->ticket, out);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = 1.0;
    S->omega = 1.0;
    S->tol2 = tol2;
    S->maxit = maxit;
    S->iter = 0;
    S->done = 0;
    S->status = KS_OK;
  }
  if (last && threadIdx.x == 0) {
    S->rr_last = out[0];
    S->rho = out[0];
    S->rhat2 = out[0];
    S->next_stop = stop_code(out[0], 0, maxit, tol2, false);
  }
}

// B: stop test, then v = J phat and (rhat, v), (v, v); alpha.
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_B(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (bicg_over(S)) return;
  const int ns = S->next_stop;
  if (ns != 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->done = 1;
      S->status = ns - 1;
    }
    return;
  }
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  Acc<T> acc[2] = {Acc<T>::zero(), Acc<T>::zero()};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, v.phat, y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      v.v[i * B + a] = y[a];
      acc[0].add_prod(v.rhat[i * B + a], y[a]);
      acc[1].add_prod(y[a], y[a]);
    }
  }
  double out[2];
  if (grid_sum<T, 2>(acc, v.red, &S->ticket, out) && threadIdx.x == 0) {
    const double rv = out[0], vv = out[1];
    S->acc_rv = rv;
    S->acc_vv = vv;
    // (near) breakdown: rhat and v almost orthogonal, relative to FP32 vectors
    const bool brk = !(fabs(rv) > 1e-7 * sqrt(vv * S->rhat2));
    const double alpha = brk ? 0.0 : S->rho / rv;
    S->c_break = brk ? 1 : 0;
    S->alpha = alpha;
    S->alpha_f = (float)alpha;
  }
}

// C: s = r - alpha v; shat = M^-1 s (elementwise: its dot products (s,s) and
// (rhat,s) are taken by D, which reads s anyway).  The row's r and v are
// loaded before the scalars, so that the two latencies overlap.
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_C(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *K.nrow;
  long long i = 0;
  T rr_[B], vv_[B];
  if (row < nrow) {
    i = K.rows[row];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      rr_[a] = v.r[i * B + a];
      vv_[a] = v.v[i * B + a];
    }
  }
  if (bicg_over(S)) return;
  if (S->c_break) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->done = 1;
      S->status = KS_BREAKDOWN;
    }
    return;
  }
  const T ta = scal<T>(S->alpha, S->alpha_f);
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  if (row < nrow) {
    T sv[B], z[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      sv[a] = rr_[a] - ta * vv_[a];
      v.s[i * B + a] = sv[a];
    }
    precond_apply<B, T>(K, row, sv, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.shat[i * B + a] = z[a];
  }
}

// D: t = J shat; (t,s), (t,t), (rhat,t), (s,s), (rhat,s); omega, rho',
// ||r||^2, beta and the stop decision for the next iteration.
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_D(DevGrid G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  if (bicg_over(S)) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  Acc<T> acc[5] = {Acc<T>::zero(), Acc<T>::zero(), Acc<T>::zero(), Acc<T>::zero(), Acc<T>::zero()};
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    stencil_row_product<D, T, B>(K, row, i, G.nx1, G.ny1, v.shat, y);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      v.t[d] = y[a];
      const T sd = v.s[d], rh = v.rhat[d];
      acc[0].add_prod(y[a], sd);
      acc[1].add_prod(y[a], y[a]);
      acc[2].add_prod(rh, y[a]);
      acc[3].add_prod(sd, sd);
      acc[4].add_prod(rh, sd);
    }
  }
  double out[5];
  if (grid_sum<T, 5>(acc, v.red, &S->ticket, out) && threadIdx.x == 0) {
    const double ts = out[0], tt = out[1], rt = out[2], ss = out[3], rs = out[4];
    S->acc_ts = ts;
    S->acc_tt = tt;
    S->acc_rt = rt;
    S->acc_ss = ss;
    S->acc_rs = rs;
    const double omega = (tt > 0.0) ? ts / tt : 0.0;
    const double rho = S->rho, alpha = S->alpha;
    const double rho_new = rs - omega * rt;
    const double rr = fmax(ss - 2.0 * omega * ts + omega * omega * tt, 0.0);
    const double beta = (omega != 0.0 && rho != 0.0) ? (rho_new / rho) * (alpha / omega) : 0.0;
    const int it = S->iter + 1;
    S->iter = it;
    S->omega = omega;
    S->rho = rho_new;
    S->rr_last = rr;
    S->beta = beta;
    S->omega_f = (float)omega;
    S->beta_f = (float)beta;
    S->next_stop = stop_code(rr, it, S->maxit, S->tol2, rho_new == 0.0 || omega == 0.0);
  }
}

// A: x and r updates; the next search direction p and phat.
template <int D, class T, int B>
__global__ void __launch_bounds__(KTPB) k_bicg_A(DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S) {
  // the row's vectors are loaded before the scalars (the latencies overlap)
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *K.nrow;
  long long i = 0;
  T xs[B], ph[B], sh[B], ss[B], ts[B], ps[B], vs[B];
  if (row < nrow) {
    i = K.rows[row];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      xs[a] = v.x[d]; ph[a] = v.phat[d]; sh[a] = v.shat[d]; ss[a] = v.s[d];
      ts[a] = v.t[d]; ps[a] = v.p[d]; vs[a] = v.v[d];
    }
  }
  if (bicg_over(S)) return;
  const T ta = scal<T>(S->alpha, S->alpha_f), tw = scal<T>(S->omega, S->omega_f),
          tb = scal<T>(S->beta, S->beta_f);
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  if (row < nrow) {
    T p[B], z[B];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      v.x[d] = xs[a] + (ta * ph[a] + tw * sh[a]);
      const T rn = ss[a] - tw * ts[a];
      v.r[d] = rn;
      p[a] = rn + tb * (ps[a] - tw * vs[a]);
      v.p[d] = p[a];
    }
    precond_apply<B, T>(K, row, p, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
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
  Acc<T> acc[1] = {Acc<T>::zero()};
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
      acc[0].add_prod(r[a], r[a]);
    }
    precond_apply<B, T>(K, row, r, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) v.phat[i * B + a] = z[a];
  }
  double out[1];
  const bool last = grid_sum<T, 1>(acc, v.red, &S->ticket, out);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->alpha = 1.0;
    S->omega = 1.0;
    S->tol2 = tol2;
    S->maxit = maxit;
    S->iter = 0;
    S->done = 0;
    S->status = KS_OK;
  }
  if (last && threadIdx.x == 0) {
    S->rr_last = out[0];
    S->rho = out[0];
    S->rhat2 = out[0];
    S->next_stop = stop_code(out[0], 0, maxit, tol2, false);
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
