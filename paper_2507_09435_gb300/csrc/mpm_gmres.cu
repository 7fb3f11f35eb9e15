// Restarted GMRES(m), right block-Jacobi preconditioning, classical
// Gram-Schmidt applied twice (CGS2), on J d = b with d0 = 0.
//
// One Arnoldi step j is four kernels, each a single pass over the active rows:
//   S: w = J z_j ; h1_i = (v_i, w), i <= j
//   O1: w -= sum h1_i v_i ; h2_i = (v_i, w)
//   O2: w -= sum h2_i v_i ; (w, w) ; H(:, j) = h1 + h2
//   N: H(j+1, j) = ||w|| ; v_{j+1} = w / ||w|| ; z_{j+1} = M^-1 v_{j+1};
//      one thread applies the previous Givens rotations to H(:, j), forms the
//      new one, updates g and the residual estimate |g_{j+1}|.
// A cycle ends with a one-thread upper-triangular solve H y = g and the
// update x += M^-1 (V y).  All scalars live in device memory (GmresState); a
// kernel returns at once when the cycle is done, so one CUDA graph holds a
// whole cycle and the host polls once per cycle.  A kernel's lead thread
// only writes fields that no other block of the same kernel reads.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int GTPB = KRYLOV_TPB;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce n (<= GMRES_MMAX + 1) partial sums held in acc and add them to out.
__device__ __forceinline__ void block_add_n(double* acc, int n, double* out) {
  __shared__ double sh[GMRES_MMAX + 1][GTPB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    double v = wsum(acc[k]);
    if (lane == 0) sh[k][w] = v;
  }
  __syncthreads();
  for (int k = w; k < n; k += GTPB / 32) {
    double t = (lane < GTPB / 32) ? sh[k][lane] : 0.0;
    t = wsum(t);
    if (lane == 0 && t != 0.0) atomicAdd(&out[k], t);
  }
}


template <int D, class T, int B>
__device__ __forceinline__ void spmv(const DevMatrix<T>& K, int row, long long i, int nx1, int ny1, const T* x,
                                     T y[B]) {
  stencil_row_product<D, T, B>(K, row, i, nx1, ny1, x, y);
}

enum { GS_OK = 0, GS_MAXIT = 1, GS_BREAKDOWN = 2 };
}  // namespace

// basis vector i of the work area
template <class T>
__device__ __forceinline__ T* gvec(const GmresVecs<T>& g, int i) {
  return g.base + (long long)i * g.stride + g.pad;
}

// start of a cycle: v0 = r (r = b on the first cycle, b - J x on a restart;
// x = 0 on the first cycle); accumulates ||r||^2 into st->wn2.
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_residual(DevGrid G, DevMatrix<T> K, const double* __restrict__ res,
                                                         const uint8_t* __restrict__ fixed, GmresVecs<T> g, T* x,
                                                         GmresState* st, int first) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    if (first) {
#pragma unroll
      for (int a = 0; a < B; ++a) y[a] = (T)0;
    } else {
      spmv<D, T, B>(K, row, i, G.nx1, G.ny1, x, y);
    }
    T* v0 = gvec(g, 0);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      const T b = fixed[d] ? (T)0 : (T)(-res[d]);
      const T r = b - y[a];
      if (first) x[d] = (T)0;
      v0[d] = r;
      acc += (double)r * (double)r;
    }
  }
  block_add_n(&acc, 1, &st->wn2);
}

// v0 /= beta; z = M^-1 v0; g = beta e1; reset the cycle.
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_start(DevMatrix<T> K, GmresVecs<T> g, GmresState* st) {
  const double beta = sqrt(st->wn2);
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const bool zero = !(beta > st->tol);
  const unsigned live = __ballot_sync(0xffffffffu, !zero && row < *K.nrow);
  if (!zero && row < *K.nrow) {
    const long long i = K.rows[row];
    T* v0 = gvec(g, 0);
    T u[B], z[B];
    const T ib = (T)(1.0 / beta);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      u[a] = v0[i * B + a] * ib;
      v0[i * B + a] = u[a];
    }
    precond_apply<B, T>(K, row, u, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) g.z[i * B + a] = z[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int k = 0; k <= GMRES_MMAX; ++k) {
      st->gv[k] = 0.0;
      st->h1[k] = 0.0;
      st->h2[k] = 0.0;
    }
    st->gv[0] = beta;
    st->jdone = 0;
    st->res = beta;
    st->wn2b = 0.0;
    if (zero) {
      st->done = 1;
      st->finished = 1;
      st->status = GS_OK;
    }
  }
}

// S_j: w = J z ; h1_i = (v_i, w), i <= j
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_spmv(DevGrid G, DevMatrix<T> K, GmresVecs<T> g, GmresState* st,
                                                     int j) {
  if (st->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[GMRES_MMAX + 1];
  for (int k = 0; k <= j; ++k) acc[k] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->wn2b = 0.0;   // read last in the previous N kernel
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T y[B];
    spmv<D, T, B>(K, row, i, G.nx1, G.ny1, g.z, y);
#pragma unroll
    for (int a = 0; a < B; ++a) g.w[i * B + a] = y[a];
    for (int k = 0; k <= j; ++k) {
      const T* vk = gvec(g, k);
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < B; ++a) s += (double)vk[i * B + a] * (double)y[a];
      acc[k] = s;
    }
  }
  block_add_n(acc, j + 1, st->h1);
}

// O1_j: w -= sum h1_i v_i ; h2_i = (v_i, w)
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_orth1(DevMatrix<T> K, GmresVecs<T> g, GmresState* st, int j) {
  if (st->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[GMRES_MMAX + 1];
  for (int k = 0; k <= j; ++k) acc[k] = 0.0;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T w[B];
#pragma unroll
    for (int a = 0; a < B; ++a) w[a] = g.w[i * B + a];
    for (int k = 0; k <= j; ++k) {
      const T* vk = gvec(g, k);
      const T h = (T)st->h1[k];
#pragma unroll
      for (int a = 0; a < B; ++a) w[a] -= h * vk[i * B + a];
    }
    for (int k = 0; k <= j; ++k) {
      const T* vk = gvec(g, k);
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < B; ++a) s += (double)vk[i * B + a] * (double)w[a];
      acc[k] = s;
    }
#pragma unroll
    for (int a = 0; a < B; ++a) g.w[i * B + a] = w[a];
  }
  block_add_n(acc, j + 1, st->h2);
}

// O2_j: w -= sum h2_i v_i ; (w, w) ; H(:, j) = h1 + h2
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_orth2(DevMatrix<T> K, GmresVecs<T> g, GmresState* st, int j) {
  if (st->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (row < *K.nrow) {
    const long long i = K.rows[row];
    T w[B];
#pragma unroll
    for (int a = 0; a < B; ++a) w[a] = g.w[i * B + a];
    for (int k = 0; k <= j; ++k) {
      const T* vk = gvec(g, k);
      const T h = (T)st->h2[k];
#pragma unroll
      for (int a = 0; a < B; ++a) w[a] -= h * vk[i * B + a];
    }
#pragma unroll
    for (int a = 0; a < B; ++a) {
      g.w[i * B + a] = w[a];
      acc += (double)w[a] * (double)w[a];
    }
  }
  block_add_n(&acc, 1, &st->wn2b);
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k <= j; ++k) st->H[k + (GMRES_MMAX + 1) * j] = st->h1[k] + st->h2[k];
}

// N_j: H(j+1,j) = ||w|| ; v_{j+1} = w/||w|| ; z = M^-1 v_{j+1} ; Givens.
template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_norm(DevMatrix<T> K, GmresVecs<T> g, GmresState* st, int j, int m) {
  if (st->done) return;
  const double hn = sqrt(st->wn2b);
  const bool lucky = !(hn > 1e-300);
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, !lucky && j + 1 <= m && row < *K.nrow);
  if (!lucky && j + 1 <= m && row < *K.nrow) {
    const long long i = K.rows[row];
    T* vn = gvec(g, j + 1);
    T u[B], z[B];
    const T ih = (T)(1.0 / hn);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      u[a] = g.w[i * B + a] * ih;
      vn[i * B + a] = u[a];
    }
    precond_apply<B, T>(K, row, u, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) g.z[i * B + a] = z[a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double* Hj = st->H + (GMRES_MMAX + 1) * j;
    Hj[j + 1] = hn;
    for (int k = 0; k < j; ++k) {
      const double a = Hj[k], b = Hj[k + 1];
      Hj[k] = st->cs[k] * a + st->sn[k] * b;
      Hj[k + 1] = -st->sn[k] * a + st->cs[k] * b;
    }
    const double a = Hj[j], b = Hj[j + 1];
    const double den = sqrt(a * a + b * b);
    const double c = (den > 0.0) ? a / den : 1.0, s = (den > 0.0) ? b / den : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    Hj[j] = den;
    Hj[j + 1] = 0.0;
    st->gv[j + 1] = -s * st->gv[j];
    st->gv[j] = c * st->gv[j];
    st->res = fabs(st->gv[j + 1]);
    st->jdone = j + 1;
    st->iter += 1;
    for (int k = 0; k <= j; ++k) {
      st->h1[k] = 0.0;
      st->h2[k] = 0.0;
    }
    const bool conv = st->res <= st->tol;
    const bool maxed = st->iter >= st->maxit;
    const bool nan = !(st->res == st->res);
    if (conv || lucky || maxed || nan || j + 1 == m) {
      // the cycle ends; the solve is finished unless only the cycle length ran out
      st->done = 1;
      st->finished = (conv || lucky || maxed || nan) ? 1 : 0;
      st->status = (conv || lucky) ? GS_OK : (maxed ? GS_MAXIT : (nan ? GS_BREAKDOWN : GS_OK));
    }
  }
}

__global__ void k_gmres_set(GmresState* st, double tol, int maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->tol = tol;
    st->maxit = maxit;
  }
}

// end of a cycle: y = H^-1 g (k x k upper triangular, one thread), then
// x += M^-1 (V y) over the rows.
__global__ void k_gmres_solve(GmresState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->jdone;
  for (int r = k - 1; r >= 0; --r) {
    double s = st->gv[r];
    for (int c = r + 1; c < k; ++c) s -= st->H[r + (GMRES_MMAX + 1) * c] * st->y[c];
    const double d = st->H[r + (GMRES_MMAX + 1) * r];
    st->y[r] = (d != 0.0) ? s / d : 0.0;
  }
}

template <int D, class T, int B>
__global__ void __launch_bounds__(GTPB) k_gmres_update(DevMatrix<T> K, GmresVecs<T> g, GmresState* st, T* x) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned live = __ballot_sync(0xffffffffu, row < *K.nrow);
  if (row >= *K.nrow) return;
  const int k = st->jdone;
  const long long i = K.rows[row];
  T u[B], z[B];
#pragma unroll
  for (int a = 0; a < B; ++a) u[a] = (T)0;
  for (int c = 0; c < k; ++c) {
    const T* vc = gvec(g, c);
    const T yc = (T)st->y[c];
#pragma unroll
    for (int a = 0; a < B; ++a) u[a] += yc * vc[i * B + a];
  }
  precond_apply<B, T>(K, row, u, z, live);
#pragma unroll
  for (int a = 0; a < B; ++a) x[i * B + a] += z[a];
}

template <int D, class T, int B>
cudaError_t launch_gmres_begin(const DevGrid& G, DevMatrix<T> K, const double* res, const uint8_t* fixed,
                               GmresVecs<T> g, T* x, GmresState* st, int first, double tol, int maxit_left,
                               int nblk, cudaStream_t s) {
  // keep iter/maxit/tol across restarts: reset only the cycle fields
  if (first) {
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(GmresState), s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(&st->wn2, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&st->done, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&st->finished, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_gmres_set<<<1, 1, 0, s>>>(st, tol, maxit_left);
  k_gmres_residual<D, T, B><<<nblk, GTPB, 0, s>>>(G, K, res, fixed, g, x, st, first);
  k_gmres_start<D, T, B><<<nblk, GTPB, 0, s>>>(K, g, st);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_gmres_cycle(const DevGrid& G, DevMatrix<T> K, GmresVecs<T> g, T* x, GmresState* st, int m,
                               int nblk, cudaStream_t s) {
  for (int j = 0; j < m; ++j) {
    k_gmres_spmv<D, T, B><<<nblk, GTPB, 0, s>>>(G, K, g, st, j);
    k_gmres_orth1<D, T, B><<<nblk, GTPB, 0, s>>>(K, g, st, j);
    k_gmres_orth2<D, T, B><<<nblk, GTPB, 0, s>>>(K, g, st, j);
    k_gmres_norm<D, T, B><<<nblk, GTPB, 0, s>>>(K, g, st, j, m);
  }
  k_gmres_solve<<<1, 32, 0, s>>>(st);
  k_gmres_update<D, T, B><<<nblk, GTPB, 0, s>>>(K, g, st, x);
  return cudaGetLastError();
}

#define MPM_GMRES_INST(D, T, B)                                                                            \
  template cudaError_t launch_gmres_begin<D, T, B>(const DevGrid&, DevMatrix<T>, const double*, const uint8_t*, \
                                                GmresVecs<T>, T*, GmresState*, int, double, int, int,   \
                                                cudaStream_t);                                          \
  template cudaError_t launch_gmres_cycle<D, T, B>(const DevGrid&, DevMatrix<T>, GmresVecs<T>, T*, GmresState*, \
                                                int, int, cudaStream_t);
MPM_GMRES_INST(2, float, 2)
MPM_GMRES_INST(2, double, 2)
MPM_GMRES_INST(3, float, 3)
MPM_GMRES_INST(3, double, 3)
MPM_GMRES_INST(2, float, 3)
MPM_GMRES_INST(2, double, 3)

}  // namespace mpm
