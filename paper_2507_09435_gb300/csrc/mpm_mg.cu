// Geometric multigrid V-cycle preconditioner for the Newton correction
// system J d = -r.
//
// The paper hands this system to AMG or a direct solver on the host (Sec. 2.2,
// remark on linear solvers) and names stronger block preconditioning as future
// work (Sec. 5).  Here the preconditioner is a geometric V-cycle on the
// background grid itself:
// * level l+1 is the grid of every second node of level l (node J of level
//   l+1 sits at node 2J of level l; a level of n1 nodes per axis has
//   n1/2 + 1 coarse nodes);
// * the prolongation P interpolates each node component linearly per axis
//   (weight 1 from the coincident coarse node, 1/2 and 1/2 from the two
//   neighbours of an odd fine node); rows of prescribed fine DOFs are zero;
// * the coarse operator is the Galerkin product P^T A P.  The quadratic
//   B-spline Jacobian couples nodes up to two apart per axis and P reaches
//   one node, so the product again couples coarse nodes up to two apart: every
//   level has the same stencil-BSR layout and the same row kernels;
// * a coarse DOF none of whose fine DOFs is free becomes an identity row;
// * smoother: damped block Jacobi, z += w D^-1 (b - A z), with
//   w = c / lambda_max(D^-1 A) from a power iteration (the block inverses are
//   stored pre-multiplied by w); MG_NU0 sweeps before and after the coarse
//   correction on the finest level, one on the coarse levels;
// * coarsest level (at most MG_DENSE_MAX unknowns): a dense inverse by
//   Gauss-Jordan elimination with partial pivoting in shared memory;
// * the levels with at most MG_TAIL_ROWS rows run, with the dense solve,
//   inside one kernel of one thread-block cluster (cluster barriers between
//   the steps); the levels above take one launch per step (residual,
//   restriction with the coarse level's first sweep, prolongation,
//   post-smoothing).
// The V-cycle is a fixed linear operator, so it serves as the right
// preconditioner of BiCGStab.  Every apply kernel returns at once when the
// Krylov solve is done (the graph chunks of iterations run to their end).
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "mpm_internal.h"

namespace mpm {

namespace cg = cooperative_groups;

namespace {
constexpr int MTPB = KRYLOV_TPB;

__device__ __forceinline__ float wt1(int s) { return s == 0 ? 1.0f : 0.5f; }

template <int D>
__device__ __forceinline__ void node_xyz(long long i, int nx1, int ny1, int& x, int& y, int& z) {
  x = (int)(i % nx1);
  y = (int)((i / nx1) % ny1);
  z = (D == 3) ? (int)(i / ((long long)nx1 * ny1)) : 0;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The grid's sum of v written to *out in an order fixed by the grid: each
// block stores its sum in part[block] and takes a ticket; the block that
// takes the last one adds the stored sums in block order and resets the
// ticket.  Every block of the grid calls this once.
__device__ __forceinline__ void grid_add(double v, double* out, double* part, unsigned* ticket) {
  __shared__ double sh[MTPB / 32];
  __shared__ int last;
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < MTPB / 32; ++q) t += sh[q];
    part[blockIdx.x] = t;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += MTPB) t += __ldcg(&part[b]);
  t = wsum(t);
  __syncthreads();
  if (lane == 0) sh[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int q = 0; q < MTPB / 32; ++q) u += sh[q];
    *out = u;
    *ticket = 0u;
  }
}

__device__ __forceinline__ bool is_done(const int* done) { return done && *(volatile const int*)done; }

// Coarse nodes: active when one of the fine nodes it interpolates to is
// active.  flag has nc + 1 entries (the last is 0, for the exclusive scan).
template <int D>
__global__ void k_mg_flags(int fx, int fy, int fz, const int* __restrict__ n2r_f, int cx, int cy, long long nc,
                           int* flag) {
  const long long J = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (J > nc) return;
  if (J == nc) { flag[nc] = 0; return; }
  int X, Y, Z;
  node_xyz<D>(J, cx, cy, X, Y, Z);
  int on = 0;
  constexpr int ZR = (D == 3) ? 1 : 0;
  for (int sz = -ZR; sz <= ZR; ++sz) {
    const int iz = 2 * Z + sz;
    if (iz < 0 || iz >= fz) continue;
    for (int sy = -1; sy <= 1; ++sy) {
      const int iy = 2 * Y + sy;
      if (iy < 0 || iy >= fy) continue;
      for (int sx = -1; sx <= 1; ++sx) {
        const int ix = 2 * X + sx;
        if (ix < 0 || ix >= fx) continue;
        on |= (n2r_f[ix + (long long)fx * (iy + (long long)fy * iz)] >= 0) ? 1 : 0;
      }
    }
  }
  flag[J] = on;
}

// Coarse prescribed DOFs: component a of coarse node J is prescribed when no
// active fine node it interpolates to has component a free.
template <int D, int B>
__global__ void k_mg_fixed(int fx, int fy, int fz, const int* __restrict__ n2r_f, const uint8_t* __restrict__ fix_f,
                           int cx, int cy, long long nc, uint8_t* fix_c) {
  const long long J = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (J >= nc) return;
  int X, Y, Z;
  node_xyz<D>(J, cx, cy, X, Y, Z);
  bool freec[B];
#pragma unroll
  for (int a = 0; a < B; ++a) freec[a] = false;
  constexpr int ZR = (D == 3) ? 1 : 0;
  for (int sz = -ZR; sz <= ZR; ++sz) {
    const int iz = 2 * Z + sz;
    if (iz < 0 || iz >= fz) continue;
    for (int sy = -1; sy <= 1; ++sy) {
      const int iy = 2 * Y + sy;
      if (iy < 0 || iy >= fy) continue;
      for (int sx = -1; sx <= 1; ++sx) {
        const int ix = 2 * X + sx;
        if (ix < 0 || ix >= fx) continue;
        const long long i = ix + (long long)fx * (iy + (long long)fy * iz);
        if (n2r_f[i] < 0) continue;
#pragma unroll
        for (int a = 0; a < B; ++a) freec[a] |= (fix_f[i * B + a] == 0);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < B; ++a) fix_c[J * B + a] = freec[a] ? 0 : 1;
}

// Galerkin product: block (J, J+O) of P^T A P, one thread per (coarse row,
// slot).  Per axis the pairs (s, t) of fine offsets i = 2J + s, j = 2(J+O) + t
// with |j - i| <= 2 are enumerated directly (9, 6 or 1 pairs for |O| = 0, 1,
// 2).  Every block of every coarse row is written (no zero fill).
template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_galerkin(MgLevel<T> f, MgLevel<T> c) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = blockIdx.y;
  if (row >= *c.K.nrow) return;
  const long long J = c.K.rows[row];
  int X, Y, Z;
  node_xyz<D>(J, c.nx1, c.ny1, X, Y, Z);
  const int ox = slot % 5 - 2, oy = (slot / 5) % 5 - 2, oz = (D == 3) ? slot / 25 - 2 : 0;
  const int KX = X + ox, KY = Y + oy, KZ = Z + oz;
  T acc[B * B];
#pragma unroll
  for (int k = 0; k < B * B; ++k) acc[k] = (T)0;
  const bool kin = KX >= 0 && KY >= 0 && KZ >= 0 && KX < c.nx1 && KY < c.ny1 && (D == 2 || KZ < c.nz1);
  if (kin) {
    constexpr int ZR = (D == 3) ? 1 : 0;
    for (int sz = -ZR; sz <= ZR; ++sz) {
      const int iz = 2 * Z + sz;
      if (iz < 0 || iz >= f.nz1) continue;
      const int tz0 = (D == 3) ? max(-1, sz - 2 - 2 * oz) : 0, tz1 = (D == 3) ? min(1, sz + 2 - 2 * oz) : 0;
      for (int sy = -1; sy <= 1; ++sy) {
        const int iy = 2 * Y + sy;
        if (iy < 0 || iy >= f.ny1) continue;
        const int ty0 = max(-1, sy - 2 - 2 * oy), ty1 = min(1, sy + 2 - 2 * oy);
        for (int sx = -1; sx <= 1; ++sx) {
          const int ix = 2 * X + sx;
          if (ix < 0 || ix >= f.nx1) continue;
          const long long i = ix + (long long)f.nx1 * (iy + (long long)f.ny1 * iz);
          const int fr = f.node2row[i];
          if (fr < 0) continue;
          T mi[B];
#pragma unroll
          for (int a = 0; a < B; ++a) mi[a] = f.fixed[i * B + a] ? (T)0 : (T)1;
          const T wi = (T)(wt1(sx) * wt1(sy) * wt1(sz));
          const int tx0 = max(-1, sx - 2 - 2 * ox), tx1 = min(1, sx + 2 - 2 * ox);
          for (int tz = tz0; tz <= tz1; ++tz) {
            const int jz = 2 * KZ + tz;
            if (jz < 0 || jz >= f.nz1) continue;
            for (int ty = ty0; ty <= ty1; ++ty) {
              const int jy = 2 * KY + ty;
              if (jy < 0 || jy >= f.ny1) continue;
              for (int tx = tx0; tx <= tx1; ++tx) {
                const int jx = 2 * KX + tx;
                if (jx < 0 || jx >= f.nx1) continue;
                const long long j = jx + (long long)f.nx1 * (jy + (long long)f.ny1 * jz);
                const int dx = jx - ix, dy = jy - iy, dz = jz - iz;
                const int fs = (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
                const T w = wi * (T)(wt1(tx) * wt1(ty) * wt1(tz));
                T kb[B * B];
                ld_block<B, T>(&f.K.val[((long long)fs * f.K.cap + fr) * (B * B)], kb);
#pragma unroll
                for (int b = 0; b < B; ++b) {
                  const T wb = f.fixed[j * B + b] ? (T)0 : w;
#pragma unroll
                  for (int a = 0; a < B; ++a) acc[a * B + b] += mi[a] * wb * kb[a * B + b];
                }
              }
            }
          }
        }
      }
    }
  }
  constexpr int CENTER = (D == 2) ? 12 : 62;
  if (slot == CENTER) {
#pragma unroll
    for (int a = 0; a < B; ++a)
      if (c.fixed[J * B + a]) acc[a * B + a] = (T)1;
  }
  T* out = &c.K.val[((long long)slot * c.K.cap + row) * (B * B)];
#pragma unroll
  for (int k = 0; k < B * B; ++k) out[k] = acc[k];
}

// splitmix64 of the DOF index, mapped to [-1, 1): the start of the power
// iteration (deterministic, independent of launch shape)
__device__ __forceinline__ double hash_unit(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_power_init(MgLevel<T> l, T* v, double* nrm, double* part,
                                                        unsigned* ticket) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (row < *l.K.nrow) {
    const long long i = l.K.rows[row];
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const long long d = i * B + a;
      const T x = l.fixed[d] ? (T)0 : (T)hash_unit((unsigned long long)d);
      v[d] = x;
      acc += (double)x * (double)x;
    }
  }
  grid_add(acc, nrm, part, ticket);
}

// dst = D^-1 A src / ||src||, accumulating ||dst||^2 (D^-1: the unscaled
// block-Jacobi inverse, node blocks or row segments)
template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_power(MgLevel<T> l, const T* src, T* dst, const double* nin,
                                                   double* nout, double* part, unsigned* ticket) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *l.K.nrow;
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  const double n2 = *nin;
  const T sc = (n2 > 0.0 && n2 < 1e300) ? (T)(1.0 / sqrt(n2)) : (T)0;
  double acc = 0.0;
  if (row < nrow) {
    const long long i = l.K.rows[row];
    T y[B], z[B];
    stencil_row_product<D, T, B>(l.K, row, i, l.nx1, l.ny1, src, y);
    precond_apply<B, T>(l.K, row, y, z, live);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      const T t = z[a] * sc;
      dst[i * B + a] = t;
      acc += (double)t * (double)t;
    }
  }
  grid_add(acc, nout, part, ticket);
}

// dinv *= c / lambda, lambda = sqrt(*nrm) (the last power-iteration norm);
// w = 1/2 when the estimate is unusable
template <class T>
__global__ void k_mg_scale(T* dinv, long long n, const double* nrm, double c) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double lam = sqrt(*nrm);
  const double w = (lam >= 1e-3 && lam < 1e30) ? c / lam : 0.5;
  dinv[k] = (T)((double)dinv[k] * w);
}

// Dense inverse of the coarsest level (n = nrow * B <= MG_DENSE_MAX) by
// Gauss-Jordan elimination with partial pivoting on [A | I] in shared memory,
// one block of 32 x 32 threads.  Per column, warp 0 picks the pivot, swaps it
// into place and stages the normalised pivot row and the elimination factors;
// then every thread updates its rows (ty + 32k) and columns (tx + 32m).  A
// pivot that vanishes is replaced by 1 (the preconditioner stays defined).
// Written transposed: invT[j*n + k] = (A^-1)[k][j].
template <int D, class T, int B>
__global__ void __launch_bounds__(1024) k_mg_dense_inverse(MgLevel<T> c, float* invT) {
  extern __shared__ float sm[];
  __shared__ float fac[MG_DENSE_MAX];
  __shared__ float prow[2 * MG_DENSE_MAX];
  const int nrow = *c.K.nrow;
  const int n = nrow * B, W = 2 * n;
  if (n <= 0 || n > MG_DENSE_MAX) return;
  float* a = sm;   // a[r * W + col]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < n; r += 32)
    for (int j = tx; j < W; j += 32) a[r * W + j] = (j == n + r) ? 1.0f : 0.0f;
  __syncthreads();
  constexpr int S = (D == 2) ? 25 : 125;
  for (int k = threadIdx.x; k < nrow * S; k += blockDim.x) {
    const int rr = k / S, slot = k % S;
    const long long J = c.K.rows[rr];
    int X, Y, Z;
    node_xyz<D>(J, c.nx1, c.ny1, X, Y, Z);
    const int KX = X + slot % 5 - 2, KY = Y + (slot / 5) % 5 - 2, KZ = Z + ((D == 3) ? slot / 25 - 2 : 0);
    if (KX < 0 || KY < 0 || KZ < 0 || KX >= c.nx1 || KY >= c.ny1 || (D == 3 && KZ >= c.nz1)) continue;
    const int cc = c.node2row[KX + (long long)c.nx1 * (KY + (long long)c.ny1 * KZ)];
    if (cc < 0) continue;
    const T* blk = &c.K.val[((long long)slot * c.K.cap + rr) * (B * B)];
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
      for (int y = 0; y < B; ++y) a[(rr * B + x) * W + cc * B + y] = (float)blk[x * B + y];
  }
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    if (ty == 0) {
      float best = -1.0f;
      int bi = col;
      for (int r = col + tx; r < n; r += 32) {
        const float v = fabsf(a[r * W + col]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const bool bad = !(best > 1e-30f) || !(best < 3e38f);
      if (bi != col)
        for (int j = tx; j < W; j += 32) {
          const float t = a[col * W + j];
          a[col * W + j] = a[bi * W + j];
          a[bi * W + j] = t;
        }
      __syncwarp();
      const float ip = bad ? 1.0f : 1.0f / a[col * W + col];
      for (int j = tx; j < W; j += 32) prow[j] = (j == col) ? 1.0f : a[col * W + j] * ip;
      for (int r = tx; r < n; r += 32) fac[r] = (r == col) ? 0.0f : a[r * W + col];
    }
    __syncthreads();
    for (int r = ty; r < n; r += 32) {
      const float f = fac[r];
      if (r == col) {
        for (int j = tx; j < W; j += 32) a[r * W + j] = prow[j];
      } else if (f != 0.0f) {
        for (int j = tx; j < W; j += 32) a[r * W + j] -= f * prow[j];
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) {
    const int r = k / n, j = k % n;
    invT[j * n + r] = a[r * W + n + j];
  }
}

// ---- one row of each V-cycle step (used by the per-level kernels and by the
// cluster tail; COH: the input vector was written earlier in the same kernel,
// so it is read with ordinary loads)

// r = b - A z
template <int D, class T, int B, bool COH>
__device__ __forceinline__ void row_residual(const MgLevel<T>& l, int row, const T* b, const T* z, T* r) {
  const long long i = l.K.rows[row];
  T y[B];
  stencil_row_product<D, T, B, COH>(l.K, row, i, l.nx1, l.ny1, z, y);
#pragma unroll
  for (int a = 0; a < B; ++a) r[i * B + a] = b[i * B + a] - y[a];
}

// b_c = P^T r_f for coarse row `row`; with `presmooth`, also the first
// smoothing sweep of the coarse level from zero, z_c = w D_c^-1 b_c (coarse
// levels use node blocks)
template <int D, class T, int B>
__device__ __forceinline__ void row_restrict(const MgLevel<T>& f, const T* rf, const MgLevel<T>& c, int row,
                                             bool presmooth) {
  const long long J = c.K.rows[row];
  int X, Y, Z;
  node_xyz<D>(J, c.nx1, c.ny1, X, Y, Z);
  T acc[B];
#pragma unroll
  for (int a = 0; a < B; ++a) acc[a] = (T)0;
  constexpr int ZR = (D == 3) ? 1 : 0;
  for (int sz = -ZR; sz <= ZR; ++sz) {
    const int iz = 2 * Z + sz;
    if (iz < 0 || iz >= f.nz1) continue;
    for (int sy = -1; sy <= 1; ++sy) {
      const int iy = 2 * Y + sy;
      if (iy < 0 || iy >= f.ny1) continue;
      for (int sx = -1; sx <= 1; ++sx) {
        const int ix = 2 * X + sx;
        if (ix < 0 || ix >= f.nx1) continue;
        const long long i = ix + (long long)f.nx1 * (iy + (long long)f.ny1 * iz);
        if (f.node2row[i] < 0) continue;
        const T w = (T)(wt1(sx) * wt1(sy) * wt1(sz));
#pragma unroll
        for (int a = 0; a < B; ++a)
          if (!f.fixed[i * B + a]) acc[a] += w * rf[i * B + a];
      }
    }
  }
#pragma unroll
  for (int a = 0; a < B; ++a) c.b[J * B + a] = acc[a];
  if (presmooth) {
    T z[B];
    precond_apply<B, T>(c.K, row, acc, z, 0u);
#pragma unroll
    for (int a = 0; a < B; ++a) c.z[J * B + a] = z[a];
  }
}

// out = z_f + P z_c for fine row `row` (prescribed DOFs keep z_f)
template <int D, class T, int B>
__device__ __forceinline__ void row_prolong(const MgLevel<T>& f, const T* zf, const MgLevel<T>& c, T* out, int row) {
  const long long i = f.K.rows[row];
  int ix, iy, iz;
  node_xyz<D>(i, f.nx1, f.ny1, ix, iy, iz);
  T acc[B];
#pragma unroll
  for (int a = 0; a < B; ++a) acc[a] = (T)0;
  // parents per axis: i even -> i/2 (weight 1); i odd -> (i-1)/2, (i+1)/2 (1/2 each)
  const int x0 = ix >> 1, x1 = (ix + 1) >> 1, y0 = iy >> 1, y1 = (iy + 1) >> 1;
  const int z0 = (D == 3) ? (iz >> 1) : 0, z1 = (D == 3) ? ((iz + 1) >> 1) : 0;
  const T w = ((x0 == x1) ? (T)1 : (T)0.5) * ((y0 == y1) ? (T)1 : (T)0.5) * ((z0 == z1) ? (T)1 : (T)0.5);
  for (int Z = z0; Z <= z1; ++Z)
    for (int Y = y0; Y <= y1; ++Y)
      for (int X = x0; X <= x1; ++X) {
        const long long J = X + (long long)c.nx1 * (Y + (long long)c.ny1 * Z);
#pragma unroll
        for (int a = 0; a < B; ++a) acc[a] += w * c.z[J * B + a];
      }
#pragma unroll
  for (int a = 0; a < B; ++a) {
    const long long d = i * B + a;
    out[d] = zf[d] + (f.fixed[d] ? (T)0 : acc[a]);
  }
}

// zout = zin + w D^-1 (b - A zin)  (the stored inverses carry w)
template <int D, class T, int B, bool COH>
__device__ __forceinline__ void row_smooth(const MgLevel<T>& l, int row, const T* b, const T* zin, T* zout,
                                           unsigned live) {
  const long long i = l.K.rows[row];
  T y[B], res[B], z[B];
  stencil_row_product<D, T, B, COH>(l.K, row, i, l.nx1, l.ny1, zin, y);
#pragma unroll
  for (int a = 0; a < B; ++a) res[a] = b[i * B + a] - y[a];
  precond_apply<B, T>(l.K, row, res, z, live);
#pragma unroll
  for (int a = 0; a < B; ++a) zout[i * B + a] = zin[i * B + a] + z[a];
}

// z = A^-1 b on the dense level (L == 1: the finest level itself), by one
// block; bv is shared scratch of MG_DENSE_MAX entries.  Ends with a block
// barrier.
template <class T, int B>
__device__ __forceinline__ void block_dense_apply(const MgLevel<T>& c, const float* invT, const T* b, T* z,
                                                  float* bv) {
  const int n = *c.K.nrow * B;
  if (n <= 0 || n > MG_DENSE_MAX) return;
  for (int k = threadIdx.x; k < n; k += blockDim.x) bv[k] = (float)b[(long long)c.K.rows[k / B] * B + k % B];
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    float s = 0.0f;
    for (int j = 0; j < n; ++j) s += invT[j * n + k] * bv[j];
    z[(long long)c.K.rows[k / B] * B + k % B] = (T)s;
  }
  __syncthreads();
}

// ---- per-level kernels (one launch per V-cycle step) ----

template <class T, int B>
__global__ void __launch_bounds__(MG_DENSE_MAX) k_mg_dense_apply(MgLevel<T> c, const float* __restrict__ invT,
                                                                 const T* b, T* z, const int* done) {
  if (is_done(done)) return;
  __shared__ float bv[MG_DENSE_MAX];
  block_dense_apply<T, B>(c, invT, b, z, bv);
}

template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_residual(MgLevel<T> l, const T* b, const T* z, T* r, const int* done) {
  if (is_done(done)) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *l.K.nrow) return;
  row_residual<D, T, B, false>(l, row, b, z, r);
}

template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_restrict(MgLevel<T> f, const T* rf, MgLevel<T> c, int presmooth,
                                                      const int* done) {
  if (is_done(done)) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *c.K.nrow) return;
  row_restrict<D, T, B>(f, rf, c, row, presmooth != 0);
}

template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_prolong(MgLevel<T> f, const T* zf, MgLevel<T> c, T* out,
                                                     const int* done) {
  if (is_done(done)) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= *f.K.nrow) return;
  row_prolong<D, T, B>(f, zf, c, out, row);
}

template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_smooth(MgLevel<T> l, const T* b, const T* zin, T* zout,
                                                    const int* done) {
  if (is_done(done)) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = *l.K.nrow;
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  if (row >= nrow) return;
  row_smooth<D, T, B, false>(l, row, b, zin, zout, live);
}

// Levels mg.tail .. L-1 of the V-cycle in one thread-block cluster: the
// coarse levels are too small to fill the GPU, so their steps run back to
// back, separated by cluster barriers (release/acquire at cluster scope, which
// makes the global-memory writes of one step visible to every block of the
// cluster), instead of one launch each.  On entry level `tail` holds its
// right-hand side and first smoothing sweep (written by the restriction
// above); on exit its corrected, post-smoothed z.  Coarse levels use node
// blocks, so the smoother needs no warp exchange.  Every block reads the
// same done flag, so either all return or none does.
template <int D, class T, int B>
__global__ void __launch_bounds__(MG_TAIL_TPB) k_mg_tail(const __grid_constant__ MgApply<T> mg, const int* done) {
  if (is_done(done)) return;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float bv[MG_DENSE_MAX];
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, ts = gridDim.x * blockDim.x;
  const int L = mg.L, l0 = mg.tail;
  for (int l = l0; l + 1 < L; ++l) {
    const MgLevel<T>& f = mg.lev[l];
    const MgLevel<T>& c = mg.lev[l + 1];
    const int nf = *f.K.nrow, nc = *c.K.nrow;
    for (int row = t0; row < nf; row += ts) row_residual<D, T, B, true>(f, row, f.b, f.z, f.r);
    cl.sync();
    for (int row = t0; row < nc; row += ts) row_restrict<D, T, B>(f, f.r, c, row, l + 2 < L);
    cl.sync();
  }
  {
    const MgLevel<T>& c = mg.lev[L - 1];
    const int n = *c.K.nrow * B;
    if (n > 0 && n <= MG_DENSE_MAX) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) bv[k] = (float)c.b[(long long)c.K.rows[k / B] * B + k % B];
      __syncthreads();
      for (int k = t0; k < n; k += ts) {
        float s = 0.0f;
        for (int j = 0; j < n; ++j) s += mg.invT[j * n + k] * bv[j];
        c.z[(long long)c.K.rows[k / B] * B + k % B] = (T)s;
      }
    }
    cl.sync();
  }
  for (int l = L - 2; l >= l0; --l) {
    const MgLevel<T>& f = mg.lev[l];
    const MgLevel<T>& c = mg.lev[l + 1];
    const int nf = *f.K.nrow;
    for (int row = t0; row < nf; row += ts) row_prolong<D, T, B>(f, f.z, c, f.r, row);
    cl.sync();
    for (int row = t0; row < nf; row += ts) row_smooth<D, T, B, true>(f, row, f.b, f.r, f.z, 0u);
    cl.sync();
  }
}

inline int nblk_rows(int cap) { return (cap + MTPB - 1) / MTPB; }
}  // namespace

template <int D>
cudaError_t launch_mg_flags(int fx, int fy, int fz, const int* n2r_f, int cx, int cy, long long nc, int* flag,
                            cudaStream_t st) {
  k_mg_flags<D><<<(unsigned)((nc + 1 + 255) / 256), 256, 0, st>>>(fx, fy, fz, n2r_f, cx, cy, nc, flag);
  return cudaGetLastError();
}

template <int D, int B>
cudaError_t launch_mg_fixed(int fx, int fy, int fz, const int* n2r_f, const uint8_t* fix_f, int cx, int cy,
                            long long nc, uint8_t* fix_c, cudaStream_t st) {
  if (nc == 0) return cudaSuccess;
  k_mg_fixed<D, B><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(fx, fy, fz, n2r_f, fix_f, cx, cy, nc, fix_c);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_mg_galerkin(MgLevel<T> f, MgLevel<T> c, int nrow_c, cudaStream_t st) {
  if (nrow_c <= 0) return cudaSuccess;
  constexpr int S = (D == 2) ? 25 : 125;
  dim3 grid((unsigned)nblk_rows(nrow_c), S);
  k_mg_galerkin<D, T, B><<<grid, MTPB, 0, st>>>(f, c);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_mg_power(MgLevel<T> l, int cap, T* va, T* vb, double* nrm, int iters, double* part,
                            unsigned* ticket, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(nrm, 0, (iters + 1) * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int nb = nblk_rows(cap);
  k_mg_power_init<D, T, B><<<nb, MTPB, 0, st>>>(l, va, nrm, part, ticket);
  for (int k = 0; k < iters; ++k) {
    const T* src = (k & 1) ? vb : va;
    T* dst = (k & 1) ? va : vb;
    k_mg_power<D, T, B><<<nb, MTPB, 0, st>>>(l, src, dst, nrm + k, nrm + k + 1, part, ticket);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_mg_scale(T* dinv, long long n, const double* nrm, double c, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mg_scale<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dinv, n, nrm, c);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_mg_dense_inverse(MgLevel<T> c, float* invT, cudaStream_t st) {
  const int bytes = MG_DENSE_MAX * 2 * MG_DENSE_MAX * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_mg_dense_inverse<D, T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes);
  if (e != cudaSuccess) return e;
  k_mg_dense_inverse<D, T, B><<<1, 1024, bytes, st>>>(c, invT);
  return cudaGetLastError();
}

template <int D, class T, int B>
cudaError_t launch_mg_vcycle(const MgApply<T>& mg, const T* b0, T* z0, const int* done, cudaStream_t st) {
  const int L = mg.L;
  if (L < 1) return cudaSuccess;
  const MgLevel<T>* lev = mg.lev;
  if (L == 1) {
    k_mg_dense_apply<T, B><<<1, MG_DENSE_MAX, 0, st>>>(lev[0], mg.invT, b0, z0, done);
    return cudaGetLastError();
  }
  const int l0 = std::min(std::max(mg.tail, 1), L - 1);
  // level 0: MG_NU0 smoothing sweeps before and after the coarse correction
  // (the first pre-sweep is fused into the Krylov kernel that produced z0);
  // lev[0].z is a scratch vector there
  const T* zc0 = z0;
  for (int k = 1; k < MG_NU0; ++k) {
    T* dst = (k & 1) ? lev[0].z : z0;
    k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(lev[0], b0, zc0, dst, done);
    zc0 = dst;
  }
  // down to the tail: residual, restriction (+ the next level's first sweep)
  for (int l = 0; l < l0; ++l) {
    const T* b = (l == 0) ? b0 : lev[l].b;
    const T* z = (l == 0) ? zc0 : lev[l].z;
    k_mg_residual<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], b, z, lev[l].r, done);
    k_mg_restrict<D, T, B><<<nblk_rows(mg.caps[l + 1]), MTPB, 0, st>>>(lev[l], lev[l].r, lev[l + 1],
                                                                       (l + 2 < L) ? 1 : 0, done);
  }
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)mg.cluster);
    cfg.blockDim = dim3(MG_TAIL_TPB);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)mg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_mg_tail<D, T, B>, mg, done);
    if (e != cudaSuccess) return e;
  }
  // up from the tail: prolongation into the residual buffer, post-smoothing
  for (int l = l0 - 1; l >= 1; --l) {
    k_mg_prolong<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], lev[l].z, lev[l + 1], lev[l].r, done);
    k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], lev[l].b, lev[l].r, lev[l].z, done);
  }
  k_mg_prolong<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(lev[0], zc0, lev[1], lev[0].r, done);
  {
    // sweeps r -> (z scratch -> r ...) -> z0, the last one into z0
    const T* src = lev[0].r;
    for (int k = 0; k < MG_NU0; ++k) {
      T* dst = (k == MG_NU0 - 1) ? z0 : ((src == lev[0].r) ? lev[0].z : lev[0].r);
      k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(lev[0], b0, src, dst, done);
      src = dst;
    }
  }
  return cudaGetLastError();
}

// Blocks of the tail cluster: 16 (a non-portable cluster size) where the
// device can co-schedule such a cluster of the tail kernel, else 8.
template <int D, class T, int B>
int mg_tail_cluster() {
  static std::atomic<int> c{0};   // scenes of several host threads (serving) may ask at once
  if (const int v = c.load()) return v;
  int size = 8;
  if (cudaFuncSetAttribute(k_mg_tail<D, T, B>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(MG_TAIL_TPB);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_tail<D, T, B>, &cfg) == cudaSuccess && nclusters >= 1)
      size = 16;
  }
  cudaGetLastError();
  c.store(size);
  return size;
}

int mg_vcycle_launches(int L, int tail) {
  if (L <= 1) return 1;
  return 4 * std::min(std::max(tail, 1), L - 1) + 1 + 2 * (MG_NU0 - 1);
}

#define MPM_MG_INST(D, T, B)                                                                                   \
  template cudaError_t launch_mg_galerkin<D, T, B>(MgLevel<T>, MgLevel<T>, int, cudaStream_t);                \
  template cudaError_t launch_mg_power<D, T, B>(MgLevel<T>, int, T*, T*, double*, int, double*, unsigned*,  \
                                                cudaStream_t);                                           \
  template cudaError_t launch_mg_dense_inverse<D, T, B>(MgLevel<T>, float*, cudaStream_t);                    \
  template cudaError_t launch_mg_vcycle<D, T, B>(const MgApply<T>&, const T*, T*, const int*, cudaStream_t); \
  template int mg_tail_cluster<D, T, B>();
MPM_MG_INST(2, float, 2)
MPM_MG_INST(2, double, 2)
MPM_MG_INST(3, float, 3)
MPM_MG_INST(3, double, 3)
MPM_MG_INST(2, float, 3)
MPM_MG_INST(2, double, 3)
template cudaError_t launch_mg_flags<2>(int, int, int, const int*, int, int, long long, int*, cudaStream_t);
template cudaError_t launch_mg_flags<3>(int, int, int, const int*, int, int, long long, int*, cudaStream_t);
template cudaError_t launch_mg_fixed<2, 2>(int, int, int, const int*, const uint8_t*, int, int, long long,
                                           uint8_t*, cudaStream_t);
template cudaError_t launch_mg_fixed<3, 3>(int, int, int, const int*, const uint8_t*, int, int, long long,
                                           uint8_t*, cudaStream_t);
template cudaError_t launch_mg_fixed<2, 3>(int, int, int, const int*, const uint8_t*, int, int, long long,
                                           uint8_t*, cudaStream_t);
template cudaError_t launch_mg_scale<float>(float*, long long, const double*, double, cudaStream_t);
template cudaError_t launch_mg_scale<double>(double*, long long, const double*, double, cudaStream_t);

}  // namespace mpm
