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
// ticket.  The nb blocks of one sum (bid: this block's place among them)
// call this once each.
__device__ __forceinline__ void grid_add(double v, double* out, double* part, unsigned* ticket, int bid, int nb) {
  __shared__ double sh[MTPB / 32];
  __shared__ int last;
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < MTPB / 32; ++q) t += sh[q];
    part[bid] = t;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == (unsigned)nb - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += MTPB) t += __ldcg(&part[b]);
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

// Level of block b in a power-iteration set (start: first block per level).
__device__ __forceinline__ int set_level(const int* start, int n, int b) {
  int l = 0;
  while (l + 1 < n && b >= start[l + 1]) ++l;
  return l;
}

// v = a fixed pseudo-random start vector (zero on prescribed DOFs), with
// ||v||^2, for every level of the set at once
template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_power_init(const __grid_constant__ MgPowerSet<T> ps, double* nrm,
                                                        int stride, double* part, unsigned* tickets) {
  const int lv = set_level(ps.start, ps.n, blockIdx.x);
  const int bid = blockIdx.x - ps.start[lv], nb = ps.start[lv + 1] - ps.start[lv];
  const MgLevel<T>& l = ps.lev[lv];
  T* v = ps.va[lv];
  const int row = bid * blockDim.x + threadIdx.x;
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
  grid_add(acc, nrm + (long long)lv * stride, part + ps.start[lv], tickets + lv, bid, nb);
}

// Step k of every level's power iteration: dst = D^-1 A src / ||src||,
// accumulating ||dst||^2 (D^-1: the unscaled block-Jacobi inverse, node
// blocks or row segments; src, dst alternate between va and vb)
template <int D, class T, int B>
__global__ void __launch_bounds__(MTPB) k_mg_power(const __grid_constant__ MgPowerSet<T> ps, int k, double* nrm,
                                                   int stride, double* part, unsigned* tickets) {
  const int lv = set_level(ps.start, ps.n, blockIdx.x);
  const int bid = blockIdx.x - ps.start[lv], nb = ps.start[lv + 1] - ps.start[lv];
  const MgLevel<T>& l = ps.lev[lv];
  const T* src = (k & 1) ? ps.vb[lv] : ps.va[lv];
  T* dst = (k & 1) ? ps.va[lv] : ps.vb[lv];
  double* nl = nrm + (long long)lv * stride;
  const int row = bid * blockDim.x + threadIdx.x;
  const int nrow = *l.K.nrow;
  const unsigned live = __ballot_sync(0xffffffffu, row < nrow);
  const double n2 = nl[k];
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
  grid_add(acc, nl + k + 1, part + ps.start[lv], tickets + lv, bid, nb);
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
// Gauss-Jordan elimination with partial pivoting, in place, one block of 32
// warps with the matrix in registers: warp w holds columns w + 32 s (s < 4),
// lane l rows l + 32 q (q < 4).  Rows are not swapped: the pivot of column k
// is the largest remaining entry of the column among the rows not chosen yet
// (ties: the lowest row).  Its row p_k is divided by it and column k is
// eliminated from every other row; on [A | I] that makes column k of the
// left half e_{p_k} and column p_k of the right half the first nonzero one
// in the rows other than p_k, so that right-half column is stored in column
// k's registers (ip in row p_k, -a_rk ip in the others, the same operations
// as on [A | I]).  At the end [A | I] has become [P | R] with P e_k = e_{p_k},
// so (A^-1)[k][j] = R[p_k][j], and R[r][p_c] sits in column c.  The warp that
// owns column k + 1 picks its pivot right after eliminating column k and
// stages the column (double-buffered), the pivot row and the pivot's
// reciprocal ip in shared memory, so one block barrier per column suffices.  A pivot that vanishes is replaced by 1 (the
// preconditioner stays defined).  Written transposed:
// invT[j*n + k] = (A^-1)[k][j].
__device__ __forceinline__ void gj_select(const float (&a)[4][4], unsigned used, int col, int n,
                                          float (*fac)[MG_DENSE_MAX], int* prow, float* pinv) {
  const int lane = threadIdx.x & 31, sc = col >> 5;
  float best = -1.0f, bval = 0.0f;
  int bi = 1 << 30;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float x = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s == sc) x = a[q][s];
    const int r = lane + 32 * q;
    if (r < n) fac[col & 1][r] = x;
    if (!((used >> q) & 1u)) {
      float v = fabsf(x);
      if (!(v >= 0.0f)) v = -0.5f;   // NaN: still a candidate, after every number
      if (v > best) { best = v; bi = r; bval = x; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    const float ov = __shfl_xor_sync(0xffffffffu, bval, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bval = ov; }
  }
  if (lane == 0) {
    const float m = fabsf(bval);
    const bool bad = !(m > 1e-30f) || !(m < 3e38f);
    prow[col] = bi;
    pinv[col] = bad ? 1.0f : 1.0f / bval;
  }
}

template <int D, class T, int B>
__global__ void __launch_bounds__(1024) k_mg_dense_inverse(MgLevel<T> c, float* invT) {
  extern __shared__ float A[];   // A[r * n + k]
  __shared__ float fac[2][MG_DENSE_MAX];
  __shared__ float pinv[MG_DENSE_MAX];   // 1 / pivot (1 for a vanishing pivot)
  __shared__ int prow[MG_DENSE_MAX], kof[MG_DENSE_MAX];
  const int nrow = *c.K.nrow;
  const int n = nrow * B;
  if (n <= 0 || n > MG_DENSE_MAX) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.0f;
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
      for (int y = 0; y < B; ++y) A[(rr * B + x) * n + cc * B + y] = (float)blk[x * B + y];
  }
  __syncthreads();
  float a[4][4];
  unsigned used = 0;   // bit q: row lane + 32 q is a pivot row already (or beyond n)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = lane + 32 * q;
    if (r >= n) used |= 1u << q;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int col = w + 32 * s;
      a[q][s] = (r < n && col < n) ? A[r * n + col] : 0.0f;
    }
  }
  if (w == 0) gj_select(a, used, 0, n, fac, prow, pinv);
  for (int col = 0; col < n; ++col) {
    __syncthreads();
    const int p = prow[col];
    const float ip = pinv[col];
    const int pl = p & 31, pq = p >> 5;   // the same for the whole block
    float f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = lane + 32 * q;
      f[q] = (r < n && r != p) ? fac[col & 1][r] : 0.0f;
    }
    // the normalised pivot row on this warp's columns (ip on column col)
    float pr[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      float t = a[0][s];
      if (pq == 1) t = a[1][s];
      if (pq == 2) t = a[2][s];
      if (pq == 3) t = a[3][s];
      t = __shfl_sync(0xffffffffu, t, pl);
      pr[s] = (w + 32 * s == col) ? ip : t * ip;
    }
    // column col leaves the left half; right-half column p takes its place
    // (zero off the pivot row before the elimination)
    if (w == (col & 31)) {
      const int sc = col >> 5;
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (s == sc) a[q][s] = 0.0f;
    }
    // eliminate (f = 0 on the pivot row, which is then replaced)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int s = 0; s < 4; ++s) a[q][s] -= f[q] * pr[s];
    if (lane == pl) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q == pq) {
#pragma unroll
          for (int s = 0; s < 4; ++s) a[q][s] = pr[s];
        }
      used |= 1u << pq;
    }
    if (col + 1 < n && w == ((col + 1) & 31)) gj_select(a, used, col + 1, n, fac, prow, pinv);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) kof[prow[k]] = k;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = lane + 32 * q;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int col = w + 32 * s;
      if (r < n && col < n) invT[prow[col] * n + kof[r]] = a[q][s];
    }
  }
}

// ---- one row of each V-cycle step (used by the per-level kernels and by the
// cluster tail; COH: the input vector was written earlier in the same kernel,
// so it is read with ordinary loads; GEN: the level's matrix is staged in
// shared memory, so it is read with ordinary loads too)

// r = b - A z
template <int D, class T, int B, bool COH, bool GEN = false>
__device__ __forceinline__ void row_residual(const MgLevel<T>& l, int row, const T* b, const T* z, T* r) {
  const long long i = l.K.rows[row];
  T y[B];
  stencil_row_product<D, T, B, COH, GEN>(l.K, row, i, l.nx1, l.ny1, z, y);
#pragma unroll
  for (int a = 0; a < B; ++a) r[i * B + a] = b[i * B + a] - y[a];
}

// b_c = P^T r_f for coarse row `row`; with `presmooth`, also the first
// smoothing sweep of the coarse level from zero, z_c = w D_c^-1 b_c (coarse
// levels use node blocks)
template <int D, class T, int B, bool GEN = false>
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
    precond_apply<B, T, GEN>(c.K, row, acc, z, 0u);
#pragma unroll
    for (int a = 0; a < B; ++a) c.z[J * B + a] = z[a];
  }
}

// v = z_f + P z_c at fine node i (prescribed DOFs keep z_f)
template <int D, class T, int B>
__device__ __forceinline__ void prolong_value(const MgLevel<T>& f, const T* zf, const MgLevel<T>& c, long long i,
                                              T v[B]) {
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
    v[a] = zf[d] + (f.fixed[d] ? (T)0 : acc[a]);
  }
}

// out = z_f + P z_c for fine row `row`
template <int D, class T, int B>
__device__ __forceinline__ void row_prolong(const MgLevel<T>& f, const T* zf, const MgLevel<T>& c, T* out, int row) {
  const long long i = f.K.rows[row];
  T v[B];
  prolong_value<D, T, B>(f, zf, c, i, v);
#pragma unroll
  for (int a = 0; a < B; ++a) out[i * B + a] = v[a];
}

// zout = zin + w D^-1 (b - A zin)  (the stored inverses carry w)
template <int D, class T, int B, bool COH, bool GEN = false>
__device__ __forceinline__ void row_smooth(const MgLevel<T>& l, int row, const T* b, const T* zin, T* zout,
                                           unsigned live) {
  const long long i = l.K.rows[row];
  T y[B], res[B], z[B];
  stencil_row_product<D, T, B, COH, GEN>(l.K, row, i, l.nx1, l.ny1, zin, y);
#pragma unroll
  for (int a = 0; a < B; ++a) res[a] = b[i * B + a] - y[a];
  precond_apply<B, T, GEN>(l.K, row, res, z, live);
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

// ---- fused 2D steps of the levels above the tail (node tiles; node-block
// smoother).  Each computes exactly what the two kernels it replaces compute,
// in the same order, without the round trip of the intermediate vector
// through memory and without a launch.

// Coarse nodes per tile of the fused residual + restriction, and the fine
// nodes the tile reads (2 TX + 1 by 2 TY + 1, at most one per thread).
constexpr int RR_TX = 8, RR_TY = 7, RR_FX = 2 * RR_TX + 1, RR_FY = 2 * RR_TY + 1;
constexpr int RR_TPB = 256;
static_assert(RR_FX * RR_FY <= RR_TPB, "one fine node per thread");

// r_f = b - A_f z on the fine nodes under a tile of coarse nodes (in shared
// memory; zero at prescribed DOFs, nodes without a row and outside the
// grid, which the restriction skips), then b_c = P^T r_f and, with
// `presmooth`, z_c = w D_c^-1 b_c for the tile's coarse rows.
template <class T, int B>
__global__ void __launch_bounds__(RR_TPB) k_mg_residual_restrict(MgLevel<T> f, const T* b, const T* z, MgLevel<T> c,
                                                                 int presmooth, const int* done) {
  if (is_done(done)) return;
  __shared__ T rs[RR_FX * RR_FY * B];
  const int X0 = blockIdx.x * RR_TX, Y0 = blockIdx.y * RR_TY, t = threadIdx.x;
  if (t < RR_FX * RR_FY) {
    const int ix = 2 * X0 - 1 + t % RR_FX, iy = 2 * Y0 - 1 + t / RR_FX;
    T r[B];
#pragma unroll
    for (int a = 0; a < B; ++a) r[a] = (T)0;
    if (ix >= 0 && iy >= 0 && ix < f.nx1 && iy < f.ny1) {
      const long long i = ix + (long long)f.nx1 * iy;
      const int row = f.node2row[i];
      if (row >= 0) {
        T y[B];
        stencil_row_product<2, T, B>(f.K, row, i, f.nx1, f.ny1, z, y);
#pragma unroll
        for (int a = 0; a < B; ++a) r[a] = f.fixed[i * B + a] ? (T)0 : b[i * B + a] - y[a];
      }
    }
#pragma unroll
    for (int a = 0; a < B; ++a) rs[t * B + a] = r[a];
  }
  __syncthreads();
  if (t >= RR_TX * RR_TY) return;
  const int X = X0 + t % RR_TX, Y = Y0 + t / RR_TX;
  if (X >= c.nx1 || Y >= c.ny1) return;
  const long long J = X + (long long)c.nx1 * Y;
  const int crow = c.node2row[J];
  if (crow < 0) return;
  T acc[B];
#pragma unroll
  for (int a = 0; a < B; ++a) acc[a] = (T)0;
  for (int sy = -1; sy <= 1; ++sy) {
    const int iy = 2 * Y + sy;
    if (iy < 0 || iy >= f.ny1) continue;
    for (int sx = -1; sx <= 1; ++sx) {
      const int ix = 2 * X + sx;
      if (ix < 0 || ix >= f.nx1) continue;
      const T w = (T)(wt1(sx) * wt1(sy) * wt1(0));
      const T* rv = &rs[((iy - 2 * Y0 + 1) * RR_FX + (ix - 2 * X0 + 1)) * B];
#pragma unroll
      for (int a = 0; a < B; ++a) acc[a] += w * rv[a];
    }
  }
#pragma unroll
  for (int a = 0; a < B; ++a) c.b[J * B + a] = acc[a];
  if (presmooth) {
    T zc[B];
    precond_apply<B, T>(c.K, crow, acc, zc, 0u);
#pragma unroll
    for (int a = 0; a < B; ++a) c.z[J * B + a] = zc[a];
  }
}

// Fine nodes per tile side of the fused prolongation + smoothing sweep, and
// with the stencil's halo of 2.
constexpr int PS_T = 16, PS_H = PS_T + 4, PS_TPB = PS_T * PS_T;

// zin = z_f + P z_c on a tile of fine nodes and its halo (in shared memory;
// zero at nodes without a row and outside the grid, which the matrix reaches
// with zero blocks only), then one sweep zout = zin + w D^-1 (b - A zin) on
// the tile's rows.
template <class T, int B>
__global__ void __launch_bounds__(PS_TPB) k_mg_prolong_smooth(MgLevel<T> f, const T* zf, MgLevel<T> c, const T* b,
                                                              T* zout, const int* done) {
  if (is_done(done)) return;
  __shared__ T zs[PS_H * PS_H * B];
  const int ix0 = blockIdx.x * PS_T, iy0 = blockIdx.y * PS_T;
  for (int k = threadIdx.x; k < PS_H * PS_H; k += PS_TPB) {
    const int hx = ix0 - 2 + k % PS_H, hy = iy0 - 2 + k / PS_H;
    T v[B];
#pragma unroll
    for (int a = 0; a < B; ++a) v[a] = (T)0;
    if (hx >= 0 && hy >= 0 && hx < f.nx1 && hy < f.ny1) {
      const long long i = hx + (long long)f.nx1 * hy;
      if (f.node2row[i] >= 0) prolong_value<2, T, B>(f, zf, c, i, v);
    }
#pragma unroll
    for (int a = 0; a < B; ++a) zs[k * B + a] = v[a];
  }
  __syncthreads();
  const int ix = ix0 + threadIdx.x % PS_T, iy = iy0 + threadIdx.x / PS_T;
  if (ix >= f.nx1 || iy >= f.ny1) return;
  const long long i = ix + (long long)f.nx1 * iy;
  const int row = f.node2row[i];
  if (row < 0) return;
  // the stencil product of row_smooth, its neighbours' zin from the tile
  const int cl = (threadIdx.x / PS_T + 2) * PS_H + (threadIdx.x % PS_T + 2);
  T y[B];
#pragma unroll
  for (int a = 0; a < B; ++a) y[a] = (T)0;
  const long long cap = f.K.cap;
  unsigned pm[1];
  load_pmask<2>(f.K.pmask, row, pm);
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const int slot = (dx + 2) + 5 * (dy + 2);
      const bool on = (pm[0] >> slot) & 1u;
      T xj[B], kb[B * B];
      if (on) {
#pragma unroll
        for (int q = 0; q < B; ++q) xj[q] = zs[(cl + dx + PS_H * dy) * B + q];
        ld_block<B, T>(&f.K.val[((long long)slot * cap + row) * (B * B)], kb);
      } else {
#pragma unroll
        for (int q = 0; q < B; ++q) xj[q] = (T)0;
#pragma unroll
        for (int q = 0; q < B * B; ++q) kb[q] = (T)0;
      }
#pragma unroll
      for (int a = 0; a < B; ++a)
#pragma unroll
        for (int q = 0; q < B; ++q) y[a] += kb[a * B + q] * xj[q];
    }
  T res[B], zz[B];
#pragma unroll
  for (int a = 0; a < B; ++a) res[a] = b[i * B + a] - y[a];
  precond_apply<B, T>(f.K, row, res, zz, 0u);
#pragma unroll
  for (int a = 0; a < B; ++a) zout[i * B + a] = zs[cl * B + a] + zz[a];
}

// ---- staging of the small coarse levels in the tail's shared memory

// Copies `bytes` (a multiple of 4) from global to shared memory by
// asynchronous copies spread over the block: 16 bytes each when both ends are
// 16-byte aligned and the length is whole 16-byte units, else 4 bytes each.
__device__ __forceinline__ void stage_async(unsigned char* dst, const void* src, int bytes) {
  const unsigned char* g = static_cast<const unsigned char*>(src);
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(g) | (uintptr_t)bytes) & 15u) == 0) {
    for (int k = threadIdx.x * 16; k < bytes; k += blockDim.x * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst + k)),
                   "l"(g + k)
                   : "memory");
  } else {
    for (int k = threadIdx.x * 4; k + 4 <= bytes; k += blockDim.x * 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst + k)),
                   "l"(g + k)
                   : "memory");
  }
}

__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Starts the copies of the staged levels' row lists, blocks, block inverses,
// maps and flags and of the dense inverse, and zeroes their vectors (nodes
// without a row and the padding read as zero, like the global vectors' zero
// blocks against them).
template <class T>
__device__ __forceinline__ void tail_stage(const MgApply<T>& mg, unsigned char* sm) {
  for (int l = mg.staged; l < mg.L; ++l) {
    const MgStage& g = mg.stg[l];
    const MgLevel<T>& v = mg.lev[l];
    const void* src[5] = {v.K.rows, v.K.val, v.K.dinv, v.node2row, v.fixed};
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (g.off[k] >= 0) stage_async(sm + g.off[k], src[k], g.len[k]);
#pragma unroll
    for (int k = 5; k < 8; ++k)
      if (g.off[k] >= 0) {
        uint4* d = reinterpret_cast<uint4*>(sm + g.off[k]);
        const int n16 = (g.len[k] + 15) / 16;
        for (int q = threadIdx.x; q < n16; q += blockDim.x) d[q] = make_uint4(0u, 0u, 0u, 0u);
      }
  }
  if (mg.inv_len > 0) stage_async(sm + mg.inv_off, mg.invT, mg.inv_len);
}

// Level l with its staged arrays in place of the global ones.
template <class T>
__device__ __forceinline__ MgLevel<T> staged_level(const MgApply<T>& mg, int l, unsigned char* sm) {
  MgLevel<T> v = mg.lev[l];
  const MgStage& g = mg.stg[l];
  v.K.rows = reinterpret_cast<const int*>(sm + g.off[0]);
  if (g.off[1] >= 0) v.K.val = reinterpret_cast<T*>(sm + g.off[1]);
  if (g.off[2] >= 0) v.K.dinv = reinterpret_cast<T*>(sm + g.off[2]);
  if (g.off[3] >= 0) v.node2row = reinterpret_cast<const int*>(sm + g.off[3]);
  if (g.off[4] >= 0) v.fixed = sm + g.off[4];
  v.b = reinterpret_cast<T*>(sm + g.off[5]) + g.vpad;
  v.z = reinterpret_cast<T*>(sm + g.off[6]) + g.vpad;
  if (g.off[7] >= 0) v.r = reinterpret_cast<T*>(sm + g.off[7]) + g.vpad;
  return v;
}

// z = A^-1 b on the dense level, spread over `nt` threads from thread `t`;
// bv holds b in row order (shared, MG_DENSE_MAX entries).
template <class T, int B>
__device__ __forceinline__ void dense_rows(const MgLevel<T>& c, const float* invT, const float* bv, int n, int t,
                                           int nt) {
  for (int k = t; k < n; k += nt) {
    float s = 0.0f;
    for (int j = 0; j < n; ++j) s += invT[j * n + k] * bv[j];
    c.z[(long long)c.K.rows[k / B] * B + k % B] = (T)s;
  }
}

// Rows of a cluster step for this block: an equal contiguous share of the
// level's n rows per block (so that small levels spread over every SM of the
// cluster), one row per thread and pass.
__device__ __forceinline__ int row_lo(int n) {
  return blockIdx.x * ((n + (int)gridDim.x - 1) / (int)gridDim.x) + threadIdx.x;
}
__device__ __forceinline__ int row_hi(int n) {
  return min(n, (int)(blockIdx.x + 1) * ((n + (int)gridDim.x - 1) / (int)gridDim.x));
}

// Levels mg.tail .. L-1 of the V-cycle in one thread-block cluster: the
// coarse levels are too small to fill the GPU, so their steps run back to
// back, separated by cluster barriers (release/acquire at cluster scope, which
// makes the global-memory writes of one step visible to every block of the
// cluster), instead of one launch each.  The levels from mg.staged down are
// copied into every block's shared memory while the levels above run; each
// block then restricts into them, runs their whole V-cycle (down to the dense
// solve and back) by itself between block barriers, and prolongs out of its
// own copy, so that these levels cost no cluster barrier and no L2 round
// trip.  Every block computes the same values in the same order, so the
// copies agree bit for bit, and the result is the same as running those
// levels across the cluster.  On entry level `tail` holds its right-hand
// side and first smoothing sweep (written by the restriction above); on exit
// its corrected, post-smoothed z.  Coarse levels use node blocks, so the
// smoother needs no warp exchange.  Every block reads the same done flag, so
// either all return or none does.
template <int D, class T, int B>
__global__ void __launch_bounds__(mg_tail_tpb<T, B>()) k_mg_tail(const __grid_constant__ MgApply<T> mg, const int* done) {
  if (is_done(done)) return;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float bv[MG_DENSE_MAX];
  extern __shared__ __align__(16) unsigned char tsm[];
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, ts = gridDim.x * blockDim.x;
  const int L = mg.L, l0 = mg.tail;
  const int ls = (mg.staged > l0 && mg.staged < L) ? mg.staged : L;   // first staged level (L: none)
  if (ls < L) tail_stage<T>(mg, tsm);
  // down through the cluster levels
  for (int l = l0; l + 1 < L && l < ls; ++l) {
    const MgLevel<T>& f = mg.lev[l];
    const int nf = *f.K.nrow;
    for (int row = row_lo(nf); row < row_hi(nf); row += blockDim.x)
      row_residual<D, T, B, true>(f, row, f.b, f.z, f.r);
    cl.sync();
    if (l + 1 < ls) {
      const MgLevel<T>& c = mg.lev[l + 1];
      const int nc = *c.K.nrow;
      for (int row = row_lo(nc); row < row_hi(nc); row += blockDim.x)
        row_restrict<D, T, B>(f, f.r, c, row, l + 2 < L);
      cl.sync();
    }
  }
  if (ls == L) {
    // dense level across the cluster
    const MgLevel<T>& c = mg.lev[L - 1];
    const int n = *c.K.nrow * B;
    if (n > 0 && n <= MG_DENSE_MAX) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) bv[k] = (float)c.b[(long long)c.K.rows[k / B] * B + k % B];
      __syncthreads();
      dense_rows<T, B>(c, mg.invT, bv, n, t0, ts);
    }
    cl.sync();
  } else {
    // staged levels, in full in every block
    stage_wait();
    __syncthreads();
    {
      const MgLevel<T>& f = mg.lev[ls - 1];
      const MgLevel<T> c = staged_level<T>(mg, ls, tsm);
      const int nc = *c.K.nrow;
      for (int row = threadIdx.x; row < nc; row += blockDim.x)
        row_restrict<D, T, B, true>(f, f.r, c, row, ls + 1 < L);
      __syncthreads();
    }
    for (int l = ls; l + 1 < L; ++l) {
      const MgLevel<T> f = staged_level<T>(mg, l, tsm), c = staged_level<T>(mg, l + 1, tsm);
      const int nf = *f.K.nrow, nc = *c.K.nrow;
      for (int row = threadIdx.x; row < nf; row += blockDim.x)
        row_residual<D, T, B, true, true>(f, row, f.b, f.z, f.r);
      __syncthreads();
      for (int row = threadIdx.x; row < nc; row += blockDim.x)
        row_restrict<D, T, B, true>(f, f.r, c, row, l + 2 < L);
      __syncthreads();
    }
    {
      const MgLevel<T> c = staged_level<T>(mg, L - 1, tsm);
      const int n = *c.K.nrow * B;
      if (n > 0 && n <= MG_DENSE_MAX && n * n * (int)sizeof(float) <= mg.inv_len) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) bv[k] = (float)c.b[(long long)c.K.rows[k / B] * B + k % B];
        __syncthreads();
        dense_rows<T, B>(c, reinterpret_cast<const float*>(tsm + mg.inv_off), bv, n, threadIdx.x, blockDim.x);
      }
      __syncthreads();
    }
    for (int l = L - 2; l >= ls; --l) {
      const MgLevel<T> f = staged_level<T>(mg, l, tsm), c = staged_level<T>(mg, l + 1, tsm);
      const int nf = *f.K.nrow;
      for (int row = threadIdx.x; row < nf; row += blockDim.x) row_prolong<D, T, B>(f, f.z, c, f.r, row);
      __syncthreads();
      for (int row = threadIdx.x; row < nf; row += blockDim.x)
        row_smooth<D, T, B, true, true>(f, row, f.b, f.r, f.z, 0u);
      __syncthreads();
    }
  }
  // up through the cluster levels (the first prolongation from the staged
  // copy, when there is one); the kernel's end orders the last sweep
  for (int l = (ls < L) ? ls - 1 : L - 2; l >= l0; --l) {
    const MgLevel<T>& f = mg.lev[l];
    const int nf = *f.K.nrow;
    if (l + 1 == ls) {
      const MgLevel<T> c = staged_level<T>(mg, ls, tsm);
      for (int row = row_lo(nf); row < row_hi(nf); row += blockDim.x) row_prolong<D, T, B>(f, f.z, c, f.r, row);
    } else {
      const MgLevel<T>& c = mg.lev[l + 1];
      for (int row = row_lo(nf); row < row_hi(nf); row += blockDim.x) row_prolong<D, T, B>(f, f.z, c, f.r, row);
    }
    cl.sync();
    for (int row = row_lo(nf); row < row_hi(nf); row += blockDim.x)
      row_smooth<D, T, B, true>(f, row, f.b, f.r, f.z, 0u);
    if (l > l0) cl.sync();
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

int mg_power_blocks(const int* caps, int n) {
  int nb = 0;
  for (int l = 0; l < n; ++l) nb += nblk_rows(caps[l]);
  return nb;
}

template <int D, class T, int B>
cudaError_t launch_mg_power(MgPowerSet<T> ps, const int* caps, double* nrm, int iters, double* part,
                            unsigned* tickets, cudaStream_t st) {
  if (ps.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(nrm, 0, (size_t)ps.n * (iters + 1) * sizeof(double), st);
  if (e != cudaSuccess) return e;
  ps.start[0] = 0;
  for (int l = 0; l < ps.n; ++l) ps.start[l + 1] = ps.start[l] + nblk_rows(caps[l]);
  const int nb = ps.start[ps.n];
  k_mg_power_init<D, T, B><<<nb, MTPB, 0, st>>>(ps, nrm, iters + 1, part, tickets);
  for (int k = 0; k < iters; ++k) k_mg_power<D, T, B><<<nb, MTPB, 0, st>>>(ps, k, nrm, iters + 1, part, tickets);
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
  const int bytes = MG_DENSE_MAX * MG_DENSE_MAX * (int)sizeof(float);
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
  const bool fused = (D == 2) && mg.fused;
  for (int l = 0; l < l0; ++l) {
    const T* b = (l == 0) ? b0 : lev[l].b;
    const T* z = (l == 0) ? zc0 : lev[l].z;
    const int pre = (l + 2 < L) ? 1 : 0;
    if (fused) {
      const dim3 g((unsigned)((lev[l + 1].nx1 + RR_TX - 1) / RR_TX), (unsigned)((lev[l + 1].ny1 + RR_TY - 1) / RR_TY));
      k_mg_residual_restrict<T, B><<<g, RR_TPB, 0, st>>>(lev[l], b, z, lev[l + 1], pre, done);
    } else {
      k_mg_residual<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], b, z, lev[l].r, done);
      k_mg_restrict<D, T, B><<<nblk_rows(mg.caps[l + 1]), MTPB, 0, st>>>(lev[l], lev[l].r, lev[l + 1], pre, done);
    }
  }
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)mg.cluster);
    cfg.blockDim = dim3(mg_tail_tpb<T, B>());
    cfg.dynamicSmemBytes = (size_t)(mg.staged < L ? mg.smem : 0);
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
  // up from the tail: prolongation into the residual buffer, post-smoothing;
  // fused, the prolongation stays in shared memory and the sweep writes the
  // residual buffer (its input z is still being read by neighbouring tiles),
  // so `cz` is the coarse level as the next prolongation reads it
  MgLevel<T> cz = lev[l0];
  for (int l = l0 - 1; l >= 1; --l) {
    if (fused) {
      const dim3 g((unsigned)((lev[l].nx1 + PS_T - 1) / PS_T), (unsigned)((lev[l].ny1 + PS_T - 1) / PS_T));
      k_mg_prolong_smooth<T, B><<<g, PS_TPB, 0, st>>>(lev[l], lev[l].z, cz, lev[l].b, lev[l].r, done);
      cz = lev[l];
      cz.z = lev[l].r;
    } else {
      k_mg_prolong<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], lev[l].z, cz, lev[l].r, done);
      k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[l]), MTPB, 0, st>>>(lev[l], lev[l].b, lev[l].r, lev[l].z, done);
      cz = lev[l];
    }
  }
  {
    // sweeps r -> (z scratch -> r ...) -> z0, the last one into z0 (fused:
    // the prolongation and the first sweep into r, as zc0 may be the z
    // scratch)
    const T* src = lev[0].r;
    int k = 0;
    if (fused) {
      const dim3 g((unsigned)((lev[0].nx1 + PS_T - 1) / PS_T), (unsigned)((lev[0].ny1 + PS_T - 1) / PS_T));
      k_mg_prolong_smooth<T, B><<<g, PS_TPB, 0, st>>>(lev[0], zc0, cz, b0, lev[0].r, done);
      k = 1;
    } else {
      k_mg_prolong<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(lev[0], zc0, cz, lev[0].r, done);
    }
    for (; k < MG_NU0; ++k) {
      T* dst = (k == MG_NU0 - 1) ? z0 : ((src == lev[0].r) ? lev[0].z : lev[0].r);
      k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(lev[0], b0, src, dst, done);
      src = dst;
    }
  }
  return cudaGetLastError();
}

// Blocks of the tail cluster: 16 (a non-portable cluster size) where the
// device can co-schedule such a cluster of the tail kernel with its largest
// staging, else 8.  *staging: whether the kernel may take MG_TAIL_SMEM_MAX
// bytes of dynamic shared memory (set here).
template <int D, class T, int B>
int mg_tail_cluster(bool* staging) {
  // scenes of several host threads (serving) may ask at once
  static std::atomic<int> c{0};
  static std::atomic<bool> smem_ok{false};
  if (const int v = c.load()) {
    *staging = smem_ok.load();
    return v;
  }
  int size = 8;
  const bool ok = cudaFuncSetAttribute(k_mg_tail<D, T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MG_TAIL_SMEM_MAX) == cudaSuccess;
  cudaGetLastError();
  if (cudaFuncSetAttribute(k_mg_tail<D, T, B>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(mg_tail_tpb<T, B>());
    cfg.dynamicSmemBytes = ok ? MG_TAIL_SMEM_MAX : 0;
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
  smem_ok.store(ok);
  c.store(size);
  *staging = ok;
  return size;
}

template <int D, class T, int B>
cudaError_t launch_mg_apply(const MgApply<T>& mg, const T* b0, const T* zero, T* z0, cudaStream_t st) {
  if (mg.L >= 2) {
    k_mg_smooth<D, T, B><<<nblk_rows(mg.caps[0]), MTPB, 0, st>>>(mg.lev[0], b0, zero, z0, nullptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_mg_vcycle<D, T, B>(mg, b0, z0, nullptr, st);
}

int mg_vcycle_launches(int L, int tail, int fused) {
  if (L <= 1) return 1;
  const int l0 = std::min(std::max(tail, 1), L - 1);
  return (fused ? 2 : 4) * l0 + 1 + 2 * (MG_NU0 - 1);
}

#define MPM_MG_INST(D, T, B)                                                                                   \
  template cudaError_t launch_mg_galerkin<D, T, B>(MgLevel<T>, MgLevel<T>, int, cudaStream_t);                \
  template cudaError_t launch_mg_power<D, T, B>(MgPowerSet<T>, const int*, double*, int, double*, unsigned*, \
                                                cudaStream_t);                                            \
  template cudaError_t launch_mg_dense_inverse<D, T, B>(MgLevel<T>, float*, cudaStream_t);                    \
  template cudaError_t launch_mg_vcycle<D, T, B>(const MgApply<T>&, const T*, T*, const int*, cudaStream_t); \
  template cudaError_t launch_mg_apply<D, T, B>(const MgApply<T>&, const T*, const T*, T*, cudaStream_t);   \
  template int mg_tail_cluster<D, T, B>(bool*);
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
