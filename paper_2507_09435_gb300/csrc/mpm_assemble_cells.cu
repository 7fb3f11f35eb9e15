// Assembly of the 3D single-phase Jacobian (a4) in two phases, both
// owner-computes, with no atomics:
//
//   1. k_cell_blocks: for every occupied cell c (the base node shared by its
//      particles) the block product of all 27 x 27 node pairs of its
//      particles' stencils,
//        K^c_ij[a][b] = sum_{p in c} sum_{c', e} G_ip[c'] A_p[a][c'][b][e] G_jp[e],
//      with G_ip = grad w_ip and A_p[a][c'][b][e] = dP_p[a][c'] / d dF_p[b][e]
//      the particle's consistent tangent (written by the residual pass,
//      entry-major: A[k * np + p], k = 27a + 9c' + 3b + e).  Written as a
//      matrix product per cell,
//        K^c[(i, ab)][j] = sum_{(p, e)} U[(i, ab)][(p, e)] G_jp[e],
//        U[(i, ab)][(p, e)] = sum_{c'} G_ip[c'] A_p[a][c'][b][e],
//      (M = 27 x 9 = 243, N = 27, K = 3 x particles), it runs on the FP32 (or
//      FP64) FMA pipe with register tiles: a CTA of 96 threads per cell,
//      particles staged in chunks of CB_Q, 81 threads each owning a 9 x 9
//      output tile (the nine (a, b) of one node i and nine nodes j: 81
//      multiply-adds per six 4-wide shared-memory loads).
//      The cell's block is stored at blk[cellpos * CBLK + 243 i + 9 j + ab].
//   2. k_gather_rows: one warp per active row (node i) adds, in a fixed cell
//      order, the 27 x 9 entries of its 27 cells (cell i - k holds node i at
//      stencil position k) into its 125 slot blocks (warp-private shared
//      memory) and stores the row; blocks coupling to an inactive node (below
//      the activity threshold, not an unknown of the step) are stored as
//      zeros.
//
// The cell blocks make a round trip through HBM (27 x 27 x 9 values per
// occupied cell, written once and read once), in exchange for a dense,
// register-tiled contraction: the row-by-row form recontracts each particle
// for each of its 27 rows and keeps only about half of a warp's lanes busy.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int CB_TPB = 96;    // threads per cell (81 own an output tile)
constexpr int CB_Q = 8;       // particles per staged chunk
constexpr int CB_AST = 84;    // tangent row stride in shared memory (81 used)
constexpr int CB_UST = 12;    // (a, b) stride of U in shared memory (9 used)
constexpr int CB_TILES = 27 * 3;   // output tiles: node i x group of nine nodes j
constexpr int CBLK = CELL_BLOCK_VALUES;
static_assert(CBLK >= 27 * 243 && CBLK % 4 == 0, "cell block layout");

template <class T>
struct CellSmem {
  T A[CB_Q][CB_AST];             // tangents of the chunk's particles
  T W[CB_Q][3][8];               // per particle and axis: N0..2, 0, dN0..2 (x 1/h), 0
  T GT[CB_Q][3][3][12];          // the same as [p][e][j / 9][j % 9] (+ pad), the GEMM's B
  T U[CB_Q * 3][27][CB_UST];     // U[(p, e)][i][ab] (+ pad)
};

template <class T>
__device__ __forceinline__ void lds4(const T* p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
  } else {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 w = *(reinterpret_cast<const double2*>(p) + 1);
    v[0] = u.x; v[1] = u.y; v[2] = w.x; v[3] = w.y;
  }
}

template <class T>
__global__ void __launch_bounds__(CB_TPB, sizeof(T) == 4 ? 5 : 2) k_cell_blocks(DevParticles P, DevGrid G, const int* __restrict__ cells,
                                                       int ncell, const int* __restrict__ cstart,
                                                       const T* __restrict__ A, T* __restrict__ blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem<T>& sm = *reinterpret_cast<CellSmem<T>*>(smem_raw);
  const int tid = threadIdx.x;
  const T ih = (T)G.ih;
  const long long plane = (long long)G.nx1 * G.ny1;
  int cb = blockIdx.x;
  if (cb >= ncell) return;
  // the chunk being staged: cell, its base node, particle range, first particle
  int cell = cells[cb], p1 = cstart[cell + 1], q0 = cstart[cell];
  // registers of the next chunk's loads (issued a chunk ahead): tangent
  // entries idx = tid + CB_TPB m of the CB_Q x 81 block, and one coordinate
  constexpr int NPF = (CB_Q * 81 + CB_TPB - 1) / CB_TPB;
  T pf[NPF];
  double px = 0.0;
  auto prefetch = [&](int qq0, int nq) {
#pragma unroll
    for (int m = 0; m < NPF; ++m) {
      const int idx = tid + CB_TPB * m, k = idx / CB_Q, q = idx - CB_Q * k;
      pf[m] = (idx < CB_Q * 81 && q < nq) ? A[(long long)k * P.np + qq0 + q] : (T)0;
    }
    if (tid < 3 * CB_Q) {
      const int q = tid / 3, a = tid - 3 * q;
      if (q < nq) px = (a == 0) ? P.x[0][qq0 + q] : ((a == 1) ? P.x[1][qq0 + q] : P.x[2][qq0 + q]);
    }
  };
  prefetch(q0, min(CB_Q, p1 - q0));
  // this thread's tile (tid < CB_TILES): node i = tid / 3, nodes j = 9 (tid %
  // 3) + jj, all nine (a, b)
  T acc[9][9];
#pragma unroll
  for (int ab = 0; ab < 9; ++ab)
#pragma unroll
    for (int jj = 0; jj < 9; ++jj) acc[ab][jj] = (T)0;
  for (;;) {
    const int nq = min(CB_Q, p1 - q0);
    const int cx = cell % G.nx1, cy = (int)((cell / G.nx1) % G.ny1), cz = (int)(cell / plane);
    __syncthreads();   // the previous chunk's readers are done
    // 1. stage the chunk: tangents (zeros past the last particle) and the
    //    B-spline factors of each particle and axis
#pragma unroll
    for (int m = 0; m < NPF; ++m) {
      const int idx = tid + CB_TPB * m, k = idx / CB_Q, q = idx - CB_Q * k;
      if (idx < CB_Q * 81) sm.A[q][k] = pf[m];
    }
    if (tid < 3 * CB_Q) {
      const int q = tid / 3, a = tid - 3 * q;
      T* w = sm.W[q][a];
      if (q < nq) {
        const int base = (a == 0) ? cx : ((a == 1) ? cy : cz);
        const double oa = (a == 0) ? G.o[0] : ((a == 1) ? G.o[1] : G.o[2]);
        const T t = (T)((px - oa) * G.ih - (double)base - 0.5);
        const T u = (T)1 - t, cm = t - (T)0.5;
        w[0] = (T)0.5 * u * u; w[1] = (T)0.75 - cm * cm; w[2] = (T)0.5 * t * t; w[3] = (T)0;
        w[4] = -u * ih; w[5] = (T)-2 * cm * ih; w[6] = t * ih; w[7] = (T)0;
      } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) w[m] = (T)0;
      }
    }
    // the next chunk (of this cell, else the next cell of this CTA) and its loads
    const int cb_cur = cb;
    const bool cell_done = q0 + CB_Q >= p1;
    bool more = true;
    if (!cell_done) {
      q0 += CB_Q;
    } else {
      cb += gridDim.x;
      more = cb < ncell;
      if (more) {
        cell = cells[cb];
        q0 = cstart[cell];
        p1 = cstart[cell + 1];
      }
    }
    if (more) prefetch(q0, min(CB_Q, p1 - q0));
    __syncthreads();
    // 2. per (q, i): G_iq[c'] from the factors (node i = kx + 3 ky + 9 kz),
    //    its copy as the product's B operand, and U[(q, e)][i][ab] =
    //    sum_c' G_iq[c'] A_q[a][c'][b][e]
    for (int t = tid; t < CB_Q * 27; t += CB_TPB) {
      const int q = t / 27, i = t - 27 * q;
      const int kx = i % 3, ky = (i / 3) % 3, kz = i / 9;
      const T* wx = sm.W[q][0];
      const T* wy = sm.W[q][1];
      const T* wz = sm.W[q][2];
      const T g0 = wx[4 + kx] * wy[ky] * wz[kz];
      const T g1 = wx[kx] * wy[4 + ky] * wz[kz];
      const T g2 = wx[kx] * wy[ky] * wz[4 + kz];
      const int gg = i / 9, jj = i - 9 * gg;
      sm.GT[q][0][gg][jj] = g0;
      sm.GT[q][1][gg][jj] = g1;
      sm.GT[q][2][gg][jj] = g2;
      if (jj < 3) {   // the pad entries 9..11
        sm.GT[q][0][gg][9 + jj] = (T)0;
        sm.GT[q][1][gg][9 + jj] = (T)0;
        sm.GT[q][2][gg][9 + jj] = (T)0;
      }
      const T* aq = sm.A[q];
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int o = (ab / 3) * 27 + (ab % 3) * 3;
#pragma unroll
        for (int e = 0; e < 3; ++e)
          sm.U[q * 3 + e][i][ab] = g0 * aq[o + e] + g1 * aq[o + 9 + e] + g2 * aq[o + 18 + e];
      }
    }
    __syncthreads();
    // 3. the tile: acc[ab][jj] += U[(q, e)][i][ab] G_jq[e], j = 9 g + jj
    if (tid < CB_TILES) {
      const int i = tid / 3, g = tid - 3 * i;
#pragma unroll 2
      for (int k = 0; k < CB_Q * 3; ++k) {
        T uv[12], gj[12];
        lds4<T>(&sm.U[k][i][0], uv);
        lds4<T>(&sm.U[k][i][4], uv + 4);
        lds4<T>(&sm.U[k][i][8], uv + 8);
        lds4<T>(&sm.GT[k / 3][k % 3][g][0], gj);
        lds4<T>(&sm.GT[k / 3][k % 3][g][4], gj + 4);
        lds4<T>(&sm.GT[k / 3][k % 3][g][8], gj + 8);
#pragma unroll
        for (int ab = 0; ab < 9; ++ab)
#pragma unroll
          for (int jj = 0; jj < 9; ++jj) acc[ab][jj] += uv[ab] * gj[jj];
      }
    }
    if (cell_done) {
      // the cell's block, [i][j][ab], through shared memory (U is free once
      // every tile has read it) for full-width stores
      __syncthreads();
      T* so = &sm.U[0][0][0];
      if (tid < CB_TILES) {
        const int i = tid / 3, g = tid - 3 * i;
        T* o = so + i * 243 + g * 81;
#pragma unroll
        for (int jj = 0; jj < 9; ++jj)
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) o[jj * 9 + ab] = acc[ab][jj];
      }
#pragma unroll
      for (int ab = 0; ab < 9; ++ab)
#pragma unroll
        for (int jj = 0; jj < 9; ++jj) acc[ab][jj] = (T)0;
      __syncthreads();
      T* out = blk + (long long)cb_cur * CBLK;
      if constexpr (sizeof(T) == 4) {
        for (int v = tid; v < CBLK / 4; v += CB_TPB)
          reinterpret_cast<float4*>(out)[v] = reinterpret_cast<const float4*>(so)[v];
      } else {
        for (int v = tid; v < CBLK / 2; v += CB_TPB)
          reinterpret_cast<double2*>(out)[v] = reinterpret_cast<const double2*>(so)[v];
      }
    }
    if (!more) break;
  }
}

constexpr int GR_WARPS = 8;   // rows (warps) per CTA of the gather

template <class T>
__global__ void __launch_bounds__(GR_WARPS * 32) k_gather_rows(DevGrid G, const int* __restrict__ count,
                                                              const int* __restrict__ cellpos,
                                                              const int* __restrict__ node2row,
                                                              const T* __restrict__ blk, DevMatrix<T> K,
                                                              int nrow) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* acc = reinterpret_cast<T*>(smem_raw) + warp * (125 * 9);
  const long long plane = (long long)G.nx1 * G.ny1;
  // entry e = 9 jl + ab of a cell's block row (jl = jx + 3 jy + 9 jz) lands
  // at acc[off_k + rel(e)], rel(e) = 9 (jx + 5 jy + 25 jz) + ab and off_k = 9
  // ((2 - kx) + 5 (2 - ky) + 25 (2 - kz)) for the row's stencil position k;
  // lane l handles e = l + 32 m
  int rel[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int e = lane + 32 * m, jl = e / 9, ab = e - 9 * jl;
    rel[m] = (e < 243) ? 9 * (jl % 3 + 5 * ((jl / 3) % 3) + 25 * (jl / 9)) + ab : -1;
  }
  for (int row = blockIdx.x * GR_WARPS + warp; row < nrow; row += gridDim.x * GR_WARPS) {
    const long long i = K.rows[row];
    const int ix = (int)(i % G.nx1), iy = (int)((i / G.nx1) % G.ny1), iz = (int)(i / plane);
    for (int t = lane; t < 125 * 9; t += 32) acc[t] = (T)0;
    // lane k < 27: the block of cell i - k (k = kx + 3 ky + 9 kz), or -1
    long long mine = -1;
    if (lane < 27) {
      const int kx = lane % 3, ky = (lane / 3) % 3, kz = lane / 9;
      const int cxx = ix - kx, cyy = iy - ky, czz = iz - kz;
      if (cxx >= 0 && cyy >= 0 && czz >= 0) {
        const long long cell = cxx + (long long)G.nx1 * (cyy + (long long)G.ny1 * czz);
        if (count[cell] > 0) mine = (long long)cellpos[cell] * CBLK + lane * 243;
      }
    }
    // live slots (neighbour inside the grid and active), 32 per word
    unsigned live[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int slot = lane + 32 * w;
      bool ok = false;
      if (slot < 125) {
        const int jx = ix + slot % 5 - 2, jy = iy + (slot / 5) % 5 - 2, jz = iz + slot / 25 - 2;
        ok = jx >= 0 && jy >= 0 && jz >= 0 && jx < G.nx1 && jy < G.ny1 && jz < G.nz1 &&
             node2row[jx + (long long)G.nx1 * (jy + (long long)G.ny1 * jz)] >= 0;
      }
      live[w] = __ballot_sync(0xffffffffu, ok);
    }
    __syncwarp();
    // the occupied cells among the 27 in a fixed order (increasing k), the
    // next cell's entries loaded while the current one is added
    unsigned todo = __ballot_sync(0xffffffffu, mine >= 0);
    T v[8], vn[8];
    auto load = [&](int k, T* dst) {
      const T* b = blk + __shfl_sync(0xffffffffu, mine, k);
#pragma unroll
      for (int m = 0; m < 8; ++m) dst[m] = (rel[m] >= 0) ? __ldcs(b + lane + 32 * m) : (T)0;
    };
    int k = todo ? __ffs(todo) - 1 : -1;
    if (k >= 0) {
      load(k, v);
      todo &= todo - 1;
    }
    while (k >= 0) {
      const int kn = todo ? __ffs(todo) - 1 : -1;
      if (kn >= 0) {
        load(kn, vn);
        todo &= todo - 1;
      }
      const int kx = k % 3, ky = (k / 3) % 3, kz = k / 9;
      const int off = 9 * ((2 - kx) + 5 * ((2 - ky) + 5 * (2 - kz)));
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (rel[m] >= 0) acc[off + rel[m]] += v[m];
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = vn[m];
      k = kn;
    }
    // the row: 9 consecutive values per slot plane
    for (int t = lane; t < 125 * 9; t += 32) {
      const int slot = t / 9, e = t - 9 * slot;
      const unsigned lw = (slot < 32) ? live[0] : ((slot < 64) ? live[1] : ((slot < 96) ? live[2] : live[3]));
      const bool ok = (lw >> (slot & 31)) & 1u;
      K.val[((long long)slot * K.cap + row) * 9 + e] = ok ? acc[t] : (T)0;
    }
    __syncwarp();
  }
}

template <class T>
cudaError_t occupancy_grid(const void* fn, int threads, size_t bytes, long long need, int& nblk) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, bytes);
  if (e != cudaSuccess) return e;
  nblk = (int)std::max<long long>(1, std::min<long long>(need, (long long)sms * std::max(1, per_sm)));
  return cudaSuccess;
}
}  // namespace

template <class T>
cudaError_t launch_assemble_cells3(const DevParticles& P, const DevGrid& G, const Asm3<T>& a3, const int* cstart,
                                   const int* node2row, const T* A, DevMatrix<T> K, int nrow_host,
                                   cudaStream_t st) {
  if (P.np == 0 || nrow_host <= 0 || a3.ncell <= 0) return cudaSuccess;
  const size_t b1 = sizeof(CellSmem<T>);
  static_assert(sizeof(CellSmem<T>) <= 227 * 1024, "cell CTA too large");
  cudaError_t e = cudaFuncSetAttribute(k_cell_blocks<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1);
  if (e != cudaSuccess) return e;
  int nb1 = 0;
  e = occupancy_grid<T>((const void*)k_cell_blocks<T>, CB_TPB, b1, a3.ncell, nb1);
  if (e != cudaSuccess) return e;
  k_cell_blocks<T><<<nb1, CB_TPB, b1, st>>>(P, G, a3.cells, a3.ncell, cstart, A, a3.blk);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t b2 = sizeof(T) * 125 * 9 * GR_WARPS;
  e = cudaFuncSetAttribute(k_gather_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2);
  if (e != cudaSuccess) return e;
  int nb2 = 0;
  e = occupancy_grid<T>((const void*)k_gather_rows<T>, GR_WARPS * 32, b2, (nrow_host + GR_WARPS - 1) / GR_WARPS, nb2);
  if (e != cudaSuccess) return e;
  k_gather_rows<T><<<nb2, GR_WARPS * 32, b2, st>>>(G, a3.count, a3.cellpos, node2row, a3.blk, K, nrow_host);
  return cudaGetLastError();
}

template cudaError_t launch_assemble_cells3<float>(const DevParticles&, const DevGrid&, const Asm3<float>&,
                                                   const int*, const int*, const float*, DevMatrix<float>, int,
                                                   cudaStream_t);
template cudaError_t launch_assemble_cells3<double>(const DevParticles&, const DevGrid&, const Asm3<double>&,
                                                    const int*, const int*, const double*, DevMatrix<double>,
                                                    int, cudaStream_t);

}  // namespace mpm
