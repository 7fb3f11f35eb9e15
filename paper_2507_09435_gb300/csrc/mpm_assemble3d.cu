// Assembly of the 3D single-phase Jacobian (a4): one warp per triple of
// x-neighbouring node rows.
//
// Row i of J holds the 125 blocks K_ij = sum_p G_ip^T A_p G_jp over the
// particles whose 27-node B-spline stencil contains i, where A_p[a][c][b][e] =
// dP_p[a][c] / d dF_p[b][e] is the particle's consistent tangent (written by
// the residual pass) and G_ip[c] the gradient of w_ip.  Those particles sit
// in the 27 cells (base nodes) i - (kx, ky, kz), k in {0,1,2}^3; in cell
// i - k, node i is node k of every particle's stencil and node j of the
// stencil lands in slot (j - k + 2) of row i.
//
// Owner computes, with no atomics and no block-wide barrier: a warp owns the
// rows (ix0 + r, iy, iz), r = 0, 1, 2, ix0 a multiple of 3 (the triples with
// an active row, listed once per load step by k_triple_leaders and taken in
// a grid-stride loop; inactive rows are skipped), keeps their
// 3 x 125 x 9 accumulator in warp-private shared memory, and walks the 45
// cells (5 along x, 3 along y and z) that reach any of them, in batches of
// QB particles (a batch is always QB: missing particles are zeros):
//   1. the batch's tangents are copied to shared memory (coalesced over
//      particles: A is stored entry-major, A[k * np + p]; the next batch's
//      loads are issued into registers before the current batch is
//      processed), each particle's per-axis B-spline weights and derivatives
//      are evaluated (FP64 offset from the base node, then the working type
//      T), and G_ip of the triple's rows;
//   2. lane (ab, r), ab = 3a + b < 9, r < 3, whose row r is reached by the
//      cell, forms U[e] = sum_c G_ip[c] A_p[a][c][b][e] and adds K_j[a][b] =
//      sum_e U[e] G_jp[e] for all 27 stencil nodes j into 27 registers, by
//      the tensor-product form of G_jp (dN carrying 1/h):
//        K_j = Nz(jz) (Ny(jy) U0 dNx(jx) + dNy(jy) U1 Nx(jx))
//            + dNz(jz) Ny(jy) U2 Nx(jx);
//      every loaded tangent entry and B-spline factor serves 27 outputs;
//   3. after the cell, the lanes add their registers into the slots of
//      their row; after the triple, the warp stores its rows.
#include <algorithm>

#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int R3_QB = 8;   // particles per staged batch
constexpr int R3_NC = 45;  // cells reaching a row triple: 5 x 3 x 3

template <class T>
struct R3Cfg;
template <>
struct R3Cfg<float> {
  static constexpr int WARPS = 4;
};
template <>
struct R3Cfg<double> {
  static constexpr int WARPS = 2;
};

// Warp-private shared memory, in elements of T; every vector-read region
// starts at a multiple of 4 elements (16 bytes for float, 32 for double).
// The tangent rows are padded to 84 entries: the staging stores (lanes: 8
// particles x 4 consecutive entries) then hit 32 distinct banks.
struct R3Smem {
  static constexpr int AST = 84;                     // tangent row stride
  static constexpr int GI = 0;                       // [QB][3 rows][4] G_ip
  static constexpr int SW = GI + R3_QB * 3 * 4;      // [QB][3 axes][8] N0..2, 0, dN0..2 / h, 0
  static constexpr int SA = SW + R3_QB * 3 * 8;      // [QB][AST] tangents
  static constexpr int ACC = SA + R3_QB * AST;       // [3 rows][125][9] the rows' blocks
  static constexpr int PER_WARP = (ACC + 3 * 125 * 9 + 3) / 4 * 4;
};

template <class T>
__device__ __forceinline__ void lds4v(const T* p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
  } else {
    const double2 u = reinterpret_cast<const double2*>(p)[0];
    const double2 w = reinterpret_cast<const double2*>(p)[1];
    v[0] = u.x; v[1] = u.y; v[2] = w.x; v[3] = w.y;
  }
}

template <class T>
__device__ __forceinline__ void sts4v(T* p, T a, T b, T c, T d) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
}
}  // namespace

template <class T>
__global__ void __launch_bounds__(R3Cfg<T>::WARPS * 32, 3)
    k_assemble_rows3(DevParticles P, DevGrid G, const int* __restrict__ cstart,
                     const int* __restrict__ node2row, const T* __restrict__ A, DevMatrix<T> K,
                     const int* __restrict__ tri, const int* __restrict__ ntri) {
  constexpr int W = R3Cfg<T>::WARPS;
  using L = R3Smem;
  constexpr int AST = L::AST;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* wbase = sm + warp * L::PER_WARP;
  T* sGi = wbase + L::GI;
  T* sW = wbase + L::SW;
  T* sA = wbase + L::SA;
  T* acc = wbase + L::ACC;
  // lane < 27: (ab, r) with ab = 3a + b, the tangent offset a*27 + b*3, and
  // the lane's row r of the triple
  const int ab = lane % 9, lr = lane / 9;
  const int ao = (ab / 3) * 27 + (ab % 3) * 3;
  constexpr int NPF = (81 + 32 / R3_QB - 1) / (32 / R3_QB);   // tangent loads per lane per batch
  const int lq = lane & (R3_QB - 1), lk = lane / R3_QB;
  const T ih = (T)G.ih;
  const long long plane = (long long)G.nx1 * G.ny1;
  const int ntask = *ntri;
  for (int task = blockIdx.x * W + warp; task < ntask; task += gridDim.x * W) {
    // the triple holding the node of row tri[task], its first active row
    const long long i = K.rows[tri[task]];
    const int ixr = (int)(i % G.nx1), iy = (int)((i / G.nx1) % G.ny1), iz = (int)(i / plane);
    const int ix0 = ixr - ixr % 3;
    // the triple's rows (-1: inactive or outside the grid); every lane holds all three
    int rowof[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int ix = ix0 + r;
      rowof[r] = (ix < G.nx1) ? node2row[ix + (long long)G.nx1 * (iy + (long long)G.ny1 * iz)] : -1;
    }
    const bool myrow_live = (lr == 0) ? rowof[0] >= 0 : ((lr == 1) ? rowof[1] >= 0 : (lr == 2 && rowof[2] >= 0));
    for (int t = lane; t < 3 * 125 * 9; t += 32) acc[t] = (T)0;
    // cell c = xo + 5 (ky + 3 kz): base node (ix0 - 2 + xo, iy - ky, iz - kz);
    // lanes c and c + 32 look up their particle ranges, the warp reads them by
    // shuffles
    int my_pb[2] = {0, 0}, my_pe[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (c < R3_NC) {
        const int cx = ix0 - 2 + c % 5, cy = iy - (c / 5) % 3, cz = iz - c / 15;
        if (cx >= 0 && cy >= 0 && cz >= 0 && cx < G.nx1) {
          const long long cell = cx + (long long)G.nx1 * (cy + (long long)G.ny1 * cz);
          my_pb[h] = cstart[cell];
          my_pe[h] = cstart[cell + 1];
        }
      }
    }
    int c = 0, q0 = 0, pe = 0;
    auto seek = [&](int from) {   // first non-empty cell >= from (R3_NC: none)
      for (c = from; c < R3_NC; ++c) {
        const int b0 = __shfl_sync(0xffffffffu, my_pb[0], c & 31);
        const int e0 = __shfl_sync(0xffffffffu, my_pe[0], c & 31);
        const int b1 = __shfl_sync(0xffffffffu, my_pb[1], c & 31);
        const int e1 = __shfl_sync(0xffffffffu, my_pe[1], c & 31);
        q0 = (c < 32) ? b0 : b1;
        pe = (c < 32) ? e0 : e1;
        if (q0 < pe) return;
      }
    };
    T pf[NPF];
    double px = 0.0;
    auto prefetch = [&](int qq0, int nq) {
#pragma unroll
      for (int m = 0; m < NPF; ++m) {
        const int k = lk + (32 / R3_QB) * m;
        pf[m] = (lq < nq && k < 81) ? A[(long long)k * P.np + qq0 + lq] : (T)0;
      }
      if (lane < 3 * nq) {
        const int q = lane / 3, a = lane - 3 * (lane / 3);
        // (selects, not a dynamic index into the parameter arrays)
        const double* xa = (a == 0) ? P.x[0] : ((a == 1) ? P.x[1] : P.x[2]);
        px = xa[qq0 + q];
      }
    };
    seek(0);
    if (c < R3_NC) prefetch(q0, min(R3_QB, pe - q0));
    T kr[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) kr[k] = (T)0;
    while (c < R3_NC) {
      const int cc = c, nq = min(R3_QB, pe - q0);
      __syncwarp();   // the previous batch's readers are done
      // a batch is always QB particles: the slots past nq hold zeros (their
      // G_ip and B-spline factors are zero too)
#pragma unroll
      for (int m = 0; m < NPF; ++m) {
        const int k = lk + (32 / R3_QB) * m;
        if (k < 81) sA[lq * AST + k] = pf[m];
      }
      const double pxc = px;
      // advance to the next item and start its loads
      if (q0 + R3_QB < pe) {
        q0 += R3_QB;
      } else {
        seek(c + 1);
      }
      if (c < R3_NC) prefetch(q0, min(R3_QB, pe - q0));
      const int xo = cc % 5, ky = (cc / 5) % 3, kz = cc / 15;
      if (lane < 3 * R3_QB) {
        const int q = lane / 3, a = lane - 3 * (lane / 3);
        // two 4-wide stores per lane (scalar stores at an 8-element stride
        // would serialise on a quarter of the banks)
        if (q < nq) {
          const int base = (a == 0) ? ix0 - 2 + xo : ((a == 1) ? iy - ky : iz - kz);
          const double oa = (a == 0) ? G.o[0] : ((a == 1) ? G.o[1] : G.o[2]);
          const T t = (T)((pxc - oa) * G.ih - (double)base - 0.5);
          // quadratic B-spline at nodes base, base + 1, base + 2
          const T u = (T)1 - t, cm = t - (T)0.5;
          sts4v(sW + (q * 3 + a) * 8, (T)0.5 * u * u, (T)0.75 - cm * cm, (T)0.5 * t * t, (T)0);
          sts4v(sW + (q * 3 + a) * 8 + 4, -u * ih, (T)-2 * cm * ih, t * ih, (T)0);
        } else {
          sts4v(sW + (q * 3 + a) * 8, (T)0, (T)0, (T)0, (T)0);
          sts4v(sW + (q * 3 + a) * 8 + 4, (T)0, (T)0, (T)0, (T)0);
        }
      }
      __syncwarp();
      // G_ip of row r: node kx_r = r + 2 - xo of the particle's stencil
      if (lane < 3 * R3_QB) {
        const int q = lane / 3, r = lane - 3 * (lane / 3);
        const int kx = r + 2 - xo;
        const T* w = sW + q * 24;
        if (kx >= 0 && kx <= 2)
          sts4v(sGi + (q * 3 + r) * 4, w[4 + kx] * w[8 + ky] * w[16 + kz], w[kx] * w[12 + ky] * w[16 + kz],
                w[kx] * w[8 + ky] * w[20 + kz], (T)0);
      }
      __syncwarp();
      // lanes whose row is reached by this cell: r + 2 - xo in [0, 2]
      const int lkx = lr + 2 - xo;
      const bool mine = lane < 27 && lkx >= 0 && lkx <= 2 && myrow_live;
      if (mine) {
#pragma unroll
        for (int q = 0; q < R3_QB; ++q) {
          T gi[4];
          lds4v(sGi + (q * 3 + lr) * 4, gi);
          const T* aq = sA + q * AST + ao;
          T U[3];
#pragma unroll
          for (int e = 0; e < 3; ++e) U[e] = gi[0] * aq[e] + gi[1] * aq[9 + e] + gi[2] * aq[18 + e];
          const T* w = sW + q * 24;
          T nx[4], dnx[4], ny[4], dny[4], nz[4], dnz[4];
          lds4v(w, nx);
          lds4v(w + 4, dnx);
          lds4v(w + 8, ny);
          lds4v(w + 12, dny);
          lds4v(w + 16, nz);
          lds4v(w + 20, dnz);
#pragma unroll
          for (int jx = 0; jx < 3; ++jx) {
            const T a0 = U[0] * dnx[jx], a1 = U[1] * nx[jx], a2 = U[2] * nx[jx];
#pragma unroll
            for (int jy = 0; jy < 3; ++jy) {
              const T Ax = ny[jy] * a0 + dny[jy] * a1, Bx = ny[jy] * a2;
#pragma unroll
              for (int jz = 0; jz < 3; ++jz) kr[jx + 3 * jy + 9 * jz] += nz[jz] * Ax + dnz[jz] * Bx;
            }
          }
        }
      }
      if (c != cc) {
        // the cell is done: into the accumulator slots of the lane's row
        if (mine) {
          T* racc = acc + lr * (125 * 9);
#pragma unroll
          for (int jz = 0; jz < 3; ++jz)
#pragma unroll
            for (int jy = 0; jy < 3; ++jy)
#pragma unroll
              for (int jx = 0; jx < 3; ++jx) {
                const int slot = (jx - lkx + 2) + 5 * ((jy - ky + 2) + 5 * (jz - kz + 2));
                racc[slot * 9 + ab] += kr[jx + 3 * jy + 9 * jz];
              }
        }
#pragma unroll
        for (int k = 0; k < 27; ++k) kr[k] = (T)0;
      }
    }
    __syncwarp();
    // store the rows: 9 consecutive values per slot plane; blocks coupling to
    // an inactive node (below the activity threshold, not an unknown of the
    // step) are stored as zeros
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = rowof[r];
      if (row < 0) continue;
      const int ix = ix0 + r;
      for (int t = lane; t < 125 * 9; t += 32) {
        const int slot = t / 9, e = t - 9 * slot;
        const int jx = ix + slot % 5 - 2, jy = iy + (slot / 5) % 5 - 2, jz = iz + slot / 25 - 2;
        const bool live = jx >= 0 && jy >= 0 && jz >= 0 && jx < G.nx1 && jy < G.ny1 && jz < G.nz1 &&
                          node2row[jx + (long long)G.nx1 * (jy + (long long)G.ny1 * jz)] >= 0;
        K.val[((long long)slot * K.cap + row) * 9 + e] = live ? acc[r * (125 * 9) + t] : (T)0;
      }
    }
    __syncwarp();
  }
}

// one thread per row: the row is listed when it is the first active row of
// its triple (ix0 = ix - ix % 3, ix0 + 1, ix0 + 2 at the same y and z);
// warp-aggregated append
__global__ void k_triple_leaders(DevGrid G, const int* __restrict__ rows, int nrow,
                                 const int* __restrict__ node2row, int* __restrict__ list, int* __restrict__ count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  bool lead = false;
  if (r < nrow) {
    const long long i = rows[r];
    const int ix = (int)(i % G.nx1);
    const long long base = i - ix % 3;   // node of ix0 at the same y and z
    int first = -1;
    for (int k = 0; k < 3 && first < 0; ++k)
      if (ix - ix % 3 + k < G.nx1) first = node2row[base + k];
    lead = (first == r);
  }
  const unsigned m = __ballot_sync(0xffffffffu, lead);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  int at = 0;
  if (lane == __ffs(m) - 1) at = atomicAdd(count, __popc(m));
  at = __shfl_sync(0xffffffffu, at, __ffs(m) - 1);
  if (lead) list[at + __popc(m & ((1u << lane) - 1u))] = r;
}

cudaError_t launch_triple_leaders(const DevGrid& G, const int* rows, int nrow_host, const int* node2row, int* list,
                                  int* count, cudaStream_t st) {
  if (nrow_host <= 0) return cudaSuccess;
  k_triple_leaders<<<(nrow_host + 255) / 256, 256, 0, st>>>(G, rows, nrow_host, node2row, list, count);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_assemble_rows3(const DevParticles& P, const DevGrid& G, const int* cstart,
                                  const int* node2row, const T* A, DevMatrix<T> K, int nrow_host,
                                  const int* tri, const int* ntri, cudaStream_t st) {
  if (P.np == 0 || nrow_host <= 0) return cudaSuccess;
  constexpr int W = R3Cfg<T>::WARPS;
  const size_t bytes = sizeof(T) * (size_t)R3Smem::PER_WARP * W;
  static_assert(sizeof(T) * R3Smem::PER_WARP * R3Cfg<T>::WARPS <= 227 * 1024, "assembly CTA too large");
  cudaError_t e = cudaFuncSetAttribute(k_assemble_rows3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  // grid-stride warps over the row triples of the whole grid: at most the
  // CTAs that fit on the device at once
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assemble_rows3<T>, W * 32, bytes);
  if (e != cudaSuccess) return e;
  // the triples number between nrow / 3 and nrow
  const long long need = ((long long)nrow_host + W - 1) / W;
  const int nblk = (int)std::min<long long>(need, (long long)std::max(1, sms * std::max(1, per_sm)));
  k_assemble_rows3<T><<<nblk, W * 32, bytes, st>>>(P, G, cstart, node2row, A, K, tri, ntri);
  return cudaGetLastError();
}

template cudaError_t launch_assemble_rows3<float>(const DevParticles&, const DevGrid&, const int*, const int*,
                                                  const float*, DevMatrix<float>, int, const int*, const int*,
                                                  cudaStream_t);
template cudaError_t launch_assemble_rows3<double>(const DevParticles&, const DevGrid&, const int*, const int*,
                                                   const double*, DevMatrix<double>, int, const int*, const int*,
                                                   cudaStream_t);

}  // namespace mpm
