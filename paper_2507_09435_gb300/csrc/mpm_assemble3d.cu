// Assembly of the 3D single-phase Jacobian (a4): one warp per active node row.
//
// Row i of J holds the 125 blocks K_ij = sum_p G_ip^T A_p G_jp over the
// particles whose 27-node B-spline stencil contains i, where A_p[a][c][b][e] =
// dP_p[a][c] / d dF_p[b][e] is the particle's consistent tangent (written by
// the residual pass) and G_ip[c] the gradient of w_ip.  Those particles sit
// in the 27 cells (base nodes) i - (kx, ky, kz), k in {0,1,2}^3; in cell
// i - k, node i is node k of every particle's stencil and node j of the
// stencil lands in slot (j - k + 2) of row i.
//
// Owner computes, with no atomics and no block-wide barrier: each warp owns
// one row at a time (rows in a grid-stride loop, consecutive warps of a CTA
// on consecutive rows, which share two thirds of their particles through
// L1), keeps its 125 x 9 accumulator in warp-private shared memory, and walks
// its 27 cells in batches of QB particles:
//   1. the batch's tangents are copied to shared memory (coalesced over
//      particles: A is stored entry-major, A[k * np + p]; the loads of the
//      next batch are issued into registers before the current batch is
//      processed, so their latency overlaps the arithmetic) and each
//      particle's per-axis B-spline weights and derivatives are evaluated
//      (FP64 offset from the base node, then the working type T);
//   2. lane (ab, jz), ab = 3a + b < 9, jz < 3, forms U[e] = sum_c G_ip[c]
//      A_p[a][c][b][e] and adds K_j[a][b] = sum_e U[e] G_jp[e] for the nine
//      stencil nodes j = (jx, jy, jz) of its layer, using the tensor-product
//      form of G_jp: K_j = Ny(jy) (Nz U0 dNx(jx) + dNz U2 Nx(jx))
//      + dNy(jy) (Nz U1 Nx(jx)) (dN carrying 1/h), nine registers per lane;
//   3. after the cell, the lanes add their registers into the slots of
//      their nodes; after the row, the warp stores it.
#include <algorithm>

#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int R3_QB = 8;   // particles per staged batch

template <class T>
struct R3Cfg;
template <>
struct R3Cfg<float> {
  static constexpr int WARPS = 8;
};
template <>
struct R3Cfg<double> {
  static constexpr int WARPS = 4;
};

// Warp-private shared memory, in elements of T; every vector-read region
// starts at a multiple of 4 elements (16 bytes for float, 32 for double).
// The tangent rows are padded to 84 entries: the staging stores (lanes: 8
// particles x 4 consecutive entries) then hit 32 distinct banks.
struct R3Smem {
  static constexpr int AST = 84;                     // tangent row stride
  static constexpr int GI = 0;                       // [QB][4]  G_ip of each particle
  static constexpr int SW = GI + R3_QB * 4;          // [QB][3][8] per axis N0..2, 0, dN0..2 / h, 0
  static constexpr int SA = SW + R3_QB * 3 * 8;      // [QB][AST] tangents
  static constexpr int ACC = SA + R3_QB * AST;       // [125][9] the row's blocks
  static constexpr int PER_WARP = (ACC + 125 * 9 + 3) / 4 * 4;
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
                     const int* __restrict__ node2row, const T* __restrict__ A, DevMatrix<T> K, int nrow) {
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
  const long long plane = (long long)G.nx1 * G.ny1;
  // lane < 27: (ab, jz) with ab = 3a + b, and the tangent offset a*27 + b*3
  const int ab = lane % 9, jz = lane / 9;
  const int ao = (ab / 3) * 27 + (ab % 3) * 3;
  // lane < 27 also looks up cell (c % 3, c / 3 % 3, c / 9) back from the row
  const int cxk = lane % 3, cyk = (lane / 3) % 3, czk = lane / 9;
  constexpr int NPF = (81 + 32 / R3_QB - 1) / (32 / R3_QB);   // tangent loads per lane per batch
  const int lq = lane & (R3_QB - 1), lk = lane / R3_QB;
  const T ih = (T)G.ih;
  for (int row = blockIdx.x * W + warp; row < nrow; row += gridDim.x * W) {
    for (int t = lane; t < 125 * 9; t += 32) acc[t] = (T)0;
    const long long i = K.rows[row];
    const int ix = (int)(i % G.nx1), iy = (int)((i / G.nx1) % G.ny1), iz = (int)(i / plane);
    int my_pb = 0, my_pe = 0;
    if (lane < 27) {
      const int cx = ix - cxk, cy = iy - cyk, cz = iz - czk;
      if (cx >= 0 && cy >= 0 && cz >= 0) {
        const long long cell = cx + (long long)G.nx1 * (cy + (long long)G.ny1 * cz);
        my_pb = cstart[cell];
        my_pe = cstart[cell + 1];
      }
    }
    // work items: (cell c, first particle q0) batches of up to QB particles;
    // the next item's tangents and positions are loaded into registers while
    // the current one is processed from shared memory
    int c = 0, q0 = 0, pe = 0;
    auto seek = [&](int from) {   // first non-empty cell >= from (27: none)
      for (c = from; c < 27; ++c) {
        q0 = __shfl_sync(0xffffffffu, my_pb, c);
        pe = __shfl_sync(0xffffffffu, my_pe, c);
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
    if (c < 27) prefetch(q0, min(R3_QB, pe - q0));
    T kr[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) kr[k] = (T)0;
    while (c < 27) {
      const int cc = c, nq = min(R3_QB, pe - q0);
      __syncwarp();   // the previous batch's readers are done
#pragma unroll
      for (int m = 0; m < NPF; ++m) {
        const int k = lk + (32 / R3_QB) * m;
        if (lq < nq && k < 81) sA[lq * AST + k] = pf[m];
      }
      const double pxc = px;
      // advance to the next item and start its loads
      if (q0 + R3_QB < pe) {
        q0 += R3_QB;
      } else {
        seek(c + 1);
      }
      if (c < 27) prefetch(q0, min(R3_QB, pe - q0));
      const int kx = cc % 3, ky = (cc / 3) % 3, kz = cc / 9;
      if (lane < 3 * nq) {
        const int q = lane / 3, a = lane - 3 * (lane / 3);
        const int base = (a == 0) ? ix - kx : ((a == 1) ? iy - ky : iz - kz);
        const double oa = (a == 0) ? G.o[0] : ((a == 1) ? G.o[1] : G.o[2]);
        const T t = (T)((pxc - oa) * G.ih - (double)base - 0.5);
        // quadratic B-spline at nodes base, base + 1, base + 2
        const T u = (T)1 - t, cm = t - (T)0.5;
        // two 4-wide stores per lane (scalar stores at an 8-element stride
        // would serialise on a quarter of the banks)
        sts4v(sW + (q * 3 + a) * 8, (T)0.5 * u * u, (T)0.75 - cm * cm, (T)0.5 * t * t, (T)0);
        sts4v(sW + (q * 3 + a) * 8 + 4, -u * ih, (T)-2 * cm * ih, t * ih, (T)0);
      }
      __syncwarp();
      if (lane < nq) {
        const T* w = sW + lane * 24;
        sts4v(sGi + lane * 4, w[4 + kx] * w[8 + ky] * w[16 + kz], w[kx] * w[12 + ky] * w[16 + kz],
              w[kx] * w[8 + ky] * w[20 + kz], (T)0);
      }
      __syncwarp();
      if (lane < 27) {
        for (int q = 0; q < nq; ++q) {
          T gi[4];
          lds4v(sGi + q * 4, gi);
          const T* aq = sA + q * AST + ao;
          T U[3];
#pragma unroll
          for (int e = 0; e < 3; ++e) U[e] = gi[0] * aq[e] + gi[1] * aq[9 + e] + gi[2] * aq[18 + e];
          const T* w = sW + q * 24;
          T nx[4], dnx[4], ny[4], dny[4];
          lds4v(w, nx);
          lds4v(w + 4, dnx);
          lds4v(w + 8, ny);
          lds4v(w + 12, dny);
          const T nz = w[16 + jz], dnz = w[20 + jz];
          const T V0 = nz * U[0], V1 = nz * U[1], V2 = dnz * U[2];
#pragma unroll
          for (int jx = 0; jx < 3; ++jx) {
            const T Pj = V0 * dnx[jx] + V2 * nx[jx];
            const T Qj = V1 * nx[jx];
#pragma unroll
            for (int jy = 0; jy < 3; ++jy) kr[jx + 3 * jy] += ny[jy] * Pj + dny[jy] * Qj;
          }
        }
      }
      if (c != cc) {
        // the cell is done: into the accumulator slots of the lane's nodes
        if (lane < 27) {
#pragma unroll
          for (int jy = 0; jy < 3; ++jy)
#pragma unroll
            for (int jx = 0; jx < 3; ++jx) {
              const int slot = (jx - kx + 2) + 5 * ((jy - ky + 2) + 5 * (jz - kz + 2));
              acc[slot * 9 + ab] += kr[jx + 3 * jy];
              kr[jx + 3 * jy] = (T)0;
            }
        }
      }
    }
    __syncwarp();
    // store the row: 9 consecutive values per slot plane; blocks coupling to
    // an inactive node (below the activity threshold, not an unknown of the
    // step) are stored as zeros
    for (int t = lane; t < 125 * 9; t += 32) {
      const int slot = t / 9, e = t - 9 * slot;
      const int jx = ix + slot % 5 - 2, jy = iy + (slot / 5) % 5 - 2, jz = iz + slot / 25 - 2;
      const bool live = jx >= 0 && jy >= 0 && jz >= 0 && jx < G.nx1 && jy < G.ny1 && jz < G.nz1 &&
                        node2row[jx + (long long)G.nx1 * (jy + (long long)G.ny1 * jz)] >= 0;
      K.val[((long long)slot * K.cap + row) * 9 + e] = live ? acc[t] : (T)0;
    }
    __syncwarp();
  }
}

template <class T>
cudaError_t launch_assemble_rows3(const DevParticles& P, const DevGrid& G, const int* cstart,
                                  const int* node2row, const T* A, DevMatrix<T> K, int nrow_host,
                                  cudaStream_t st) {
  if (P.np == 0 || nrow_host <= 0) return cudaSuccess;
  constexpr int W = R3Cfg<T>::WARPS;
  const size_t bytes = sizeof(T) * (size_t)R3Smem::PER_WARP * W;
  static_assert(sizeof(T) * R3Smem::PER_WARP * R3Cfg<T>::WARPS <= 227 * 1024, "assembly CTA too large");
  cudaError_t e = cudaFuncSetAttribute(k_assemble_rows3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  // grid-stride warps: at most the CTAs that fit on the device at once
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assemble_rows3<T>, W * 32, bytes);
  if (e != cudaSuccess) return e;
  const long long need = (nrow_host + W - 1) / W;
  const int nblk = (int)std::min<long long>(need, (long long)std::max(1, sms * std::max(1, per_sm)));
  k_assemble_rows3<T><<<nblk, W * 32, bytes, st>>>(P, G, cstart, node2row, A, K, nrow_host);
  return cudaGetLastError();
}

template cudaError_t launch_assemble_rows3<float>(const DevParticles&, const DevGrid&, const int*, const int*,
                                                  const float*, DevMatrix<float>, int, cudaStream_t);
template cudaError_t launch_assemble_rows3<double>(const DevParticles&, const DevGrid&, const int*, const int*,
                                                   const double*, DevMatrix<double>, int, cudaStream_t);

}  // namespace mpm
