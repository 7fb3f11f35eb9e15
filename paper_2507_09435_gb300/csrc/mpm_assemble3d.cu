// Assembly of the 3D single-phase Jacobian (a4): one warp per active node row.
//
// Row i of J holds the 125 blocks K_ij = sum_p G_ip^T A_p G_jp over the
// particles whose 27-node B-spline stencil contains i, where A_p[a][c][b][e] =
// dP_p[a][c] / d dF_p[b][e] is the particle's consistent tangent (written by
// the residual pass) and G_ip[c] the gradient of w_ip.  Those particles sit
// in the 27 cells (base nodes) i - (kx, ky, kz), k in {0,1,2}^3; in cell
// i - k, node i is node k of every particle's stencil and node j of the
// stencil (lane j) lands in slot (j - k + 2) of row i.
//
// Owner computes, with no atomics and no block-wide barrier in the loop:
// each warp owns one row, keeps its 125 x 9 accumulator in warp-private
// shared memory, and walks its 27 cells in batches of QB particles:
//   1. the batch's tangents are copied to shared memory (coalesced over
//      particles: A is stored entry-major, A[k * np + p]; the loads of the
//      next batch are issued into registers before the current batch is
//      processed, so their latency overlaps the arithmetic) and each
//      particle's per-axis B-spline weights and derivatives are evaluated
//      (FP64 offset from the base node, then the working type T);
//   2. lanes 0..26 form U_p[a][b][e] = sum_c G_ip[c] A_p[a][c][b][e];
//   3. lane j adds sum_e U_p[a][b][e] G_jp[e] for its stencil node j into
//      nine registers; after the cell, into the accumulator slot of j.
// The CTA's W warps own W consecutive rows (mostly x-neighbours, which share
// two thirds of their particles through L1) and store their rows slot-major
// at the end: W x 9 consecutive values per slot plane.
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
struct R3Smem {
  static constexpr int SU = 0;                       // [QB][28] U of each particle
  static constexpr int GI = SU + R3_QB * 28;         // [QB][4]  G_ip of each particle
  static constexpr int SW = GI + R3_QB * 4;          // [QB][3][8] N0..2, dN0..2 / h per axis
  static constexpr int SA = SW + R3_QB * 3 * 8;      // [QB][81] tangents
  static constexpr int ACC = SA + R3_QB * 81;        // [125][9] the row's blocks
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
}  // namespace

template <class T>
__global__ void __launch_bounds__(R3Cfg<T>::WARPS * 32, 3)
    k_assemble_rows3(DevParticles P, DevGrid G, const int* __restrict__ cstart, const T* __restrict__ A,
                     DevMatrix<T> K, int nrow) {
  constexpr int W = R3Cfg<T>::WARPS;
  using L = R3Smem;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* wbase = sm + warp * L::PER_WARP;
  T* sU = wbase + L::SU;
  T* sGi = wbase + L::GI;
  T* sW = wbase + L::SW;
  T* sA = wbase + L::SA;
  T* acc = wbase + L::ACC;
  const int row0 = blockIdx.x * W;
  const int row = row0 + warp;
  for (int t = lane; t < 125 * 9; t += 32) acc[t] = (T)0;
  if (row < nrow) {
    const long long i = K.rows[row];
    const long long plane = (long long)G.nx1 * G.ny1;
    const int ix = (int)(i % G.nx1), iy = (int)((i / G.nx1) % G.ny1), iz = (int)(i / plane);
    // lane j < 27: its node (jx, jy, jz) of a particle's stencil, and its
    // entry (a, b, e) of U with the tangent offset a*27 + b*3 + e
    const int jx = lane % 3, jy = (lane / 3) % 3, jz = lane / 9;
    const int uo = (lane / 9) * 27 + (lane % 9);
    const T ih = (T)G.ih;
    // lane c < 27 looks up the particle range of cell c = i - (kx, ky, kz),
    // (kx, ky, kz) = (c % 3, c / 3 % 3, c / 9); the warp walks the 27 cells
    // in that order, reading the ranges by shuffles
    int my_pb = 0, my_pe = 0;
    if (lane < 27) {
      const int cx = ix - jx, cy = iy - jy, cz = iz - jz;
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
    seek(0);
    constexpr int NPF = (81 + 32 / R3_QB - 1) / (32 / R3_QB);   // tangent loads per lane per batch
    const int lq = lane & (R3_QB - 1), lk = lane / R3_QB;
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
    if (c < 27) prefetch(q0, min(R3_QB, pe - q0));
    T kr[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) kr[ab] = (T)0;
    while (c < 27) {
      const int cc = c, nq = min(R3_QB, pe - q0);
      __syncwarp();   // the previous batch's readers are done
#pragma unroll
      for (int m = 0; m < NPF; ++m) {
        const int k = lk + (32 / R3_QB) * m;
        if (lq < nq && k < 81) sA[lq * 81 + k] = pf[m];
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
        T* w = sW + (q * 3 + a) * 8;
        w[0] = (T)0.5 * u * u;
        w[1] = (T)0.75 - cm * cm;
        w[2] = (T)0.5 * t * t;
        w[3] = -u * ih;
        w[4] = (T)-2 * cm * ih;
        w[5] = t * ih;
      }
      __syncwarp();
      if (lane < nq) {
        const T* w = sW + lane * 24;
        T* g = sGi + lane * 4;
        g[0] = w[3 + kx] * w[8 + ky] * w[16 + kz];
        g[1] = w[kx] * w[11 + ky] * w[16 + kz];
        g[2] = w[kx] * w[8 + ky] * w[19 + kz];
        g[3] = (T)0;
      }
      __syncwarp();
      if (lane < 27) {
        for (int q = 0; q < nq; ++q) {
          T gi[4];
          lds4v(sGi + q * 4, gi);
          const T* aq = sA + q * 81 + uo;
          sU[q * 28 + lane] = gi[0] * aq[0] + gi[1] * aq[9] + gi[2] * aq[18];
        }
      }
      __syncwarp();
      if (lane < 27) {
        for (int q = 0; q < nq; ++q) {
          const T* w = sW + q * 24;
          const T nx = w[jx], dnx = w[3 + jx], ny = w[8 + jy], dny = w[11 + jy];
          const T nz = w[16 + jz], dnz = w[19 + jz];
          const T g0 = dnx * ny * nz, g1 = nx * dny * nz, g2 = nx * ny * dnz;
          T u[28];
#pragma unroll
          for (int v = 0; v < 7; ++v) lds4v(sU + q * 28 + 4 * v, u + 4 * v);
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) kr[ab] += u[ab * 3] * g0 + u[ab * 3 + 1] * g1 + u[ab * 3 + 2] * g2;
        }
      }
      if (c != cc) {
        // the cell is done: into the accumulator slot of each lane's node
        if (lane < 27) {
          const int slot = (jx - kx + 2) + 5 * ((jy - ky + 2) + 5 * (jz - kz + 2));
#pragma unroll
          for (int ab = 0; ab < 9; ++ab) {
            acc[slot * 9 + ab] += kr[ab];
            kr[ab] = (T)0;
          }
        }
      }
    }
  }
  __syncthreads();
  // the CTA's rows, slot-major: nr * 9 consecutive values per slot plane
  const int nr = min(W, nrow - row0);
  if (nr <= 0) return;
  const int per_slot = nr * 9;
  for (int t = threadIdx.x; t < 125 * per_slot; t += W * 32) {
    const int slot = t / per_slot, rem = t - slot * per_slot;
    const int w = rem / 9, ab = rem - 9 * w;
    K.val[((long long)slot * K.cap + row0) * 9 + rem] = sm[w * L::PER_WARP + L::ACC + slot * 9 + ab];
  }
}

template <class T>
cudaError_t launch_assemble_rows3(const DevParticles& P, const DevGrid& G, const int* cstart, const T* A,
                                  DevMatrix<T> K, int nrow_host, cudaStream_t st) {
  if (P.np == 0 || nrow_host <= 0) return cudaSuccess;
  constexpr int W = R3Cfg<T>::WARPS;
  const size_t bytes = sizeof(T) * (size_t)R3Smem::PER_WARP * W;
  static_assert(sizeof(T) * R3Smem::PER_WARP * R3Cfg<T>::WARPS <= 227 * 1024, "assembly CTA too large");
  cudaError_t e = cudaFuncSetAttribute(k_assemble_rows3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  const int nblk = (nrow_host + W - 1) / W;
  k_assemble_rows3<T><<<nblk, W * 32, bytes, st>>>(P, G, cstart, A, K, nrow_host);
  return cudaGetLastError();
}

template cudaError_t launch_assemble_rows3<float>(const DevParticles&, const DevGrid&, const int*, const float*,
                                                  DevMatrix<float>, int, cudaStream_t);
template cudaError_t launch_assemble_rows3<double>(const DevParticles&, const DevGrid&, const int*,
                                                   const double*, DevMatrix<double>, int, cudaStream_t);

}  // namespace mpm
