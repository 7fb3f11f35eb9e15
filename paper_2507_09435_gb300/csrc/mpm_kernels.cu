// Particle and grid kernels of the implicit-MPM Newton step (sm_103a):
// counting sort by base cell, nodal mass and active set, the fused
// G2P -> constitutive -> P2G residual pass (optionally writing the consistent
// tangent of each particle), the commit pass, the per-cell tangent assembly
// into the stencil-BSR Jacobian, boundary rows/columns, block-Jacobi inverse.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int TPB = 256;
inline int nblocks(long long n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

// ---------------------------------------------------------------- scan
constexpr int SCAN_TPB = 256, SCAN_PER = 4, SCAN_TILE = SCAN_TPB * SCAN_PER;

__global__ void k_scan_tile(const int* __restrict__ in, int* out, int* bsum, int n) {
  __shared__ int wtot[SCAN_TPB / 32];
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
  int v[SCAN_PER];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    int i = base + k;
    v[k] = (i < n) ? in[i] : 0;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wtot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int t = (lane < SCAN_TPB / 32) ? wtot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < SCAN_TPB / 32) wtot[lane] = ti - t;
    if (lane == SCAN_TPB / 32 - 1 && bsum) bsum[blockIdx.x] = ti;
  }
  __syncthreads();
  int run = wtot[w] + incl - s;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    int i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

__global__ void k_scan_add(int* out, const int* __restrict__ bsum, int n) {
  int add = bsum[blockIdx.x];
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    int i = base + k;
    if (i < n) out[i] += add;
  }
}

size_t scan_tmp_ints(int n) {
  size_t tot = 0;
  long long m = n;
  while (m > SCAN_TILE) {
    m = (m + SCAN_TILE - 1) / SCAN_TILE;
    tot += (size_t)m + 32;
  }
  return tot + 32;
}

int scan_launches(long long n) {
  if (n <= 0) return 0;
  long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return nb == 1 ? 1 : 2 + scan_launches(nb);
}

cudaError_t scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    k_scan_tile<<<1, SCAN_TPB, 0, st>>>(in, out, nullptr, n);
    return cudaGetLastError();
  }
  k_scan_tile<<<nb, SCAN_TPB, 0, st>>>(in, out, tmp, n);
  cudaError_t e = scan_exclusive(tmp, tmp, nb, tmp + nb + 32, st);
  if (e != cudaSuccess) return e;
  k_scan_add<<<nb, SCAN_TPB, 0, st>>>(out, tmp, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sorting
// Grid coordinate s = (x - origin)/h and the base node floor(s - 1/2).
__device__ __forceinline__ bool base_node(const DevGrid& G, const DevParticles& P, int p, int D, int b[3]) {
  bool ok = true;
  b[0] = b[1] = b[2] = 0;
  for (int a = 0; a < D; ++a) {
    double s = (P.x[a][p] - G.o[a]) / G.h;
    double fb = floor(s - 0.5);
    ok = ok && (fb >= 0.0) && (fb <= (double)(G.n[a] - 2));
    b[a] = ok ? (int)fb : 0;
  }
  return ok;
}

template <int D>
__global__ void k_cell_keys(DevParticles P, DevGrid G, int* key, int* count, int* rank, int* err) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  int b[3];
  if (!base_node(G, P, p, D, b)) {
    atomicOr(err, ERRF_BOUNDS);
    b[0] = b[1] = b[2] = 0;
  }
  int k = b[0] + G.nx1 * (b[1] + G.ny1 * b[2]);
  key[p] = k;
  rank[p] = atomicAdd(&count[k], 1);
}

template <int D>
cudaError_t launch_cell_keys(const DevParticles& P, const DevGrid& G, int* key, int* count, int* rank,
                             int* err, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_cell_keys<D><<<nblocks(P.np), TPB, 0, st>>>(P, G, key, count, rank, err);
  return cudaGetLastError();
}

__global__ void k_sort_scatter(int np, const int* __restrict__ key, const int* __restrict__ rank,
                               const int* __restrict__ cstart, int* perm) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  perm[cstart[key[p]] + rank[p]] = p;
}
cudaError_t launch_sort_scatter(int np, const int* key, const int* rank, const int* cstart, int* perm,
                                cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  k_sort_scatter<<<nblocks(np), TPB, 0, st>>>(np, key, rank, cstart, perm);
  return cudaGetLastError();
}

__global__ void k_gather(int np, const int* __restrict__ perm, GatherArrays g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int src = perm[i];
  for (int k = 0; k < g.nd; ++k) g.ddst[k][i] = g.dsrc[k][src];
  for (int k = 0; k < g.ni; ++k) g.idst[k][i] = g.isrc[k][src];
}
cudaError_t launch_gather(int np, const int* perm, const GatherArrays& g, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  k_gather<<<nblocks(np), TPB, 0, st>>>(np, perm, g);
  return cudaGetLastError();
}

__global__ void k_flag_positive(const int* __restrict__ c, int* flag, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = c[i] > 0 ? 1 : 0;
}
cudaError_t launch_flag_positive(const int* count, int* flag, long long n, cudaStream_t st) {
  k_flag_positive<<<nblocks(n), TPB, 0, st>>>(count, flag, n);
  return cudaGetLastError();
}
__global__ void k_compact(const int* __restrict__ flag, const int* __restrict__ pos, int* list, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && flag[i]) list[pos[i]] = (int)i;
}
cudaError_t launch_compact(const int* flag, const int* pos, int* list, long long n, cudaStream_t st) {
  k_compact<<<nblocks(n), TPB, 0, st>>>(flag, pos, list, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- active set
template <int D>
__global__ void k_mass(DevParticles P, DevGrid G, double* M) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  Spline1 sp[3];
#pragma unroll
  for (int a = 0; a < D; ++a) sp[a] = spline1((P.x[a][p] - G.o[a]) / G.h);
  if (D == 2) { sp[2].base = 0; sp[2].N[0] = 1.0; }
  // a particle outside the grid interior was flagged by the sort; skip it
  for (int a = 0; a < D; ++a)
    if (sp[a].base < 0 || sp[a].base > G.n[a] - 2) return;
  const double m = P.mass[p];
  const int KZ = (D == 3) ? 3 : 1;
  for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        long long node = (sp[0].base + kx) + (long long)G.nx1 * ((sp[1].base + ky) + (long long)G.ny1 * (sp[2].base + kz));
        atomicAdd(&M[node], sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz] * m);
      }
}
template <int D>
cudaError_t launch_mass(const DevParticles& P, const DevGrid& G, double* M, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_mass<D><<<nblocks(P.np), TPB, 0, st>>>(P, G, M);
  return cudaGetLastError();
}

__global__ void k_active(const double* __restrict__ M, double thr, int* flag, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (M[i] > thr) ? 1 : 0;
}
cudaError_t launch_active(const double* M, double thr, int* flag, long long nnode, cudaStream_t st) {
  k_active<<<nblocks(nnode), TPB, 0, st>>>(M, thr, flag, nnode);
  return cudaGetLastError();
}
__global__ void k_node2row(const int* __restrict__ flag, const int* __restrict__ pos, int* node2row, int* rows,
                           long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) {
    node2row[i] = pos[i];
    rows[pos[i]] = (int)i;
  } else {
    node2row[i] = -1;
  }
}
cudaError_t launch_node2row(const int* flag, const int* pos, int* node2row, int* rows, long long nnode,
                            cudaStream_t st) {
  k_node2row<<<nblocks(nnode), TPB, 0, st>>>(flag, pos, node2row, rows, nnode);
  return cudaGetLastError();
}

__global__ void k_apply_bc(const uint8_t* __restrict__ fixed, const double* __restrict__ bcval,
                           const int* __restrict__ node2row, double* du, long long ndof, int D) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  du[i] = (fixed[i] && node2row[i / D] >= 0) ? bcval[i] : 0.0;
}
cudaError_t launch_apply_bc(const uint8_t* fixed, const double* bcval, const int* node2row, double* du,
                            long long ndof, int D, cudaStream_t st) {
  k_apply_bc<<<nblocks(ndof), TPB, 0, st>>>(fixed, bcval, node2row, du, ndof, D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- particle pass
// One thread per particle (sorted by cell): G2P of du -> dF; constitutive
// update -> P = V0 tau dF^-T; P2G: r_i += P grad w_ip - w_ip m_p g.
// MODE 1 also writes the dim^4 consistent-tangent entries of the particle
// (SoA: A[k*np + p]).  MODE 2 commits the state instead of scattering.
template <int D, class T, int MODE>
__global__ void __launch_bounds__(128) k_particles(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                   const double* __restrict__ du, double* r,
                                                   const double* __restrict__ grav, T* A, int* err,
                                                   int* nplastic) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  bool live = p < P.np;
  int plastic = 0;
  Spline1 sp[3];
  if (live) {
#pragma unroll
    for (int a = 0; a < D; ++a) sp[a] = spline1((P.x[a][p] - G.o[a]) / G.h);
    if (D == 2) { sp[2].base = 0; sp[2].N[0] = 1.0; sp[2].dN[0] = 0.0; }
    bool inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) inside = inside && sp[a].base >= 0 && sp[a].base <= G.n[a] - 2;
    if (!inside) {
      atomicOr(err, ERRF_BOUNDS);
      live = false;
    }
  }
  if (live) {
    const long long nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
    const int KZ = (D == 3) ? 3 : 1;
    PState st;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) st.F[a][c] = (a == c) ? 1.0 : 0.0;
    for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
          double g[3];
          g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
          g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
          g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            double u = du[node * D + a];
#pragma unroll
            for (int c = 0; c < D; ++c) st.F[a][c] += u * g[c];
          }
        }
    // start-of-step elastic left Cauchy-Green
    if (D == 2) {
      st.bn[0][0] = P.be[0][p]; st.bn[1][1] = P.be[1][p]; st.bn[2][2] = P.be[2][p];
      st.bn[0][1] = st.bn[1][0] = P.be[3][p];
      st.bn[0][2] = st.bn[2][0] = st.bn[1][2] = st.bn[2][1] = 0.0;
    } else {
      st.bn[0][0] = P.be[0][p]; st.bn[1][1] = P.be[1][p]; st.bn[2][2] = P.be[2][p];
      st.bn[0][1] = st.bn[1][0] = P.be[3][p];
      st.bn[1][2] = st.bn[2][1] = P.be[4][p];
      st.bn[0][2] = st.bn[2][0] = P.be[5][p];
    }
    const MatC mc = mats[P.mat[p]];
    const double V0 = P.vol0[p];
    int e = constitutive<D>(mc, P.Ep[p], P.phip[p], P.pc[p], V0, st);
    if (e) {
      atomicOr(err, e);
      // record the first failing particle's trial state for the error message
      if (P.fail_rec && atomicCAS((unsigned long long*)P.fail_rec, 0ull,
                                  (unsigned long long)__double_as_longlong(1.0)) == 0ull) {
        P.fail_rec[1] = (double)P.orig[p];
        P.fail_rec[2] = st.lam[0];
        P.fail_rec[3] = st.lam[1];
        P.fail_rec[4] = st.lam[2];
        P.fail_rec[5] = P.Ep[p];
        P.fail_rec[6] = P.phip[p];
        P.fail_rec[7] = P.pc[p];
        P.fail_rec[8] = (double)mc.model;
        P.fail_rec[9] = (double)e;
      }
    } else {
      plastic = st.mode != 0;
      if (MODE == 2) {
        double dx[3] = {0.0, 0.0, 0.0};
        for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
              double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
#pragma unroll
              for (int a = 0; a < D; ++a) dx[a] += w * du[node * D + a];
            }
#pragma unroll
        for (int a = 0; a < D; ++a) P.x[a][p] += dx[a];
        P.be[0][p] = st.benew[0][0]; P.be[1][p] = st.benew[1][1]; P.be[2][p] = st.benew[2][2];
        P.be[3][p] = 0.5 * (st.benew[0][1] + st.benew[1][0]);
        if (D == 3) {
          P.be[4][p] = 0.5 * (st.benew[1][2] + st.benew[2][1]);
          P.be[5][p] = 0.5 * (st.benew[0][2] + st.benew[2][0]);
        }
        P.pc[p] = st.pc;
        double Fo[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) Fo[a][c] = P.F[a * D + c][p];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += st.F[a][k] * Fo[k][c];
            P.F[a * D + c][p] = s;
          }
      } else {
        const double m = P.mass[p];
        double gv[3] = {grav[0], grav[1], grav[2]};
        bool finite = true;
        for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
              double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
              double g[3];
              g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
              g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
              g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
#pragma unroll
              for (int a = 0; a < D; ++a) {
                double f = -w * m * gv[a];
#pragma unroll
                for (int c = 0; c < D; ++c) f += st.P[a][c] * g[c];
                finite = finite && isfinite(f);
                atomicAdd(&r[node * D + a], f);
              }
            }
        if (!finite) atomicOr(err, ERRF_NONFINITE);
        if (MODE == 1) tangent<D, T>(st, V0, A + p, (long long)P.np);
      }
    }
  }
  if (nplastic) {
    unsigned bal = __ballot_sync(0xffffffffu, plastic);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(nplastic, __popc(bal));
  }
}

template <int D, class T>
cudaError_t launch_particles(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* du,
                             double* r, const double* grav, T* A, int mode, int* err, int* nplastic,
                             cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  const int tpb = 128;
  int nb = nblocks(P.np, tpb);
  if (mode == 0) k_particles<D, T, 0><<<nb, tpb, 0, st>>>(P, G, mats, du, r, grav, A, err, nplastic);
  else if (mode == 1) k_particles<D, T, 1><<<nb, tpb, 0, st>>>(P, G, mats, du, r, grav, A, err, nplastic);
  else k_particles<D, T, 2><<<nb, tpb, 0, st>>>(P, G, mats, du, r, grav, A, err, nplastic);
  return cudaGetLastError();
}

// Kirchhoff stress of the committed state, tau = mu (b_e - 1) + lam ln J_e 1,
// written in the caller's particle order.
template <int D>
__global__ void k_stress_out(DevParticles P, const MatC* __restrict__ mats, double* tau9) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  double b[3][3];
  b[0][0] = P.be[0][p]; b[1][1] = P.be[1][p]; b[2][2] = P.be[2][p];
  b[0][1] = b[1][0] = P.be[3][p];
  if (D == 3) { b[1][2] = b[2][1] = P.be[4][p]; b[0][2] = b[2][0] = P.be[5][p]; }
  else { b[1][2] = b[2][1] = b[0][2] = b[2][0] = 0.0; }
  const MatC mc = mats[P.mat[p]];
  Lame L = lame(P.Ep[p], mc.nu);
  double lnJ = 0.5 * log(det3(b));
  int o = P.orig[p];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      tau9[(long long)o * 9 + 3 * i + j] = L.mu * (b[i][j] - (i == j ? 1.0 : 0.0)) + (i == j ? L.lam * lnJ : 0.0);
}
template <int D>
cudaError_t launch_stress_out(const DevParticles& P, const DevGrid& G, const MatC* mats, double* tau9,
                              cudaStream_t st) {
  (void)G;
  if (P.np == 0) return cudaSuccess;
  k_stress_out<D><<<nblocks(P.np), TPB, 0, st>>>(P, mats, tau9);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- assembly
// One CTA per occupied base cell.  Every particle of the cell touches the
// same 3^D nodes, so the cell's contribution is a dense (3^D x 3^D) block
// matrix K_ij[a][b] = sum_p sum_c g_pi[c] T_pj[a c b], with
// T_pj[a c b] = sum_e A_p[a c b e] g_pj[e].  Particles are staged CH at a
// time in shared memory; each thread owns up to PPT node pairs (all D x D
// entries) and adds them to the global matrix once per cell.
template <int D>
__device__ __forceinline__ int slot_of(int dx, int dy, int dz) {
  return (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
}

template <int D, class T, int CH, int PPT>
__global__ void k_assemble(DevParticles P, DevGrid G, const int* __restrict__ cells,
                           const int* __restrict__ cstart, const int* __restrict__ node2row,
                           const T* __restrict__ A, DevMatrix<T> K) {
  constexpr int NN = (D == 2) ? 9 : 27;
  constexpr int D2 = D * D, D3 = D * D * D, D4 = D * D * D * D;
  __shared__ T sg[CH][NN][D];
  __shared__ T sA[CH][D4];
  __shared__ T sT[CH][NN][D3];
  const int cell = cells[blockIdx.x];
  const int p0 = cstart[cell], p1 = cstart[cell + 1];
  const int bx = cell % G.nx1, by = (cell / G.nx1) % G.ny1, bz = cell / (G.nx1 * G.ny1);
  T acc[PPT][D2];
#pragma unroll
  for (int k = 0; k < PPT; ++k)
#pragma unroll
    for (int e = 0; e < D2; ++e) acc[k][e] = (T)0;
  for (int c0 = p0; c0 < p1; c0 += CH) {
    const int nc = min(CH, p1 - c0);
    // stage gradients and tangents
    for (int t = threadIdx.x; t < nc * NN; t += blockDim.x) {
      int q = t / NN, l = t % NN;
      int p = c0 + q;
      int kx = l % 3, ky = (l / 3) % 3, kz = l / 9;
      // B-spline about the cell's base node (the particle's own base node)
      Spline1 a0 = spline1_at((P.x[0][p] - G.o[0]) / G.h, bx);
      Spline1 a1 = spline1_at((P.x[1][p] - G.o[1]) / G.h, by);
      double Nx = a0.N[kx], Ny = a1.N[ky], dNx = a0.dN[kx], dNy = a1.dN[ky];
      double Nz = 1.0, dNz = 0.0;
      if (D == 3) {
        Spline1 a2 = spline1_at((P.x[2][p] - G.o[2]) / G.h, bz);
        Nz = a2.N[kz];
        dNz = a2.dN[kz];
      }
      sg[q][l][0] = (T)(dNx * Ny * Nz * G.ih);
      sg[q][l][1] = (T)(Nx * dNy * Nz * G.ih);
      if (D == 3) sg[q][l][D - 1] = (T)(Nx * Ny * dNz * G.ih);
    }
    for (int t = threadIdx.x; t < nc * D4; t += blockDim.x) {
      int q = t / D4, k = t % D4;
      sA[q][k] = A[(long long)k * P.np + (c0 + q)];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nc * NN * D3; t += blockDim.x) {
      int q = t / (NN * D3), rem = t % (NN * D3);
      int j = rem / D3, acb = rem % D3;
      T s = (T)0;
#pragma unroll
      for (int e = 0; e < D; ++e) s += sA[q][acb * D + e] * sg[q][j][e];
      sT[q][j][acb] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      int pair = threadIdx.x + k * blockDim.x;
      if (pair < NN * NN) {
        int i = pair / NN, j = pair % NN;
        for (int q = 0; q < nc; ++q) {
          T gi[D];
#pragma unroll
          for (int c = 0; c < D; ++c) gi[c] = sg[q][i][c];
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) {
              T s = acc[k][a * D + b];
#pragma unroll
              for (int c = 0; c < D; ++c) s += gi[c] * sT[q][j][(a * D + c) * D + b];
              acc[k][a * D + b] = s;
            }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    int pair = threadIdx.x + k * blockDim.x;
    if (pair < NN * NN) {
      int i = pair / NN, j = pair % NN;
      int ix = i % 3, iy = (i / 3) % 3, iz = i / 9;
      int jx = j % 3, jy = (j / 3) % 3, jz = j / 9;
      long long ni = (bx + ix) + (long long)G.nx1 * ((by + iy) + (long long)G.ny1 * (bz + iz));
      int row = node2row[ni];
      if (row < 0) continue;
      int slot = slot_of<D>(jx - ix, jy - iy, jz - iz);
      T* blk = &K.val[((long long)slot * K.cap + row) * (D * D)];
      if constexpr (D == 2 && sizeof(T) == 4) {
        // one 16-byte vector atomic per 2x2 FP32 block (sm_90+)
        atomicAdd(reinterpret_cast<float4*>(blk), make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]));
      } else {
#pragma unroll
        for (int e = 0; e < D * D; ++e) atomicAdd(&blk[e], acc[k][e]);
      }
    }
  }
}

template <int D, class T>
cudaError_t launch_assemble(const DevParticles& P, const DevGrid& G, const int* cells, int ncell,
                            const int* cstart, const int* node2row, const T* A, DevMatrix<T> K,
                            cudaStream_t st) {
  if (ncell == 0) return cudaSuccess;
  if (D == 2) {
    k_assemble<D, T, 8, 1><<<ncell, 96, 0, st>>>(P, G, cells, cstart, node2row, A, K);
  } else {
    constexpr int CH = sizeof(T) == 4 ? 4 : 2;
    k_assemble<D, T, CH, 3><<<ncell, 256, 0, st>>>(P, G, cells, cstart, node2row, A, K);
  }
  return cudaGetLastError();
}

// Prescribed DOFs: their rows and columns become the identity.
template <int D, class T>
__global__ void k_bc_matrix(DevGrid G, DevMatrix<T> K, const uint8_t* __restrict__ fixed,
                            const int* __restrict__ node2row, int nrow) {
  constexpr int S = (D == 2) ? 25 : 125;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nrow * S) return;
  int row = (int)(t % nrow), slot = (int)(t / nrow);
  int i = K.rows[row];
  int ix = i % G.nx1, iy = (i / G.nx1) % G.ny1, iz = i / (G.nx1 * G.ny1);
  int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
  int jx = ix + dx, jy = iy + dy, jz = iz + dz;
  if (jx < 0 || jy < 0 || jz < 0 || jx >= G.nx1 || jy >= G.ny1 || (D == 3 && jz >= G.nz1)) return;
  long long j = jx + (long long)G.nx1 * (jy + (long long)G.ny1 * jz);
  const bool center = (dx == 0 && dy == 0 && dz == 0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    bool fa = fixed[(long long)i * D + a];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      bool fb = fixed[j * D + b];
      if (fa || fb) {
        T v = (center && a == b && fa) ? (T)1 : (T)0;
        K.val[((long long)slot * K.cap + row) * (D * D) + a * D + b] = v;
      }
    }
  }
}
template <int D, class T>
cudaError_t launch_bc_matrix(const DevGrid& G, DevMatrix<T> K, const uint8_t* fixed, const int* node2row,
                             int nrow_host, cudaStream_t st) {
  constexpr int S = (D == 2) ? 25 : 125;
  if (nrow_host == 0) return cudaSuccess;
  k_bc_matrix<D, T><<<nblocks((long long)nrow_host * S), TPB, 0, st>>>(G, K, fixed, node2row, nrow_host);
  return cudaGetLastError();
}

// Block-Jacobi: inverse of each row's diagonal D x D block (computed in FP64).
template <int D, class T>
__global__ void k_block_jacobi(DevMatrix<T> K, int nrow, int* err) {
  constexpr int C = (D == 2) ? 12 : 62;   // centre slot
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  double a[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) a[i][j] = (double)K.val[((long long)C * K.cap + row) * (D * D) + i * D + j];
  double inv[3][3], det;
  if (!inv3(a, inv, det)) {
    atomicOr(err, ERRF_NONFINITE);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) inv[i][j] = (i == j) ? 1.0 : 0.0;
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) K.dinv[(long long)row * (D * D) + i * D + j] = (T)inv[i][j];
}
template <int D, class T>
cudaError_t launch_block_jacobi(DevMatrix<T> K, int nrow_host, int* err, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  k_block_jacobi<D, T><<<nblocks(nrow_host), TPB, 0, st>>>(K, nrow_host, err);
  return cudaGetLastError();
}

// Structurally present blocks: mask[row*S + slot] = 1 when the neighbour node
// is active and the two nodes share at least one occupied base cell.
template <int D>
__global__ void k_pattern_count(DevGrid G, const int* __restrict__ rows, int nrow,
                                const int* __restrict__ node2row, const int* __restrict__ count,
                                int* mask) {
  constexpr int S = (D == 2) ? 25 : 125;
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  int i = rows[row];
  int ix = i % G.nx1, iy = (i / G.nx1) % G.ny1, iz = i / (G.nx1 * G.ny1);
  for (int slot = 0; slot < S; ++slot) {
    int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
    int j3[3] = {ix + dx, iy + dy, iz + dz};
    int i3[3] = {ix, iy, iz};
    bool inside = j3[0] >= 0 && j3[1] >= 0 && j3[0] < G.nx1 && j3[1] < G.ny1 &&
                  (D == 2 || (j3[2] >= 0 && j3[2] < G.nz1));
    if (!inside) continue;
    long long j = j3[0] + (long long)G.nx1 * (j3[1] + (long long)G.ny1 * j3[2]);
    if (node2row[j] < 0) continue;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < D) {
        lo[a] = max(max(i3[a], j3[a]) - 2, 0);
        hi[a] = min(min(i3[a], j3[a]), G.n[a] - 2);
      } else { lo[a] = 0; hi[a] = 0; }
    }
    bool hit = false;
    for (int cz = lo[2]; cz <= hi[2] && !hit; ++cz)
      for (int cy = lo[1]; cy <= hi[1] && !hit; ++cy)
        for (int cx = lo[0]; cx <= hi[0] && !hit; ++cx)
          hit = count[cx + (long long)G.nx1 * (cy + (long long)G.ny1 * cz)] > 0;
    if (hit) mask[(long long)row * S + slot] = 1;
  }
}
template <int D>
cudaError_t launch_pattern_count(const DevGrid& G, const int* rows, int nrow_host, const int* node2row,
                                 const int* count, int* mask, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  k_pattern_count<D><<<nblocks(nrow_host), TPB, 0, st>>>(G, rows, nrow_host, node2row, count, mask);
  return cudaGetLastError();
}

// ||r||^2 over free DOFs of active rows.
template <int D>
__global__ void k_norm_free(const double* __restrict__ r, const int* __restrict__ rows, int nrow,
                            const uint8_t* __restrict__ fixed, double* out) {
  __shared__ double ws[TPB / 32];
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (row < nrow) {
    long long i = rows[row];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double v = r[i * D + a];
      if (!fixed[i * D + a]) s += v * v;
    }
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < TPB / 32) ? ws[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}
template <int D>
cudaError_t launch_norm_free(const double* r, const int* rows, int nrow_host, const uint8_t* fixed,
                             double* out, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  k_norm_free<D><<<nblocks(nrow_host), TPB, 0, st>>>(r, rows, nrow_host, fixed, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- instantiations
#define MPM_INST_D(D)                                                                                   \
  template cudaError_t launch_cell_keys<D>(const DevParticles&, const DevGrid&, int*, int*, int*, int*,  \
                                           cudaStream_t);                                                \
  template cudaError_t launch_mass<D>(const DevParticles&, const DevGrid&, double*, cudaStream_t);      \
  template cudaError_t launch_stress_out<D>(const DevParticles&, const DevGrid&, const MatC*, double*,   \
                                            cudaStream_t);                                               \
  template cudaError_t launch_pattern_count<D>(const DevGrid&, const int*, int, const int*, const int*,  \
                                               int*, cudaStream_t);                                      \
  template cudaError_t launch_norm_free<D>(const double*, const int*, int, const uint8_t*, double*,      \
                                           cudaStream_t);
MPM_INST_D(2)
MPM_INST_D(3)

#define MPM_INST_DT(D, T)                                                                               \
  template cudaError_t launch_particles<D, T>(const DevParticles&, const DevGrid&, const MatC*,          \
                                              const double*, double*, const double*, T*, int, int*,      \
                                              int*, cudaStream_t);                                       \
  template cudaError_t launch_assemble<D, T>(const DevParticles&, const DevGrid&, const int*, int,       \
                                             const int*, const int*, const T*, DevMatrix<T>,             \
                                             cudaStream_t);                                              \
  template cudaError_t launch_bc_matrix<D, T>(const DevGrid&, DevMatrix<T>, const uint8_t*, const int*,  \
                                              int, cudaStream_t);                                        \
  template cudaError_t launch_block_jacobi<D, T>(DevMatrix<T>, int, int*, cudaStream_t);
MPM_INST_DT(2, float)
MPM_INST_DT(2, double)
MPM_INST_DT(3, float)
MPM_INST_DT(3, double)

}  // namespace mpm
