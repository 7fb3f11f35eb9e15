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
// Nodal mass contributions w_ip m_p of each particle, fp[k*np + p] for node k
// = kx + 3 ky + 9 kz of its stencil (zeros for a particle outside the grid
// interior, which the sort flagged), added per node by k_gather_residual in
// a fixed order.
template <int D>
__global__ void k_mass(DevParticles P, DevGrid G, double* fp) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  Spline1 sp[3];
#pragma unroll
  for (int a = 0; a < D; ++a) sp[a] = spline1((P.x[a][p] - G.o[a]) / G.h);
  if (D == 2) {
    sp[2].base = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) sp[2].N[k] = (k == 0) ? 1.0 : 0.0;
  }
  bool inside = true;
  for (int a = 0; a < D; ++a) inside = inside && sp[a].base >= 0 && sp[a].base <= G.n[a] - 2;
  const double m = inside ? P.mass[p] : 0.0;
  const int KZ = (D == 3) ? 3 : 1;
  for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
        fp[(long long)(kx + 3 * (ky + 3 * kz)) * P.np + p] = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz] * m;
}
template <int D>
cudaError_t launch_mass(const DevParticles& P, const DevGrid& G, const int* cstart, double* fp, double* M,
                        long long nnode, cudaStream_t st) {
  if (P.np == 0) return cudaMemsetAsync(M, 0, nnode * sizeof(double), st);
  k_mass<D><<<nblocks(P.np), TPB, 0, st>>>(P, G, fp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gather_residual<D, 1>(G, cstart, fp, P.np, M, nnode, st);
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
// update -> P = V0 tau dF^-T; the particle's contributions to the residual,
// P grad w_ip - w_ip m_p g for the 3^dim nodes i of its stencil, stored as
// fp[(k*D + a)*np + p] (k = kx + 3 ky + 9 kz; zeros for a particle that
// contributes nothing), which k_gather_residual adds per node in a fixed
// order.  MODE 1 also writes the dim^4 consistent-tangent entries of the
// particle (SoA: A[k*np + p]).  MODE 2 commits the state instead.
template <int D, class T, int MODE>
__global__ void __launch_bounds__(128) k_particles(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                   const double* __restrict__ du, double* fp,
                                                   const double* __restrict__ grav, T* A, int* err,
                                                   int* nplastic) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  bool live = p < P.np;
  bool wrote = false;
  int plastic = 0;
  Spline1 sp[3];
  if (live) {
#pragma unroll
    for (int a = 0; a < D; ++a) sp[a] = spline1((P.x[a][p] - G.o[a]) / G.h);
    if (D == 2) {
      sp[2].base = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sp[2].N[k] = (k == 0) ? 1.0 : 0.0;
        sp[2].dN[k] = 0.0;
      }
    }
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
    // B-spline factors with 1/h folded into the derivatives, and the weight
    // gradient of node (kx, ky, kz) in product form: grad w = (dNx Ny Nz,
    // Nx dNy Nz, Nx Ny dNz), the y-z products formed once per (ky, kz)
    double dh[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) dh[a][k] = sp[a].dN[k] * G.ih;
    for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const double nyz = sp[1].N[ky] * sp[2].N[kz], dyz = dh[1][ky] * sp[2].N[kz], ydz = sp[1].N[ky] * dh[2][kz];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
          const double g[3] = {dh[0][kx] * nyz, sp[0].N[kx] * dyz, sp[0].N[kx] * ydz};
#pragma unroll
          for (int a = 0; a < D; ++a) {
            double u = du[node * D + a];
#pragma unroll
            for (int c = 0; c < D; ++c) st.F[a][c] += u * g[c];
          }
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
        // body force per particle: gravity plus any carried external force
        double gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a] = m * grav[a] + (P.fext[a] ? P.fext[a][p] : 0.0);
        bool finite = true;
        for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky) {
            const double nyz = sp[1].N[ky] * sp[2].N[kz], dyz = dh[1][ky] * sp[2].N[kz],
                         ydz = sp[1].N[ky] * dh[2][kz];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const double w = sp[0].N[kx] * nyz;
              const double g[3] = {dh[0][kx] * nyz, sp[0].N[kx] * dyz, sp[0].N[kx] * ydz};
              const int kk = kx + 3 * (ky + 3 * kz);
#pragma unroll
              for (int a = 0; a < D; ++a) {
                double f = -w * gv[a];
#pragma unroll
                for (int c = 0; c < D; ++c) f += st.P[a][c] * g[c];
                finite = finite && isfinite(f);
                fp[((long long)kk * D + a) * P.np + p] = f;
              }
            }
          }
        wrote = true;
        if (!finite) atomicOr(err, ERRF_NONFINITE);
        if (MODE == 1) tangent<D, T>(st, V0, A + p, (long long)P.np);
      }
    }
  }
  if (MODE != 2 && p < P.np && !wrote) {
    constexpr int NS = (D == 3) ? 27 : 9;
    for (int k = 0; k < NS * D; ++k) fp[(long long)k * P.np + p] = 0.0;
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
// Owner-computes assembly, K_ij[a][b] = sum_p sum_c,e g_pi[c] A_p[a c b e] g_pj[e]
// (the Jacobian of Sec. 3 written with the consistent tangent A_p).  One CTA
// owns a tile of TX x TY x TZ grid nodes and computes every block of the rows
// of those nodes, reading the particles of the surrounding cells (the cells
// with base node in [tile - 2, tile end) per axis) in chunks through shared
// memory.  Blocks accumulate in shared memory and are stored once, so the
// matrix needs no zero fill and no global atomics.  For a row node i and a
// cell c whose 3^D nodes contain i, the row-side contraction
// U_pi[a b e] = sum_c g_pi[c] A_p[a c b e] is shared by the 3^D nodes j of c.
template <int D>
__device__ __forceinline__ int slot_of(int dx, int dy, int dz) {
  return (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
}

// Tile and chunk sizes per (dim, precision, values per node).
template <int D, class T, int B>
struct AsmCfg;
template <> struct AsmCfg<2, float, 2>  { static constexpr int TX = 16, TY = 8, TZ = 1, CHP = 64; };
template <> struct AsmCfg<2, double, 2> { static constexpr int TX = 8,  TY = 8, TZ = 1, CHP = 64; };
template <> struct AsmCfg<2, float, 3>  { static constexpr int TX = 8,  TY = 8, TZ = 1, CHP = 64; };
template <> struct AsmCfg<2, double, 3> { static constexpr int TX = 8,  TY = 4, TZ = 1, CHP = 32; };
constexpr int ASM_TPB = 256;
constexpr int ASM_UB = 8;   // particles per U batch of a 3D task

// Shared-memory layout of one assembly CTA.  A particle's tangent has
// (B * NPHI)^2 entries A[a][c][b][e] (a, b < B values per node; c, e < NPHI
// shape-function components: the D gradient entries, and for u-p the weight).
template <int D, class T, int B>
struct AsmSmem {
  static constexpr int TX = AsmCfg<D, T, B>::TX, TY = AsmCfg<D, T, B>::TY, TZ = AsmCfg<D, T, B>::TZ;
  static constexpr int CHP = AsmCfg<D, T, B>::CHP;
  static constexpr int NN = (D == 2) ? 9 : 27, S = (D == 2) ? 25 : 125;
  static constexpr int NPHI = (B > D) ? D + 1 : D;
  static constexpr int D2 = B * B, D4 = B * NPHI * B * NPHI, NT = TX * TY * TZ;
  static constexpr int AST = (D == 2) ? (D4 + 3) / 4 * 4 : D4;   // row stride of the staged tangents
  // byte offsets (all multiples of 16)
  static constexpr size_t acc = 0;
  static constexpr size_t sA = acc + sizeof(T) * NT * S * D2;
  static constexpr size_t sG = sA + ((sizeof(T) * CHP * AST + 15) / 16) * 16;
  static constexpr size_t sU = sG + sizeof(T) * CHP * NN * 4;
  static constexpr size_t sW = sU + sizeof(T) * (ASM_TPB / 32) * ASM_UB * 28;
  static constexpr size_t srow = sW + ((sizeof(T) * CHP * 3 * 6 + 15) / 16) * 16;
  static constexpr size_t bytes = srow + sizeof(int) * ((NT + 3) / 4) * 4;
};

template <class T>
__device__ __forceinline__ void lds4(const T* p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
  } else {
    const double2 u = reinterpret_cast<const double2*>(p)[0];
    const double2 w = reinterpret_cast<const double2*>(p)[1];
    v[0] = u.x; v[1] = u.y; v[2] = w.x; v[3] = w.y;
  }
}

template <int D, class T, int B>
__global__ void __launch_bounds__(ASM_TPB) k_assemble(DevParticles P, DevGrid G, const int* __restrict__ cstart,
                                                      const int* __restrict__ node2row, const T* __restrict__ A,
                                                      DevMatrix<T> K, int ntx, int nty) {
  using L = AsmSmem<D, T, B>;
  constexpr int TX = L::TX, TY = L::TY, TZ = L::TZ, CHP = L::CHP, NN = L::NN, S = L::S;
  constexpr int D2 = L::D2, D4 = L::D4, NT = L::NT, AST = L::AST, NPHI = L::NPHI;
  static_assert(D == 2, "3D rows are assembled by launch_assemble_cells3");
  extern __shared__ __align__(16) unsigned char smem[];
  T* acc = reinterpret_cast<T*>(smem + L::acc);    // [NT][S][D2]
  T* sA = reinterpret_cast<T*>(smem + L::sA);      // [CHP][AST]
  T* sG = reinterpret_cast<T*>(smem + L::sG);      // [CHP][NN][4]
  T* sU = reinterpret_cast<T*>(smem + L::sU);      // [warps][ASM_UB][28]
  T* sW = reinterpret_cast<T*>(smem + L::sW);      // [CHP][3 axes][N0..2, dN0..2]
  int* srow = reinterpret_cast<int*>(smem + L::srow);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx0 = (blockIdx.x % ntx) * TX;
  const int ty0 = ((blockIdx.x / ntx) % nty) * TY;
  const int tz0 = (blockIdx.x / (ntx * nty)) * TZ;
  // rows of the tile
  int mine = 0;
  for (int l = tid; l < NT; l += ASM_TPB) {
    const int ix = tx0 + l % TX, iy = ty0 + (l / TX) % TY, iz = tz0 + l / (TX * TY);
    int row = -1;
    if (ix < G.nx1 && iy < G.ny1 && iz < G.nz1)
      row = node2row[ix + (long long)G.nx1 * (iy + (long long)G.ny1 * iz)];
    srow[l] = row;
    mine |= (row >= 0);
  }
  if (!__syncthreads_or(mine)) return;
  for (int t = tid; t < NT * S * D2; t += ASM_TPB) acc[t] = (T)0;

  const int cx_lo = max(tx0 - 2, 0), cx_hi = min(tx0 + TX - 1, G.nx1 - 1);
  const int cy_lo = max(ty0 - 2, 0), cy_hi = min(ty0 + TY - 1, G.ny1 - 1);
  const int cz_lo = (D == 3) ? max(tz0 - 2, 0) : 0, cz_hi = (D == 3) ? min(tz0 + TZ - 1, G.nz1 - 1) : 0;
  for (int cz = cz_lo; cz <= cz_hi; ++cz)
    for (int cy = cy_lo; cy <= cy_hi; ++cy) {
      // one run of cells along x: their particles are contiguous
      const long long crow = (long long)G.nx1 * (cy + (long long)G.ny1 * cz);
      const int pb = cstart[crow + cx_lo], pe = cstart[crow + cx_hi + 1];
      // tile nodes inside the 3^D nodes of the run's cells along y and z
      const int iy_lo = max(cy, ty0), iy_hi = min(min(cy + 2, ty0 + TY - 1), G.ny1 - 1);
      const int iz_lo = (D == 3) ? max(cz, tz0) : 0;
      const int iz_hi = (D == 3) ? min(min(cz + 2, tz0 + TZ - 1), G.nz1 - 1) : 0;
      const int ny_ov = iy_hi - iy_lo + 1, nz_ov = iz_hi - iz_lo + 1;
      if (ny_ov <= 0 || nz_ov <= 0) continue;
      for (int q0 = pb; q0 < pe; q0 += CHP) {
        const int nq = min(CHP, pe - q0);
        __syncthreads();   // previous chunk's readers are done
        // tangents, k-major global reads -> [q][k] in shared memory
        for (int k = warp; k < D4; k += ASM_TPB / 32)
          for (int q = lane; q < nq; q += 32) sA[q * AST + k] = A[(long long)k * P.np + q0 + q];
        // per particle and axis: the three B-spline weights and derivatives
        // about the particle's base node (its cell's x from the run's cell
        // starts, y and z those of the run); FP64 offset, then type T
        for (int t = tid; t < nq; t += ASM_TPB) {
          const int p = q0 + t;
          int cx = cx_lo;
          while (cx < cx_hi && cstart[crow + cx + 1] <= p) ++cx;
          const int base[3] = {cx, cy, cz};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            T* w = sW + (t * 3 + a) * 6;
            if (a < D) {
              const T tt = (T)((P.x[a][p] - G.o[a]) * G.ih - (double)base[a] - 0.5);
              // quadratic B-spline of Sec. 2 at nodes base, base + 1, base + 2
              const T u = (T)1 - tt, c = tt - (T)0.5;
              w[0] = (T)0.5 * u * u;  w[3] = -u;
              w[1] = (T)0.75 - c * c; w[4] = (T)-2 * c;
              w[2] = (T)0.5 * tt * tt; w[5] = tt;
            } else {
              w[0] = (T)1; w[1] = w[2] = (T)0;
              w[3] = w[4] = w[5] = (T)0;
            }
          }
        }
        __syncthreads();
        // gradients of the 3^D nodes of each particle's base cell
        for (int t = tid; t < nq * NN; t += ASM_TPB) {
          const int q = t / NN, l = t - q * NN;
          const int kx = l % 3, ky = (l / 3) % 3, kz = l / 9;
          const T* wx = sW + (q * 3 + 0) * 6;
          const T* wy = sW + (q * 3 + 1) * 6;
          const T* wz = sW + (q * 3 + 2) * 6;
          const T ih = (T)G.ih;
          T* g = sG + (q * NN + l) * 4;
          g[0] = wx[3 + kx] * wy[ky] * wz[kz] * ih;
          g[1] = wx[kx] * wy[3 + ky] * wz[kz] * ih;
          // gradient entries, then (u-p) the weight in entry D
          g[2] = (D == 3) ? wx[kx] * wy[ky] * wz[3 + kz] * ih : ((NPHI > D) ? wx[kx] * wy[ky] : (T)0);
          g[3] = (D == 3 && NPHI > D) ? wx[kx] * wy[ky] * wz[kz] : (T)0;
        }
        __syncthreads();
        // tasks: tile nodes i with y/z overlap, one warp each, taking the x
        // offsets kx of i in the cells in a fixed order (the warp alone adds
        // into i's blocks: no atomics, the same sums for any warp order)
        const int ntask = TX * ny_ov * nz_ov;
        for (int task = warp; task < ntask; task += ASM_TPB / 32)
        for (int kx = 0; kx < 3; ++kx) {
          const int ixl = task % TX;
          const int iyl = (task / TX) % ny_ov;
          const int izl = task / (TX * ny_ov);
          const int ix = tx0 + ixl, iy = iy_lo + iyl, iz = iz_lo + izl;
          const int cx = ix - kx;
          if (cx < cx_lo || cx > cx_hi) continue;
          const int l_i = ixl + TX * ((iy - ty0) + TY * (iz - tz0));
          if (srow[l_i] < 0) continue;
          const int qa = max(cstart[crow + cx], q0) - q0;
          const int qb = min(cstart[crow + cx + 1], q0 + nq) - q0;
          if (qa >= qb) continue;
          const int ky = iy - cy, kz = (D == 3) ? iz - cz : 0;
          const int il = kx + 3 * ky + 9 * kz;   // i among the cell's nodes
          T* arow = acc + (size_t)l_i * S * D2;
          // lane = j + 9 * sub: node j of the cell, particles sub, sub+3, ...
          const int j = lane % 9, sub = lane / 9;
          T kb[D2];
#pragma unroll
          for (int e = 0; e < D2; ++e) kb[e] = (T)0;
          if (lane < 27) {
            for (int q = qa + sub; q < qb; q += 3) {
              T gi[4], gj[4], aq[AST];
              lds4(sG + (q * NN + il) * 4, gi);
              lds4(sG + (q * NN + j) * 4, gj);
#pragma unroll
              for (int v = 0; v < AST / 4; ++v) lds4(sA + q * AST + 4 * v, aq + 4 * v);
#pragma unroll
              for (int a = 0; a < B; ++a)
#pragma unroll
                for (int b = 0; b < B; ++b) {
                  T s = (T)0;
#pragma unroll
                  for (int c = 0; c < NPHI; ++c)
#pragma unroll
                    for (int e = 0; e < NPHI; ++e) s += gi[c] * aq[((a * NPHI + c) * B + b) * NPHI + e] * gj[e];
                  kb[a * B + b] += s;
                }
            }
          }
#pragma unroll
          for (int e = 0; e < D2; ++e) {
            // lanes j, j + 9, j + 18 hold the three particle subsets of node j
            const T v9 = __shfl_sync(0xffffffffu, kb[e], (lane + 9) & 31);
            const T v18 = __shfl_sync(0xffffffffu, kb[e], (lane + 18) & 31);
            kb[e] += v9 + v18;
          }
          if (lane < 9) {
            const int jx = j % 3, jy = j / 3;
            T* blk = arow + slot_of<2>(jx - kx, jy - ky, 0) * D2;
#pragma unroll
            for (int e = 0; e < D2; ++e) blk[e] += kb[e];
          }
          __syncwarp();
        }
      }
    }
  __syncthreads();
  // store the tile's rows: all S slots, slot-major so that the rows of one
  // x-line of nodes land contiguously in each slot plane; blocks coupling to
  // an inactive node (below the activity threshold, not an unknown of the
  // step) are stored as zeros
  for (int t = tid; t < NT * S * D2; t += ASM_TPB) {
    const int ab = t % D2, l = (t / D2) % NT, slot = t / (D2 * NT);
    const int row = srow[l];
    if (row < 0) continue;
    const int jx = tx0 + l % TX + slot % 5 - 2, jy = ty0 + (l / TX) % TY + slot / 5 - 2;
    const bool live = jx >= 0 && jy >= 0 && jx < G.nx1 && jy < G.ny1 &&
                      node2row[jx + (long long)G.nx1 * jy] >= 0;
    K.val[((long long)slot * K.cap + row) * D2 + ab] = live ? acc[((size_t)l * S + slot) * D2 + ab] : (T)0;
  }
}

template <int D, class T, int B>
cudaError_t launch_assemble(const DevParticles& P, const DevGrid& G, const int* cstart, const int* node2row,
                            const T* A, DevMatrix<T> K, int nrow_host, const Asm3<T>* a3, cudaStream_t st) {
  if constexpr (D == 3) {
    static_assert(B == 3, "3D assembly is written for the single-phase blocks");
    if (!a3) return cudaErrorInvalidValue;
    return launch_assemble_cells3<T>(P, G, *a3, cstart, node2row, A, K, nrow_host, st);
  } else {
  using L = AsmSmem<D, T, B>;
  if (P.np == 0) return cudaSuccess;
  static_assert(L::bytes <= 227 * 1024, "assembly tile exceeds shared memory");
  cudaError_t e = cudaFuncSetAttribute(k_assemble<D, T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::bytes);
  if (e != cudaSuccess) return e;
  const int ntx = (G.nx1 + L::TX - 1) / L::TX, nty = (G.ny1 + L::TY - 1) / L::TY;
  const int ntz = (G.nz1 + L::TZ - 1) / L::TZ;
  const long long nt = (long long)ntx * nty * ntz;
  if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_assemble<D, T, B><<<(unsigned)nt, ASM_TPB, L::bytes, st>>>(P, G, cstart, node2row, A, K, ntx, nty);
  return cudaGetLastError();
  }
}

// Prescribed DOFs: their rows and columns become the identity.
template <int D, class T, int B>
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
  for (int a = 0; a < B; ++a) {
    bool fa = fixed[(long long)i * B + a];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      bool fb = fixed[j * B + b];
      if (fa || fb) {
        T v = (center && a == b && fa) ? (T)1 : (T)0;
        K.val[((long long)slot * K.cap + row) * (B * B) + a * B + b] = v;
      }
    }
  }
}
template <int D, class T, int B>
cudaError_t launch_bc_matrix(const DevGrid& G, DevMatrix<T> K, const uint8_t* fixed, const int* node2row,
                             int nrow_host, cudaStream_t st) {
  constexpr int S = (D == 2) ? 25 : 125;
  if (nrow_host == 0) return cudaSuccess;
  k_bc_matrix<D, T, B><<<nblocks((long long)nrow_host * S), TPB, 0, st>>>(G, K, fixed, node2row, nrow_host);
  return cudaGetLastError();
}

// Block-Jacobi: inverse of each row's diagonal B x B block (computed in FP64).
template <int D, class T, int B>
__global__ void k_block_jacobi(DevMatrix<T> K, int nrow, int* err) {
  static_assert(B <= 3, "block inverse written for B <= 3");
  constexpr int C = (D == 2) ? 12 : 62;   // centre slot
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  double a[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) a[i][j] = (double)K.val[((long long)C * K.cap + row) * (B * B) + i * B + j];
  double inv[3][3], det;
  if (!inv3(a, inv, det)) {
    atomicOr(err, ERRF_NONFINITE);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) inv[i][j] = (i == j) ? 1.0 : 0.0;
  }
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) K.dinv[(long long)row * (B * B) + i * B + j] = (T)inv[i][j];
}
// Row-segment block-Jacobi: the inverse of the 4B x 4B diagonal block of the
// rows 4s..4s+3 (consecutive active nodes, mostly neighbours along x), by
// Gauss-Jordan elimination with partial pivoting in FP64.  Rows past the last
// active row are identity.  One thread per segment.
template <int D, class T, int B>
__global__ void k_segment_inverse(DevGrid G, DevMatrix<T> K, int nrow, int* err) {
  constexpr int W = 4 * B;
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg * 4 >= nrow) return;
  double a[W][2 * W];
#pragma unroll
  for (int i = 0; i < W; ++i)
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) a[i][j] = (j == W + i) ? 1.0 : 0.0;
  for (int ra = 0; ra < 4; ++ra) {
    const int row_a = sg * 4 + ra;
    if (row_a >= nrow) {
      for (int e = 0; e < B; ++e) a[ra * B + e][ra * B + e] = 1.0;
      continue;
    }
    const int na = K.rows[row_a];
    const int ax = na % G.nx1, ay = (na / G.nx1) % G.ny1, az = na / (G.nx1 * G.ny1);
    for (int rb = 0; rb < 4; ++rb) {
      const int row_b = sg * 4 + rb;
      if (row_b >= nrow) continue;
      const int nb = K.rows[row_b];
      const int dx = nb % G.nx1 - ax, dy = (nb / G.nx1) % G.ny1 - ay, dz = nb / (G.nx1 * G.ny1) - az;
      if (dx < -2 || dx > 2 || dy < -2 || dy > 2 || dz < -2 || dz > 2 || (D == 2 && dz != 0)) continue;
      const int slot = (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
      const T* blk = &K.val[((long long)slot * K.cap + row_a) * (B * B)];
      for (int e = 0; e < B; ++e)
        for (int f = 0; f < B; ++f) a[ra * B + e][rb * B + f] = (double)blk[e * B + f];
    }
  }
  bool ok = true;
  for (int c = 0; c < W; ++c) {
    int piv = c;
    double best = fabs(a[c][c]);
    for (int r = c + 1; r < W; ++r)
      if (fabs(a[r][c]) > best) { best = fabs(a[r][c]); piv = r; }
    if (!(best > 0.0) || !isfinite(best)) { ok = false; break; }
    if (piv != c)
      for (int j = 0; j < 2 * W; ++j) { const double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
    const double inv = 1.0 / a[c][c];
    for (int j = 0; j < 2 * W; ++j) a[c][j] *= inv;
    for (int r = 0; r < W; ++r) {
      if (r == c) continue;
      const double f = a[r][c];
      if (f != 0.0)
        for (int j = 0; j < 2 * W; ++j) a[r][j] -= f * a[c][j];
    }
  }
  T* M = K.dinv + (long long)sg * W * W;
  if (!ok) atomicOr(err, ERRF_NONFINITE);
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j) M[i * W + j] = ok ? (T)a[i][W + j] : (T)(i == j ? 1.0 : 0.0);
}

template <int D, class T, int B>
cudaError_t launch_block_jacobi(const DevGrid& G, DevMatrix<T> K, int nrow_host, int* err, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  if (K.seg == 4) {
    const int nseg = (nrow_host + 3) / 4;
    k_segment_inverse<D, T, B><<<nblocks(nseg, 128), 128, 0, st>>>(G, K, nrow_host, err);
    return cudaGetLastError();
  }
  k_block_jacobi<D, T, B><<<nblocks(nrow_host), TPB, 0, st>>>(K, nrow_host, err);
  return cudaGetLastError();
}

// Is block (i, i + offset of `slot`) structurally present: the neighbour is
// an active node and the pair shares an occupied cell (base node)?
template <int D>
__device__ bool pattern_hit(const DevGrid& G, int ix, int iy, int iz, int slot, const int* __restrict__ node2row,
                            const int* __restrict__ count) {
  int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
  int j3[3] = {ix + dx, iy + dy, iz + dz};
  int i3[3] = {ix, iy, iz};
  bool inside = j3[0] >= 0 && j3[1] >= 0 && j3[0] < G.nx1 && j3[1] < G.ny1 &&
                (D == 2 || (j3[2] >= 0 && j3[2] < G.nz1));
  if (!inside) return false;
  long long j = j3[0] + (long long)G.nx1 * (j3[1] + (long long)G.ny1 * j3[2]);
  if (node2row[j] < 0) return false;
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      lo[a] = max(max(i3[a], j3[a]) - 2, 0);
      hi[a] = min(min(i3[a], j3[a]), G.n[a] - 2);
    } else { lo[a] = 0; hi[a] = 0; }
  }
  for (int cz = lo[2]; cz <= hi[2]; ++cz)
    for (int cy = lo[1]; cy <= hi[1]; ++cy)
      for (int cx = lo[0]; cx <= hi[0]; ++cx)
        if (count[cx + (long long)G.nx1 * (cy + (long long)G.ny1 * cz)] > 0) return true;
  return false;
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
  for (int slot = 0; slot < S; ++slot)
    if (pattern_hit<D>(G, ix, iy, iz, slot, node2row, count)) mask[(long long)row * S + slot] = 1;
}

template <int D>
__global__ void k_pattern_bits(DevGrid G, const int* __restrict__ rows, int nrow,
                               const int* __restrict__ node2row, const int* __restrict__ count, unsigned* bits) {
  constexpr int S = (D == 2) ? 25 : 125, PW = pmask_words(D);
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  int i = rows[row];
  int ix = i % G.nx1, iy = (i / G.nx1) % G.ny1, iz = i / (G.nx1 * G.ny1);
  for (int w = 0; w < PW; ++w) {
    unsigned word = 0u;
    for (int b = 0; b < 32; ++b) {
      const int slot = 32 * w + b;
      if (slot < S && pattern_hit<D>(G, ix, iy, iz, slot, node2row, count)) word |= 1u << b;
    }
    bits[(long long)row * PW + w] = word;
  }
}
template <int D>
cudaError_t launch_pattern_count(const DevGrid& G, const int* rows, int nrow_host, const int* node2row,
                                 const int* count, int* mask, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  k_pattern_count<D><<<nblocks(nrow_host), TPB, 0, st>>>(G, rows, nrow_host, node2row, count, mask);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_pattern_bits(const DevGrid& G, const int* rows, int nrow_host, const int* node2row,
                                const int* count, unsigned* bits, cudaStream_t st) {
  if (nrow_host == 0) return cudaSuccess;
  k_pattern_bits<D><<<nblocks(nrow_host), TPB, 0, st>>>(G, rows, nrow_host, node2row, count, bits);
  return cudaGetLastError();
}

// ||r||^2 over free DOFs of active rows, summed in an order fixed by the
// grid: each block stores its sum in part[block] and takes a ticket; the
// block that takes the last one adds the stored sums in block order, writes
// *out and resets the ticket.
template <int D>
__global__ void k_norm_free(const double* __restrict__ r, const int* __restrict__ rows, int nrow,
                            const uint8_t* __restrict__ fixed, double* out, double* part, unsigned* ticket) {
  __shared__ double ws[TPB / 32];
  __shared__ int last;
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
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < TPB / 32; ++w) v += ws[w];
    part[blockIdx.x] = v;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += TPB) t += __ldcg(&part[b]);
  t = warp_sum(t);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < TPB / 32; ++w) v += ws[w];
    *out = v;
    *ticket = 0u;
  }
}
template <int D>
cudaError_t launch_norm_free(const double* r, const int* rows, int nrow_host, const uint8_t* fixed,
                             double* out, double* part, unsigned* ticket, cudaStream_t st) {
  if (nrow_host == 0) return cudaMemsetAsync(out, 0, sizeof(double), st);
  k_norm_free<D><<<nblocks(nrow_host), TPB, 0, st>>>(r, rows, nrow_host, fixed, out, part, ticket);
  return cudaGetLastError();
}

// r at every grid node: the contributions fp of the particles of the 3^dim
// cells i - k that reach it, added in cell order (k = kx + 3 ky + 9 kz) and,
// within a cell, in the particles' sorted order, so that r does not depend
// on the order in which threads run.  B values per node.
template <int D, int B>
__global__ void k_gather_residual(DevGrid G, const int* __restrict__ cstart, const double* __restrict__ fp,
                                  int np, double* r, long long nn) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int ix = (int)(i % G.nx1), iy = (int)((i / G.nx1) % G.ny1), iz = (int)(i / ((long long)G.nx1 * G.ny1));
  constexpr int KZ = (D == 3) ? 3 : 1;
  double acc[B];
#pragma unroll
  for (int a = 0; a < B; ++a) acc[a] = 0.0;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const int cx = ix - kx, cy = iy - ky, cz = iz - kz;
        if (cx < 0 || cy < 0 || cz < 0) continue;
        const long long cell = cx + (long long)G.nx1 * (cy + (long long)G.ny1 * cz);
        const int p0 = cstart[cell], p1 = cstart[cell + 1];
        const double* f = fp + (long long)(kx + 3 * (ky + 3 * kz)) * B * np;
        for (int p = p0; p < p1; ++p)
#pragma unroll
          for (int a = 0; a < B; ++a) acc[a] += f[(long long)a * np + p];
      }
#pragma unroll
  for (int a = 0; a < B; ++a) r[i * B + a] = acc[a];
}
template <int D, int B>
cudaError_t launch_gather_residual(const DevGrid& G, const int* cstart, const double* fp, int np, double* r,
                                   long long nn, cudaStream_t st) {
  if (nn == 0) return cudaSuccess;
  k_gather_residual<D, B><<<nblocks(nn), TPB, 0, st>>>(G, cstart, fp, np, r, nn);
  return cudaGetLastError();
}

// The particles of each cell in increasing source index (perm[dst] = src):
// the counting sort places a cell's particles in arrival order, which this
// makes independent of the order in which threads ran.  One thread per cell,
// insertion sort (cells hold a few dozen particles at most).
__global__ void k_sort_cells(const int* __restrict__ cstart, int* perm, long long ncells) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int p0 = cstart[c], p1 = cstart[c + 1];
  for (int a = p0 + 1; a < p1; ++a) {
    const int v = perm[a];
    int b = a - 1;
    while (b >= p0 && perm[b] > v) {
      perm[b + 1] = perm[b];
      --b;
    }
    perm[b + 1] = v;
  }
}
cudaError_t launch_sort_cells(const int* cstart, int* perm, long long ncells, cudaStream_t st) {
  if (ncells == 0) return cudaSuccess;
  k_sort_cells<<<nblocks(ncells), TPB, 0, st>>>(cstart, perm, ncells);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- instantiations
#define MPM_INST_D(D)                                                                                   \
  template cudaError_t launch_cell_keys<D>(const DevParticles&, const DevGrid&, int*, int*, int*, int*,  \
                                           cudaStream_t);                                                \
  template cudaError_t launch_mass<D>(const DevParticles&, const DevGrid&, const int*, double*, double*, \
                                      long long, cudaStream_t);                                         \
  template cudaError_t launch_stress_out<D>(const DevParticles&, const DevGrid&, const MatC*, double*,   \
                                            cudaStream_t);                                               \
  template cudaError_t launch_pattern_count<D>(const DevGrid&, const int*, int, const int*, const int*,  \
                                               int*, cudaStream_t);                                      \
  template cudaError_t launch_pattern_bits<D>(const DevGrid&, const int*, int, const int*, const int*,   \
                                              unsigned*, cudaStream_t);                                  \
  template cudaError_t launch_norm_free<D>(const double*, const int*, int, const uint8_t*, double*,      \
                                           double*, unsigned*, cudaStream_t);
MPM_INST_D(2)
MPM_INST_D(3)
template cudaError_t launch_gather_residual<2, 1>(const DevGrid&, const int*, const double*, int, double*, long long,
                                                  cudaStream_t);
template cudaError_t launch_gather_residual<3, 1>(const DevGrid&, const int*, const double*, int, double*, long long,
                                                  cudaStream_t);
template cudaError_t launch_gather_residual<2, 2>(const DevGrid&, const int*, const double*, int, double*, long long,
                                                  cudaStream_t);
template cudaError_t launch_gather_residual<2, 3>(const DevGrid&, const int*, const double*, int, double*, long long,
                                                  cudaStream_t);
template cudaError_t launch_gather_residual<3, 3>(const DevGrid&, const int*, const double*, int, double*, long long,
                                                  cudaStream_t);

#define MPM_INST_DT(D, T)                                                                               \
  template cudaError_t launch_particles<D, T>(const DevParticles&, const DevGrid&, const MatC*,          \
                                              const double*, double*, const double*, T*, int, int*,      \
                                              int*, cudaStream_t);
MPM_INST_DT(2, float)
MPM_INST_DT(2, double)
MPM_INST_DT(3, float)
MPM_INST_DT(3, double)

#define MPM_INST_DTB(D, T, B)                                                                           \
  template cudaError_t launch_assemble<D, T, B>(const DevParticles&, const DevGrid&, const int*, const int*, \
                                                const T*, DevMatrix<T>, int, const Asm3<T>*, cudaStream_t); \
  template cudaError_t launch_bc_matrix<D, T, B>(const DevGrid&, DevMatrix<T>, const uint8_t*, const int*, \
                                                 int, cudaStream_t);                                     \
  template cudaError_t launch_block_jacobi<D, T, B>(const DevGrid&, DevMatrix<T>, int, int*, cudaStream_t);
MPM_INST_DTB(2, float, 2)
MPM_INST_DTB(2, double, 2)
MPM_INST_DTB(3, float, 3)
MPM_INST_DTB(3, double, 3)
MPM_INST_DTB(2, float, 3)
MPM_INST_DTB(2, double, 3)

}  // namespace mpm
