// Adjoint of one converged implicit load step (the paper's inverse analysis,
// Sec. 4.5, differentiates through its implicit steps with the Jacobian it
// already has; here the adjoint is hand-written).  For a loss L(du) of the
// step's converged nodal increment, with r(du; theta) = 0,
//   J^T lambda = dL/du,   dL/dtheta = -lambda^T dr/dtheta,
// with J the converged Jacobian and theta the per-particle Young's modulus,
// friction angle and (u-p) hydraulic conductivity.  In the solver's scaled
// variables (pressure unknowns p / psc, mass-balance rows times psc, see
// mpm_up.cu) the same solve reads Jhat^T mu = S dL/du and
// dL/dtheta = -mu^T d rhat / dtheta.
// Kernels: the block transpose of the stencil-BSR Jacobian, P2G of a loss
// gradient given on particle displacements, the particle increment
// sum_i w_ip du_i, and the per-particle parameter gradient (G2P of mu
// against the particle's stress derivative).  The stress derivatives with
// respect to E and phi are central differences of the FP64 constitutive
// update at a relative step of 1e-6 (the return map is smooth within a
// branch; the truncation error is about 1e-12 relative); the Darcy term is
// linear in the conductivity k (kdt = k dt / gamma_w) and differentiated
// exactly.
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int ATPB = 128;
inline int ablocks(long long n, int tpb = ATPB) { return (int)((n + tpb - 1) / tpb); }

__device__ __forceinline__ bool particle_splines(const DevParticles& P, const DevGrid& G, int p, int D,
                                                 Spline1 sp[3]) {
  for (int a = 0; a < D; ++a) sp[a] = spline1((P.x[a][p] - G.o[a]) / G.h);
  if (D == 2) { sp[2].base = 0; sp[2].N[0] = 1.0; sp[2].dN[0] = 0.0; }
  bool inside = true;
  for (int a = 0; a < D; ++a) inside = inside && sp[a].base >= 0 && sp[a].base <= G.n[a] - 2;
  return inside;
}
}  // namespace

// out = blockwise transpose of K: block (row i, offset o) of out is the
// transpose of block (row of i + o, offset -o) of K; zero where i + o is not
// an active node.
template <int D, class T, int B>
__global__ void k_transpose_blocks(DevGrid G, DevMatrix<T> K, const int* __restrict__ node2row, T* out,
                                   int nrow) {
  constexpr int S = (D == 2) ? 25 : 125;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nrow * S) return;
  const int row = (int)(t % nrow), slot = (int)(t / nrow);
  const int i = K.rows[row];
  const int ix = i % G.nx1, iy = (i / G.nx1) % G.ny1, iz = i / (G.nx1 * G.ny1);
  const int dx = slot % 5 - 2, dy = (slot / 5) % 5 - 2, dz = (D == 3) ? slot / 25 - 2 : 0;
  const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
  T* o = out + ((long long)slot * K.cap + row) * (B * B);
  int rj = -1;
  if (jx >= 0 && jy >= 0 && jz >= 0 && jx < G.nx1 && jy < G.ny1 && jz < G.nz1)
    rj = node2row[jx + (long long)G.nx1 * (jy + (long long)G.ny1 * jz)];
  if (rj < 0) {
#pragma unroll
    for (int e = 0; e < B * B; ++e) o[e] = (T)0;
    return;
  }
  const T* src = K.val + ((long long)(S - 1 - slot) * K.cap + rj) * (B * B);
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int b = 0; b < B; ++b) o[a * B + b] = src[b * B + a];
}

// g[node*B + a] += sum_p w_ip dLdx[orig(p)][a]  (a < D): a loss gradient on
// the particle displacements sum_i w_ip du_i, mapped to the nodal increment.
template <int D, int B>
__global__ void k_loss_p2g(DevParticles P, DevGrid G, const double* __restrict__ dLdx, double* g, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  Spline1 sp[3];
  if (!particle_splines(P, G, p, D, sp)) {
    atomicOr(err, ERRF_BOUNDS);
    return;
  }
  const long long nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
  const int o = P.orig[p];
  double gl[3];
  for (int a = 0; a < 3; ++a) gl[a] = dLdx[3LL * o + a];
  const int KZ = (D == 3) ? 3 : 1;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
        for (int a = 0; a < D; ++a) atomicAdd(&g[node * B + a], w * gl[a]);
      }
}

// b = -(S g) on the DOFs: the Krylov solve takes J x = -b
template <int B, int D>
__global__ void k_adjoint_rhs(const double* __restrict__ g, double* b, long long ndof, double psc) {
  const long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (d >= ndof) return;
  const double sc = (B > D && d % B == D) ? psc : 1.0;
  b[d] = -sc * g[d];
}

// du_p = sum_i w_ip du_i (caller order, 3 per particle, zeros past D)
template <int D, int B>
__global__ void k_particle_increment(DevParticles P, DevGrid G, const double* __restrict__ U, double* out,
                                     int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  Spline1 sp[3];
  if (!particle_splines(P, G, p, D, sp)) {
    atomicOr(err, ERRF_BOUNDS);
    return;
  }
  const long long nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
  double dx[3] = {0.0, 0.0, 0.0};
  const int KZ = (D == 3) ? 3 : 1;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
        for (int a = 0; a < D; ++a) dx[a] += w * U[node * B + a];
      }
  const int o = P.orig[p];
  for (int a = 0; a < 3; ++a) out[3LL * o + a] = dx[a];
}

// Per-particle parameter gradients -mu^T d rhat / d theta.
template <int D, class T, int B>
__global__ void __launch_bounds__(ATPB) k_param_grad(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                     const double* __restrict__ U, const T* __restrict__ mu,
                                                     double psc, double* gE, double* gPhi, double* gK, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  Spline1 sp[3];
  if (!particle_splines(P, G, p, D, sp)) {
    atomicOr(err, ERRF_BOUNDS);
    return;
  }
  const long long nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
  const int KZ = (D == 3) ? 3 : 1;
  PState st;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) st.F[a][c] = (a == c) ? 1.0 : 0.0;
  double Lam[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // sum_i mu_i (x) grad w_ip
  double Gp[3] = {0, 0, 0}, mg[3] = {0, 0, 0};           // u-p: grad p_p, sum_i mu_p,i grad w_ip
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        double g[3];
        g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
        g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
        g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
        for (int a = 0; a < D; ++a) {
          const double u = U[node * B + a];
          const double m = (double)mu[node * B + a];
          for (int c = 0; c < D; ++c) {
            st.F[a][c] += u * g[c];
            Lam[a][c] += m * g[c];
          }
        }
        if (B > D) {
          const double pn = U[node * B + D] * psc, m = (double)mu[node * B + D];
          for (int c = 0; c < D; ++c) {
            Gp[c] += pn * g[c];
            mg[c] += m * g[c];
          }
        }
      }
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
  const double V0 = P.vol0[p], E = P.Ep[p], phi = P.phip[p], pcn = P.pc[p];
  const int o = P.orig[p];
  // dL/dtheta = -lambda^T dr/dtheta; per particle dr_i/dtheta = (dP/dtheta) grad w_ip
  // with dP/dtheta = V0 (dtau/dtheta) dF^-T (the pressure part of the u-p
  // stress depends on neither E nor phi), dtau/dtheta written out by
  // param_dtau (no finite differences)
  bool ok = true;
  if (gE || gPhi) {
    PState s2 = st;
    double dtE[3][3], dtP[3][3];
    ok = constitutive<D>(mc, E, phi, pcn, V0, s2) == 0 && param_dtau<D>(mc, E, phi, pcn, s2, dtE, dtP);
    if (ok) {
      double vE = 0.0, vP = 0.0;
      for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) {
          double pe = 0.0, pp = 0.0;
          for (int k = 0; k < 3; ++k) {
            pe += dtE[a][k] * s2.Fi[c][k];
            pp += dtP[a][k] * s2.Fi[c][k];
          }
          vE += Lam[a][c] * V0 * pe;
          vP += Lam[a][c] * V0 * pp;
        }
      if (gE) gE[o] = -vE;
      if (gPhi) gPhi[o] = (mc.model == MODEL_NH_DP) ? -vP : 0.0;
    }
  }
  if (gK && B > D && P.kdt) {
    // fl = kdt V^n det(dF) dF^-1 dF^-T grad p: linear in kdt, hence in k
    PState s2 = st;
    ok = ok && constitutive<D>(mc, E, phi, pcn, V0, s2) == 0;
    if (ok) {
      double Fn[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) Fn[a][c] = P.F[a * D + c][p];
      const double Vnew = V0 * det3(Fn) * det3(s2.F);
      const double (&X)[3][3] = s2.Fi;
      double t[3], Xt[3];
      for (int k = 0; k < 3; ++k) t[k] = X[0][k] * Gp[0] + X[1][k] * Gp[1] + X[2][k] * Gp[2];
      for (int c = 0; c < 3; ++c) Xt[c] = X[c][0] * t[0] + X[c][1] * t[1] + X[c][2] * t[2];
      double v = 0.0;
      for (int c = 0; c < D; ++c) v += mg[c] * mc.dkdt_dk * Vnew * Xt[c];
      atomicAdd(&gK[P.mat[p]], -psc * v);
    }
  }
  if (!ok) atomicOr(err, ERRF_RETURN);
}

template <int D, class T, int B>
cudaError_t launch_transpose_blocks(const DevGrid& G, DevMatrix<T> K, const int* node2row, T* out, int nrow,
                                    cudaStream_t st) {
  constexpr int S = (D == 2) ? 25 : 125;
  if (nrow == 0) return cudaSuccess;
  k_transpose_blocks<D, T, B><<<ablocks((long long)nrow * S, 256), 256, 0, st>>>(G, K, node2row, out, nrow);
  return cudaGetLastError();
}
template <int D, int B>
cudaError_t launch_loss_p2g(const DevParticles& P, const DevGrid& G, const double* dLdx, double* g, int* err,
                            cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_loss_p2g<D, B><<<ablocks(P.np), ATPB, 0, st>>>(P, G, dLdx, g, err);
  return cudaGetLastError();
}
template <int D, int B>
cudaError_t launch_adjoint_rhs(const double* g, double* b, long long ndof, double psc, cudaStream_t st) {
  if (ndof == 0) return cudaSuccess;
  k_adjoint_rhs<B, D><<<ablocks(ndof, 256), 256, 0, st>>>(g, b, ndof, psc);
  return cudaGetLastError();
}
template <int D, int B>
cudaError_t launch_particle_increment(const DevParticles& P, const DevGrid& G, const double* U, double* out,
                                      int* err, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_particle_increment<D, B><<<ablocks(P.np), ATPB, 0, st>>>(P, G, U, out, err);
  return cudaGetLastError();
}
template <int D, class T, int B>
cudaError_t launch_param_grad(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* U,
                              const T* mu, double psc, double* gE, double* gPhi, double* gK, int* err,
                              cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_param_grad<D, T, B><<<ablocks(P.np), ATPB, 0, st>>>(P, G, mats, U, mu, psc, gE, gPhi, gK, err);
  return cudaGetLastError();
}

#define MPM_ADJ_INST(D, T, B)                                                                           \
  template cudaError_t launch_transpose_blocks<D, T, B>(const DevGrid&, DevMatrix<T>, const int*, T*, int, \
                                                        cudaStream_t);                                   \
  template cudaError_t launch_param_grad<D, T, B>(const DevParticles&, const DevGrid&, const MatC*,      \
                                                  const double*, const T*, double, double*, double*,     \
                                                  double*, int*, cudaStream_t);
MPM_ADJ_INST(2, float, 2)
MPM_ADJ_INST(2, double, 2)
MPM_ADJ_INST(3, float, 3)
MPM_ADJ_INST(3, double, 3)
MPM_ADJ_INST(2, float, 3)
MPM_ADJ_INST(2, double, 3)

#define MPM_ADJ_INST_DB(D, B)                                                                           \
  template cudaError_t launch_loss_p2g<D, B>(const DevParticles&, const DevGrid&, const double*, double*, \
                                             int*, cudaStream_t);                                        \
  template cudaError_t launch_adjoint_rhs<D, B>(const double*, double*, long long, double, cudaStream_t); \
  template cudaError_t launch_particle_increment<D, B>(const DevParticles&, const DevGrid&, const double*, \
                                                       double*, int*, cudaStream_t);
MPM_ADJ_INST_DB(2, 2)
MPM_ADJ_INST_DB(3, 3)
MPM_ADJ_INST_DB(2, 3)

}  // namespace mpm
