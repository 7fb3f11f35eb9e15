// Particle pass of the coupled u-p formulation (the paper's Sec. 2.2 remark
// on poromechanics; Sec. 4.4 verifies it on one-dimensional consolidation).
// The paper defers the equations to the stabilised-MPM u-p literature; the
// form used here is: mixture momentum with the total stress sigma' - p 1,
// fluid mass balance with incompressible constituents
// (J^{n+1} - J^n) / (dt J^{n+1}) + div q = 0, Darcy q = -kappa grad p,
// backward Euler in time, the same quadratic B-splines for u and p, no
// stabilisation.  Per particle, with dF the step's deformation gradient,
// V^n = V0 det F^n, p_p = sum_j w_jp p_j and G_p = sum_j p_j grad w_jp
// (start-of-step gradients), and the mass balance multiplied by dt:
//   momentum:  r_u,i += (P'_p - p_p V^n det(dF) dF^-T) grad w_ip - w_ip f_p
//   mass:      r_p,i += w_ip V^n (det dF - 1)
//                       + kdt_p V^n det(dF) grad w_ip . (dF^-1 dF^-T G_p)
// with kdt = kappa dt.  Node values are (du_0 .. du_{D-1}, p / psc); the
// mass-balance rows of r and the pressure rows and columns of the tangent
// are multiplied by psc, which puts the pressure block on the scale of the
// displacement block (one norm for Newton and Krylov, FP32-safe entries).
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int UP_TPB = 128;
}

// MODE 0 residual, 1 residual + tangent, 2 commit.
// Tangent layout per particle (stride np): A[((a*NPHI + c)*B + b)*NPHI + e]
// with a, b < B node values and c, e < NPHI = D + 1 shape-function parts
// (gradient entries 0..D-1, weight D), so that
// K_ij[a][b] = sum_c,e phi_i[c] A[a c b e] phi_j[e], phi = (grad w, w).
template <int D, class T, int MODE>
__global__ void __launch_bounds__(UP_TPB) k_particles_up(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                         const double* __restrict__ U, double* fp,
                                                         const double* __restrict__ grav, T* A, double psc,
                                                         int* err, int* nplastic) {
  constexpr int B = D + 1, NPHI = D + 1;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  bool live = p < P.np;
  bool wrote = false;
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
    double pp = 0.0, Gp[3] = {0.0, 0.0, 0.0};
    for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
          const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
          double g[3];
          g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
          g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
          g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const double u = U[node * B + a];
#pragma unroll
            for (int c = 0; c < D; ++c) st.F[a][c] += u * g[c];
          }
          const double pn = U[node * B + D] * psc;
          pp += w * pn;
#pragma unroll
          for (int c = 0; c < D; ++c) Gp[c] += pn * g[c];
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
    const double V0 = P.vol0[p];
    int e = constitutive<D>(mc, P.Ep[p], P.phip[p], P.pc[p], V0, st);
    if (e) {
      atomicOr(err, e);
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
      // V^n from the start-of-step F (plane strain: F_zz = 1)
      double Fn[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c) Fn[a][c] = P.F[a * D + c][p];
      const double Vn = V0 * det3(Fn);
      const double jdF = det3(st.F);
      const double Vnew = Vn * jdF;
      const double (&X)[3][3] = st.Fi;   // dF^-1
      const double kdt = P.kdt[p];
      double t[3], Xt[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = X[0][k] * Gp[0] + X[1][k] * Gp[1] + X[2][k] * Gp[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) Xt[c] = X[c][0] * t[0] + X[c][1] * t[1] + X[c][2] * t[2];
      if (MODE == 2) {
        double dx[3] = {0.0, 0.0, 0.0};
        for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
              const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
#pragma unroll
              for (int a = 0; a < D; ++a) dx[a] += w * U[node * B + a];
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
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += st.F[a][k] * Fn[k][c];
            P.F[a * D + c][p] = s;
          }
        P.pp[p] = pp;
      } else {
        // total first Piola-type stress P' + Pp, Pp = -p_p V^{n+1} dF^-T
        double Pt[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) Pt[a][c] = st.P[a][c] - pp * Vnew * X[c][a];
        const double vol = Vn * (jdF - 1.0);
        double fl[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) fl[c] = kdt * Vnew * Xt[c];
        const double m = P.mass[p];
        double gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a] = m * grav[a] + (P.fext[a] ? P.fext[a][p] : 0.0);
        bool finite = true;
        for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
              const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
              double g[3];
              g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
              g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
              g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
              double* fk = fp + (long long)(kx + 3 * (ky + 3 * kz)) * B * P.np + p;
#pragma unroll
              for (int a = 0; a < D; ++a) {
                double f = -w * gv[a];
#pragma unroll
                for (int c = 0; c < D; ++c) f += Pt[a][c] * g[c];
                finite = finite && isfinite(f);
                fk[(long long)a * P.np] = f;
              }
              double q = w * vol;
#pragma unroll
              for (int c = 0; c < D; ++c) q += fl[c] * g[c];
              q *= psc;
              finite = finite && isfinite(q);
              fk[(long long)D * P.np] = q;
            }
        wrote = true;
        if (!finite) atomicOr(err, ERRF_NONFINITE);
        if (MODE == 1) {
          // effective-stress tangent of the single-phase path, then the
          // pressure, volume and flux terms differentiated in closed form
          double As[D * D * D * D];
          tangent<D, double>(st, V0, As, 1);
          double XXt[3][3];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2) XXt[c][e2] = X[c][0] * X[e2][0] + X[c][1] * X[e2][1] + X[c][2] * X[e2][2];
          T* out = A + p;
          const long long stride = P.np;
#pragma unroll
          for (int a = 0; a < B; ++a)
#pragma unroll
            for (int c = 0; c < NPHI; ++c)
#pragma unroll
              for (int b = 0; b < B; ++b)
#pragma unroll
                for (int e2 = 0; e2 < NPHI; ++e2) {
                  double v = 0.0;
                  if (a < D && b < D) {
                    // d(P' + Pp)[a][c] / d dF[b][e]
                    if (c < D && e2 < D)
                      v = As[((a * D + c) * D + b) * D + e2] -
                          pp * Vnew * (X[e2][b] * X[c][a] - X[c][b] * X[e2][a]);
                  } else if (a < D && b == D) {
                    // d Pp[a][c] / d p_p, reached through the weight of node j
                    if (c < D && e2 == D) v = -Vnew * X[c][a] * psc;
                  } else if (a == D && b < D) {
                    // volume term (tested with w_i) and flux term (with grad w_i)
                    if (c == D && e2 < D) v = Vnew * X[e2][b] * psc;
                    else if (c < D && e2 < D)
                      v = kdt * Vnew * (X[e2][b] * Xt[c] - X[c][b] * Xt[e2] - t[b] * XXt[c][e2]) * psc;
                  } else {
                    // d fl[c] / d G_p[e], reached through grad w_j
                    if (c < D && e2 < D) v = kdt * Vnew * XXt[c][e2] * psc * psc;
                  }
                  out[(long long)(((a * NPHI + c) * B + b) * NPHI + e2) * stride] = (T)v;
                }
        }
      }
    }
  }
  if (MODE != 2 && p < P.np && !wrote) {
    constexpr int NS = (D == 3) ? 27 : 9;
    for (int k = 0; k < NS * B; ++k) fp[(long long)k * P.np + p] = 0.0;
  }
  if (nplastic) {
    unsigned bal = __ballot_sync(0xffffffffu, plastic);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(nplastic, __popc(bal));
  }
}

template <int D, class T>
cudaError_t launch_particles_up(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* U,
                                double* r, const double* grav, T* A, int mode, double psc, int* err,
                                int* nplastic, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  if (!P.kdt || !P.pp) return cudaErrorInvalidValue;
  const int nb = (P.np + UP_TPB - 1) / UP_TPB;
  if (mode == 0) k_particles_up<D, T, 0><<<nb, UP_TPB, 0, st>>>(P, G, mats, U, r, grav, A, psc, err, nplastic);
  else if (mode == 1) k_particles_up<D, T, 1><<<nb, UP_TPB, 0, st>>>(P, G, mats, U, r, grav, A, psc, err, nplastic);
  else k_particles_up<D, T, 2><<<nb, UP_TPB, 0, st>>>(P, G, mats, U, r, grav, A, psc, err, nplastic);
  return cudaGetLastError();
}

template cudaError_t launch_particles_up<2, float>(const DevParticles&, const DevGrid&, const MatC*, const double*,
                                                   double*, const double*, float*, int, double, int*, int*,
                                                   cudaStream_t);
template cudaError_t launch_particles_up<2, double>(const DevParticles&, const DevGrid&, const MatC*, const double*,
                                                    double*, const double*, double*, int, double, int*, int*,
                                                    cudaStream_t);

}  // namespace mpm
