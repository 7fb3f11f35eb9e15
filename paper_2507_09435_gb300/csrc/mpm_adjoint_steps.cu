// Reverse-mode chain through a sequence of implicit load steps.  Step n maps
// the start-of-step particle state s_{n-1} = (x, b_e, p_c, F) and the
// parameters theta to its converged increment U_n (r(U_n; s_{n-1}, theta) = 0)
// and to the committed state s_n = Phi(U_n, s_{n-1}, theta).  Given the
// adjoint sbar_n of s_n and the loss's direct gradient g_n on U_n:
//   g_n    += (dPhi/dU)^T sbar_n                     (pass A, per particle)
//   J^T lambda_n = g_n                                (transposed solve)
//   thetabar   += (dPhi/dtheta)^T sbar_n - lambda_n^T dr/dtheta
//   sbar_{n-1}  = (dPhi/ds)^T sbar_n - lambda_n^T dr/ds (pass B)
// Per particle both passes differentiate one scalar function of the
// particle's local inputs: q = sbar . Phi_p - mu . rhat_p (rhat the solver's
// scaled residual, mu its adjoint) with respect to the position (through the
// B-spline weights and gradients), b_e, p_c, F, E, phi, kdt and, for pass A,
// an offset added to dF and to the particle increment (whose derivatives are
// mapped to the nodes with grad w_ip and w_ip).  The derivatives in E, phi
// and kdt are written out (local_param_grad); those in the particle state
// and in the dF / increment offsets are central differences of the FP64
// particle update (relative steps of 1e-6 to 1e-7).
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int VTPB = 64;

struct LocalZ {
  double x[3];
  double be[6];      // xx, yy, zz, xy, yz, xz
  double pc;
  double F[3][3];    // start-of-step deformation gradient
  double E, phi, kdt;
  double dFx[3][3];  // offset added to dF
  double dux[3];     // offset added to the particle increment
};

struct LocalOut {
  double h;  // sbar . Phi_p
  double f;  // -mu . rhat_p
};

// The particle's G2P at its local inputs: B-spline weights about the base
// node, dF = 1 + dFx + sum_i U_i (x) grad w_ip, the particle increment
// u_p = dux + sum_i w_ip U_i, and for u-p the pressure and its gradient;
// b_e of the start of the step into st.  Returns false if the support
// leaves the grid.
template <int D, int B>
__device__ bool local_g2p(const DevGrid& G, const double* __restrict__ U, double psc, const LocalZ& z,
                          Spline1 sp[3], long long& nb, PState& st, double up[3], double& pp, double Gp[3]) {
  for (int a = 0; a < D; ++a) sp[a] = spline1((z.x[a] - G.o[a]) / G.h);
  if (D == 2) { sp[2].base = 0; sp[2].N[0] = 1.0; sp[2].dN[0] = 0.0; }
  for (int a = 0; a < D; ++a)
    if (sp[a].base < 0 || sp[a].base > G.n[a] - 2) return false;
  nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
  const int KZ = (D == 3) ? 3 : 1;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) st.F[a][c] = ((a == c) ? 1.0 : 0.0) + z.dFx[a][c];
  for (int a = 0; a < 3; ++a) up[a] = z.dux[a];
  pp = 0.0;
  Gp[0] = Gp[1] = Gp[2] = 0.0;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
        double g[3];
        g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
        g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
        g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
        for (int a = 0; a < D; ++a) {
          const double u = U[node * B + a];
          up[a] += w * u;
          for (int c = 0; c < D; ++c) st.F[a][c] += u * g[c];
        }
        if (B > D) {
          const double pn = U[node * B + D] * psc;
          pp += w * pn;
          for (int c = 0; c < D; ++c) Gp[c] += pn * g[c];
        }
      }
  st.bn[0][0] = z.be[0]; st.bn[1][1] = z.be[1]; st.bn[2][2] = z.be[2];
  st.bn[0][1] = st.bn[1][0] = z.be[3];
  if (D == 3) {
    st.bn[1][2] = st.bn[2][1] = z.be[4];
    st.bn[0][2] = st.bn[2][0] = z.be[5];
  } else {
    st.bn[1][2] = st.bn[2][1] = st.bn[0][2] = st.bn[2][0] = 0.0;
  }
  return true;
}

// One evaluation of the particle's commit map and residual contribution.
template <int D, class T, int B>
__device__ __noinline__ bool local_eval(const DevGrid& G, const MatC& mc, double V0, double m, const double grav[3],
                           const double fe[3], const double* __restrict__ U, const T* __restrict__ mu, double psc,
                           const double* sb, const LocalZ& z, LocalOut& out) {
  Spline1 sp[3];
  long long nb;
  PState st;
  double up[3], pp, Gp[3];
  if (!local_g2p<D, B>(G, U, psc, z, sp, nb, st, up, pp, Gp)) return false;
  const int KZ = (D == 3) ? 3 : 1;
  if (constitutive<D>(mc, z.E, z.phi, z.pc, V0, st)) return false;
  // sbar . Phi: x' = x + u_p, b_e', p_c', F' = dF F
  double h = 0.0;
  for (int a = 0; a < D; ++a) h += sb[a] * (z.x[a] + up[a]);
  const double bnew[6] = {st.benew[0][0], st.benew[1][1], st.benew[2][2], 0.5 * (st.benew[0][1] + st.benew[1][0]),
                          0.5 * (st.benew[1][2] + st.benew[2][1]), 0.5 * (st.benew[0][2] + st.benew[2][0])};
  const int nbe = (D == 2) ? 4 : 6;
  for (int k = 0; k < nbe; ++k) h += sb[3 + k] * bnew[k];
  h += sb[9] * st.pc;
  for (int a = 0; a < D; ++a)
    for (int c = 0; c < D; ++c) {
      double v = 0.0;
      for (int k = 0; k < D; ++k) v += st.F[a][k] * z.F[k][c];
      h += sb[10 + 3 * a + c] * v;
    }
  out.h = h;
  out.f = 0.0;
  if (!mu) return true;
  // -mu . rhat_p: momentum rows, then (u-p) the scaled mass-balance rows
  double Pt[3][3];
  double Vnew = 0.0, vol = 0.0, fl[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) Pt[a][c] = st.P[a][c];
  if (B > D) {
    const double Vn = V0 * det3(z.F);
    const double jdF = det3(st.F);
    Vnew = Vn * jdF;
    vol = Vn * (jdF - 1.0);
    const double (&X)[3][3] = st.Fi;
    double t[3], Xt[3];
    for (int k = 0; k < 3; ++k) t[k] = X[0][k] * Gp[0] + X[1][k] * Gp[1] + X[2][k] * Gp[2];
    for (int c = 0; c < 3; ++c) Xt[c] = X[c][0] * t[0] + X[c][1] * t[1] + X[c][2] * t[2];
    for (int c = 0; c < 3; ++c) fl[c] = z.kdt * Vnew * Xt[c];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) Pt[a][c] -= pp * Vnew * X[c][a];
  }
  double s = 0.0;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
        double g[3];
        g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
        g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
        g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
        for (int a = 0; a < D; ++a) {
          double r = -w * (m * grav[a] + fe[a]);
          for (int c = 0; c < D; ++c) r += Pt[a][c] * g[c];
          s += (double)mu[node * B + a] * r;
        }
        if (B > D) {
          double q = w * vol;
          for (int c = 0; c < D; ++c) q += fl[c] * g[c];
          s += (double)mu[node * B + D] * psc * q;
        }
      }
  out.f = -s;
  return true;
}

// Derivatives of q = sbar . Phi_p - mu . rhat_p with respect to E, phi and
// kdt, written out (no differences): E and phi reach the commit map through
// the returned principal log strains, b_e' = Q diag(exp(2 eps)) Q^T and
// p_c' = p_c exp(-sum(eps^tr - eps) / (lambda - kappa)) (Cam-Clay), and the
// residual through P = V0 tau dF^-T (param_dtau); kdt enters the u-p Darcy
// term fl = kdt V det(dF) dF^-1 dF^-T grad p linearly.
template <int D, class T, int B>
__device__ __noinline__ bool local_param_grad(const DevGrid& G, const MatC& mc, double V0,
                                              const double* __restrict__ U, const T* __restrict__ mu, double psc,
                                              const double* sb, const LocalZ& z, double& qE, double& qP,
                                              double& qK) {
  Spline1 sp[3];
  long long nb;
  PState st;
  double up[3], pp, Gp[3];
  qE = qP = qK = 0.0;
  if (!local_g2p<D, B>(G, U, psc, z, sp, nb, st, up, pp, Gp)) return false;
  if (constitutive<D>(mc, z.E, z.phi, z.pc, V0, st)) return false;
  double dtE[3][3], dtP[3][3], deps[3][2];
  if (!param_dtau<D>(mc, z.E, z.phi, z.pc, st, dtE, dtP, deps)) return false;
  // commit map
  if (st.mode != 0) {
    double dbE[3][3], dbP[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double e = 0.0, f = 0.0;
        for (int A = 0; A < 3; ++A) {
          const double c = 2.0 * exp(2.0 * st.eps[A]) * st.Q[i][A] * st.Q[j][A];
          e += c * deps[A][0];
          f += c * deps[A][1];
        }
        dbE[i][j] = e;
        dbP[i][j] = f;
      }
    const int ii[6] = {0, 1, 2, 0, 1, 0}, jj[6] = {0, 1, 2, 1, 2, 2};
    const int nbe = (D == 2) ? 4 : 6;
    for (int k = 0; k < nbe; ++k) {
      qE += sb[3 + k] * dbE[ii[k]][jj[k]];
      qP += sb[3 + k] * dbP[ii[k]][jj[k]];
    }
    if (mc.model == MODEL_NH_MCC) {
      const double f = st.pc / mc.lmk;
      qE += sb[9] * f * (deps[0][0] + deps[1][0] + deps[2][0]);
      qP += sb[9] * f * (deps[0][1] + deps[1][1] + deps[2][1]);
    }
  }
  if (!mu) return true;
  // residual: d rhat_i = (V0 dtau dF^-T) grad w_ip on the momentum rows; the
  // Darcy part of the mass-balance rows for kdt
  double dPE[3][3], dPP[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double e = 0.0, f = 0.0;
      for (int k = 0; k < 3; ++k) {
        e += dtE[a][k] * st.Fi[c][k];
        f += dtP[a][k] * st.Fi[c][k];
      }
      dPE[a][c] = V0 * e;
      dPP[a][c] = V0 * f;
    }
  double Xt[3] = {0.0, 0.0, 0.0}, Vnew = 0.0;
  if (B > D) {
    Vnew = V0 * det3(z.F) * det3(st.F);
    const double (&X)[3][3] = st.Fi;
    double t[3];
    for (int k = 0; k < 3; ++k) t[k] = X[0][k] * Gp[0] + X[1][k] * Gp[1] + X[2][k] * Gp[2];
    for (int c = 0; c < 3; ++c) Xt[c] = X[c][0] * t[0] + X[c][1] * t[1] + X[c][2] * t[2];
  }
  const int KZ = (D == 3) ? 3 : 1;
  double sE = 0.0, sP = 0.0, sK = 0.0;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        double g[3];
        g[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
        g[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
        g[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
        for (int a = 0; a < D; ++a) {
          double re = 0.0, rp = 0.0;
          for (int c = 0; c < D; ++c) {
            re += dPE[a][c] * g[c];
            rp += dPP[a][c] * g[c];
          }
          const double m = (double)mu[node * B + a];
          sE += m * re;
          sP += m * rp;
        }
        if (B > D) {
          double qk = 0.0;
          for (int c = 0; c < D; ++c) qk += Vnew * Xt[c] * g[c];
          sK += (double)mu[node * B + D] * psc * qk;
        }
      }
  qE -= sE;
  qP -= sP;
  qK -= sK;
  return true;
}

template <int D>
__device__ void load_z(const DevParticles& P, int p, LocalZ& z) {
  for (int a = 0; a < 3; ++a) z.x[a] = (a < D) ? P.x[a][p] : 0.0;
  z.be[0] = P.be[0][p]; z.be[1] = P.be[1][p]; z.be[2] = P.be[2][p]; z.be[3] = P.be[3][p];
  z.be[4] = (D == 3) ? P.be[4][p] : 0.0;
  z.be[5] = (D == 3) ? P.be[5][p] : 0.0;
  z.pc = P.pc[p];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) z.F[a][c] = (a < D && c < D) ? P.F[a * D + c][p] : ((a == c) ? 1.0 : 0.0);
  z.E = P.Ep[p];
  z.phi = P.phip[p];
  z.kdt = P.kdt ? P.kdt[p] : 0.0;
  for (int a = 0; a < 3; ++a) {
    z.dux[a] = 0.0;
    for (int c = 0; c < 3; ++c) z.dFx[a][c] = 0.0;
  }
}

// pointer to the k-th perturbable input of the state part (x, b_e, p_c, F)
template <int D>
__device__ double* state_slot(LocalZ& z, int k) {
  if (k < D) return &z.x[k];
  k -= D;
  const int nbe = (D == 2) ? 4 : 6;
  if (k < nbe) return &z.be[k];
  k -= nbe;
  if (k == 0) return &z.pc;
  k -= 1;
  return &z.F[k / D][k % D];
}
}  // namespace

// Pass A: g_i += (dPhi_p/dU_i)^T sbar_p through dF and the particle increment.
template <int D, class T, int B>
__global__ void __launch_bounds__(VTPB) k_adj_commit_vjp(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                         const double* __restrict__ grav, const double* __restrict__ U,
                                                         double psc, const double* __restrict__ sbar, double* g,
                                                         int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const int o = P.orig[p];
  const double* sb = sbar + 19LL * o;
  bool any = false;
  for (int k = 0; k < 19; ++k) any = any || sb[k] != 0.0;
  if (!any) return;
  const MatC mc = mats[P.mat[p]];
  const double V0 = P.vol0[p], m = P.mass[p];
  double fe[3];
  for (int a = 0; a < 3; ++a) fe[a] = P.fext[a] ? P.fext[a][p] : 0.0;
  double gv[3] = {grav[0], grav[1], grav[2]};
  LocalZ z0;
  load_z<D>(P, p, z0);
  double dhdF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dhdu[3] = {0, 0, 0};
  bool ok = true;
  for (int a = 0; a < D && ok; ++a)
    for (int c = 0; c < D && ok; ++c) {
      const double e = 1e-7;
      LocalZ zp = z0, zm = z0;
      zp.dFx[a][c] += e;
      zm.dFx[a][c] -= e;
      LocalOut op, om;
      ok = local_eval<D, T, B>(G, mc, V0, m, gv, fe, U, (const T*)nullptr, psc, sb, zp, op) &&
           local_eval<D, T, B>(G, mc, V0, m, gv, fe, U, (const T*)nullptr, psc, sb, zm, om);
      dhdF[a][c] = (op.h - om.h) / (2.0 * e);
    }
  for (int a = 0; a < D && ok; ++a) {
    const double e = 1e-6 * G.h;
    LocalZ zp = z0, zm = z0;
    zp.dux[a] += e;
    zm.dux[a] -= e;
    LocalOut op, om;
    ok = local_eval<D, T, B>(G, mc, V0, m, gv, fe, U, (const T*)nullptr, psc, sb, zp, op) &&
         local_eval<D, T, B>(G, mc, V0, m, gv, fe, U, (const T*)nullptr, psc, sb, zm, om);
    dhdu[a] = (op.h - om.h) / (2.0 * e);
  }
  if (!ok) {
    atomicOr(err, ERRF_RETURN);
    return;
  }
  Spline1 sp[3];
  for (int a = 0; a < D; ++a) sp[a] = spline1((z0.x[a] - G.o[a]) / G.h);
  if (D == 2) { sp[2].base = 0; sp[2].N[0] = 1.0; sp[2].dN[0] = 0.0; }
  const long long nb = sp[0].base + (long long)G.nx1 * (sp[1].base + (long long)G.ny1 * sp[2].base);
  const int KZ = (D == 3) ? 3 : 1;
  for (int kz = 0; kz < KZ; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        const long long node = nb + kx + (long long)G.nx1 * (ky + (long long)G.ny1 * kz);
        const double w = sp[0].N[kx] * sp[1].N[ky] * sp[2].N[kz];
        double gw[3];
        gw[0] = sp[0].dN[kx] * sp[1].N[ky] * sp[2].N[kz] * G.ih;
        gw[1] = sp[0].N[kx] * sp[1].dN[ky] * sp[2].N[kz] * G.ih;
        gw[2] = sp[0].N[kx] * sp[1].N[ky] * sp[2].dN[kz] * G.ih;
        for (int a = 0; a < D; ++a) {
          double v = dhdu[a] * w;
          for (int c = 0; c < D; ++c) v += dhdF[a][c] * gw[c];
          atomicAdd(&g[node * B + a], v);
        }
      }
}

// Pass B: d(sbar . Phi_p - mu . rhat_p) with respect to the start-of-step
// state (written as the new sbar, caller order) and the parameters (added
// to the gradients).
template <int D, class T, int B>
__global__ void __launch_bounds__(VTPB) k_adj_state_vjp(DevParticles P, DevGrid G, const MatC* __restrict__ mats,
                                                        const double* __restrict__ grav, const double* __restrict__ U,
                                                        const T* __restrict__ mu, double psc,
                                                        const double* __restrict__ sbar, double* sbar_out, double* gE,
                                                        double* gPhi, double* gK, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const int o = P.orig[p];
  const double* sb = sbar + 19LL * o;
  const MatC mc = mats[P.mat[p]];
  const double V0 = P.vol0[p], m = P.mass[p];
  double fe[3];
  for (int a = 0; a < 3; ++a) fe[a] = P.fext[a] ? P.fext[a][p] : 0.0;
  double gv[3] = {grav[0], grav[1], grav[2]};
  LocalZ z0;
  load_z<D>(P, p, z0);
  auto q = [&](const LocalZ& z, bool& ok) -> double {
    LocalOut out;
    ok = ok && local_eval<D, T, B>(G, mc, V0, m, gv, fe, U, mu, psc, sb, z, out);
    return out.h + out.f;
  };
  bool ok = true;
  const int nbe = (D == 2) ? 4 : 6;
  const int ns = D + nbe + 1 + D * D;
  double* so = sbar_out + 19LL * o;
  for (int k = 0; k < 19; ++k) so[k] = 0.0;
  for (int k = 0; k < ns && ok; ++k) {
    LocalZ zp = z0, zm = z0;
    double* vp = state_slot<D>(zp, k);
    double* vm = state_slot<D>(zm, k);
    double e;
    if (k < D) e = 1e-6 * G.h;
    else if (k == D + nbe) e = 1e-6 * fmax(fabs(z0.pc), 1.0);
    else e = 1e-7;
    *vp += e;
    *vm -= e;
    const double d = (q(zp, ok) - q(zm, ok)) / (2.0 * e);
    int dst;
    if (k < D) dst = k;
    else if (k < D + nbe) dst = 3 + (k - D);
    else if (k == D + nbe) dst = 9;
    else {
      const int kk = k - D - nbe - 1;
      dst = 10 + 3 * (kk / D) + (kk % D);
    }
    so[dst] = d;
  }
  if ((gE || gPhi || (gK && B > D && z0.kdt > 0.0)) && ok) {
    double qE, qP, qK;
    ok = local_param_grad<D, T, B>(G, mc, V0, U, mu, psc, sb, z0, qE, qP, qK);
    if (ok) {
      if (gE) gE[o] += qE;
      if (gPhi && mc.model == MODEL_NH_DP) gPhi[o] += qP;
      if (gK && B > D && z0.kdt > 0.0) atomicAdd(&gK[P.mat[p]], qK * mc.dkdt_dk);
    }
  }
  if (!ok) atomicOr(err, ERRF_RETURN);
}

template <int D, class T, int B>
cudaError_t launch_adj_commit_vjp(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* grav,
                                  const double* U, double psc, const double* sbar, double* g, int* err,
                                  cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_adj_commit_vjp<D, T, B><<<(P.np + VTPB - 1) / VTPB, VTPB, 0, st>>>(P, G, mats, grav, U, psc, sbar, g, err);
  return cudaGetLastError();
}
template <int D, class T, int B>
cudaError_t launch_adj_state_vjp(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* grav,
                                 const double* U, const T* mu, double psc, const double* sbar, double* sbar_out,
                                 double* gE, double* gPhi, double* gK, int* err, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_adj_state_vjp<D, T, B><<<(P.np + VTPB - 1) / VTPB, VTPB, 0, st>>>(P, G, mats, grav, U, mu, psc, sbar, sbar_out,
                                                                      gE, gPhi, gK, err);
  return cudaGetLastError();
}

#define MPM_ADJS_INST(D, T, B)                                                                          \
  template cudaError_t launch_adj_commit_vjp<D, T, B>(const DevParticles&, const DevGrid&, const MatC*,  \
                                                      const double*, const double*, double, const double*, \
                                                      double*, int*, cudaStream_t);                        \
  template cudaError_t launch_adj_state_vjp<D, T, B>(const DevParticles&, const DevGrid&, const MatC*,   \
                                                     const double*, const double*, const T*, double,      \
                                                     const double*, double*, double*, double*, double*, int*, \
                                                     cudaStream_t);
MPM_ADJS_INST(2, float, 2)
MPM_ADJS_INST(2, double, 2)
MPM_ADJS_INST(3, float, 3)
MPM_ADJS_INST(3, double, 3)
MPM_ADJS_INST(2, float, 3)
MPM_ADJS_INST(2, double, 3)

}  // namespace mpm
