// Device math of the implicit-MPM Newton step: quadratic B-spline stencil,
// kinematics, Neo-Hookean stress with Drucker-Prager / modified Cam-Clay
// return mapping in principal logarithmic strain, and the hand-derived
// consistent tangent dP/d(dF) (the paper obtains J by reverse-mode AD,
// Sec. 3; here the tangent is written out).  All FP64 unless stated.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mpm {

constexpr int MODEL_NH = 0, MODEL_NH_DP = 1, MODEL_NH_MCC = 2;

// error flag bits raised by kernels
constexpr int ERRF_BOUNDS = 1, ERRF_RETURN = 2, ERRF_NONFINITE = 4, ERRF_DET = 8, ERRF_BARRIER = 16;

// Material constants as used by the kernels.
struct MatC {
  int model;
  double E, nu, rho;
  double phi, psi, coh;    // degrees, degrees, Pa
  double M, lmk;           // Cam-Clay slope, lambda - kappa
  double pc0;
  double dkdt_dk;          // u-p: d(mobility x time step) / d(hydraulic conductivity) = dt / gamma_w
};

struct Lame { double mu, lam; };
__device__ __forceinline__ Lame lame(double E, double nu) {
  Lame l;
  l.mu = E / (2.0 * (1.0 + nu));
  l.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  return l;
}
// Drucker-Prager constants matched to Mohr-Coulomb in plane strain:
// eta = 3 tan(phi)/sqrt(9 + 12 tan^2 phi), xi = 3/sqrt(9 + 12 tan^2 phi).
__device__ __forceinline__ void dp_consts(double phi_deg, double& eta, double& xi) {
  double t = tan(phi_deg * 0.017453292519943295);
  double r = rsqrt(9.0 + 12.0 * t * t);
  eta = 3.0 * t * r;
  xi = 3.0 * r;
}

// ---------------------------------------------------------------- B-spline
// Quadratic B-spline along one axis for a particle at grid coordinate s = x/h:
// base node floor(s - 1/2), weights of base..base+2 and their derivatives
// (with respect to s; divide by h for physical gradients).
struct Spline1 { int base; double N[3], dN[3]; };
// Weights for a particle at offset t = s - base - 1/2 in [0,1) past the base
// node: nodes base, base+1, base+2 sit at xi = s - node = t + 1/2, t - 1/2, t - 3/2.
__device__ __forceinline__ void spline_weights(double t, Spline1& o) {
  double a = 1.0 - t;
  o.N[0] = 0.5 * a * a;
  o.dN[0] = -a;
  double c = t - 0.5;
  o.N[1] = 0.75 - c * c;
  o.dN[1] = -2.0 * c;
  o.N[2] = 0.5 * t * t;
  o.dN[2] = t;
}
__device__ __forceinline__ Spline1 spline1(double s) {
  Spline1 o;
  double fb = floor(s - 0.5);
  o.base = (int)fb;
  spline_weights(s - fb - 0.5, o);
  return o;
}
// Same weights about a given base node (used where the base is known).
__device__ __forceinline__ Spline1 spline1_at(double s, int base) {
  Spline1 o;
  o.base = base;
  spline_weights(s - (double)base - 0.5, o);
  return o;
}

// ---------------------------------------------------------------- 3x3 helpers
__device__ __forceinline__ double det3(const double a[3][3]) {
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
         a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}
__device__ __forceinline__ bool inv3(const double a[3][3], double r[3][3], double& d) {
  d = det3(a);
  if (!(fabs(d) > 0.0)) return false;
  double id = 1.0 / d;
  r[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) * id;
  r[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
  r[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
  r[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) * id;
  r[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
  r[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
  r[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) * id;
  r[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
  r[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  return true;
}

// Solve a 4x4 system with partial pivoting; `nrhs` right-hand sides in b.
template <int NRHS>
__device__ __forceinline__ bool solve4(double a[4][4], double b[4][NRHS]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int p = k;
    double best = fabs(a[k][k]);
#pragma unroll
    for (int i = k + 1; i < 4; ++i) {
      double v = fabs(a[i][k]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best > 0.0)) return false;
    if (p != k) {
#pragma unroll
      for (int j = 0; j < 4; ++j) { double t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t; }
#pragma unroll
      for (int j = 0; j < NRHS; ++j) { double t = b[k][j]; b[k][j] = b[p][j]; b[p][j] = t; }
    }
    double ip = 1.0 / a[k][k];
#pragma unroll
    for (int i = k + 1; i < 4; ++i) {
      double f = a[i][k] * ip;
#pragma unroll
      for (int j = k; j < 4; ++j) a[i][j] -= f * a[k][j];
#pragma unroll
      for (int j = 0; j < NRHS; ++j) b[i][j] -= f * b[k][j];
    }
  }
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    double ip = 1.0 / a[k][k];
#pragma unroll
    for (int j = 0; j < NRHS; ++j) {
      double s = b[k][j];
#pragma unroll
      for (int m = k + 1; m < 4; ++m) s -= a[k][m] * b[m][j];
      b[k][j] = s * ip;
    }
  }
  return true;
}

// ---------------------------------------------------------------- eigen
// Symmetric 3x3 eigen-decomposition.  In 2D plane strain z is always a
// principal direction (b_xz = b_yz = 0): closed form for the in-plane block.
// In 3D: cyclic Jacobi rotations (Golub-Van Loan Sec. 8.5), at most 12 sweeps.
__device__ __forceinline__ void eig_plane(const double b[3][3], double lam[3], double Q[3][3]) {
  double a = b[0][0], d = b[1][1], c = b[0][1];
  double m = 0.5 * (a + d), hd = 0.5 * (a - d);
  double r = sqrt(hd * hd + c * c);
  double l1 = m + r;
  double l2 = (a * d - c * c) / l1;  // avoids the cancellation in m - r
  double th = 0.5 * atan2(2.0 * c, a - d);
  double cs, sn;
  sincos(th, &sn, &cs);
  lam[0] = l1; lam[1] = l2; lam[2] = b[2][2];
  Q[0][0] = cs; Q[0][1] = -sn; Q[0][2] = 0.0;
  Q[1][0] = sn; Q[1][1] = cs;  Q[1][2] = 0.0;
  Q[2][0] = 0.0; Q[2][1] = 0.0; Q[2][2] = 1.0;
}

__device__ __forceinline__ void eig_jacobi(const double b[3][3], double lam[3], double Q[3][3]) {
  double a00 = b[0][0], a11 = b[1][1], a22 = b[2][2];
  double a01 = b[0][1], a02 = b[0][2], a12 = b[1][2];
  double q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double scale = fabs(a00) + fabs(a11) + fabs(a22);
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = a01 * a01 + a02 * a02 + a12 * a12;
    if (!(off > 1e-64 * scale * scale)) break;
    // the three Givens-Jacobi rotations of one sweep, written per pair
#define MPM_JROT(App, Aqq, Apq, Arp, Arq, P, Qc)                                   \
    if (Apq != 0.0) {                                                           \
      double tau = (Aqq - App) / (2.0 * Apq);                                   \
      double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));      \
      double cc = rsqrt(1.0 + t * t), ss = t * cc;                              \
      App -= t * Apq; Aqq += t * Apq; Apq = 0.0;                                \
      double rp = Arp, rq = Arq;                                                \
      Arp = cc * rp - ss * rq; Arq = ss * rp + cc * rq;                         \
      for (int k = 0; k < 3; ++k) {                                             \
        double qp = q[k][P], qq = q[k][Qc];                                     \
        q[k][P] = cc * qp - ss * qq; q[k][Qc] = ss * qp + cc * qq;              \
      }                                                                         \
    }
    MPM_JROT(a00, a11, a01, a02, a12, 0, 1)
    MPM_JROT(a00, a22, a02, a01, a12, 0, 2)
    MPM_JROT(a11, a22, a12, a01, a02, 1, 2)
#undef MPM_JROT
  }
  lam[0] = a00; lam[1] = a11; lam[2] = a22;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = q[i][j];
}

// ---------------------------------------------------------------- constitutive
// Neo-Hookean: tau = mu (b - 1) + lam ln J 1, principal tau_A =
// mu (exp(2 eps_A) - 1) + lam sum eps.

struct ReturnOut {
  double eps[3];
  double deps[3][3];   // d eps_A / d eps^tr_B
  double x3;           // the converged plastic multiplier unknown (x[3])
  double pc;
  int mode;            // 0 elastic, 1 plastic, 2 DP apex
  bool ok;
};

// Drucker-Prager return in principal log strain.  Unknowns
// (eps_1..3, dgamma); equations eps - eps^tr + dgamma (n + etabar/3) = 0 and
// (sqrt(J2) + eta p - xi c)/mu = 0 with n_A = s_A / (2 sqrt(J2)).
// dp_eval gives R and (optionally) its Jacobian J = dR/dx.
__device__ inline void dp_eval(double mu, double lam, double eta, double xi, double etab, double coh,
                               const double etr[3], const double x[4], double R[4], double (*J)[4]) {
  double E[3], tau[3];
  double th = x[0] + x[1] + x[2];
#pragma unroll
  for (int A = 0; A < 3; ++A) { E[A] = exp(2.0 * x[A]); tau[A] = mu * (E[A] - 1.0) + lam * th; }
  double p = (tau[0] + tau[1] + tau[2]) * (1.0 / 3.0);
  double s[3] = {tau[0] - p, tau[1] - p, tau[2] - p};
  double q = sqrt(0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]));
  double iq = 1.0 / q;
  double n[3] = {0.5 * s[0] * iq, 0.5 * s[1] * iq, 0.5 * s[2] * iq};
#pragma unroll
  for (int A = 0; A < 3; ++A) R[A] = x[A] - etr[A] + x[3] * (n[A] + etab * (1.0 / 3.0));
  R[3] = (q + eta * p - xi * coh) / mu;
  if (!J) return;
  // C_AB = d tau_A / d eps_B ; dp_B ; ds_AB = C_AB - dp_B ; dn_A/ds_C = (d_AC - 2 n_A n_C)/(2 q)
  double dpB[3], ds[3][3];
#pragma unroll
  for (int B = 0; B < 3; ++B) dpB[B] = (2.0 * mu * E[B] + 3.0 * lam) * (1.0 / 3.0);
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int B = 0; B < 3; ++B) ds[A][B] = ((A == B) ? 2.0 * mu * E[A] : 0.0) + lam - dpB[B];
#pragma unroll
  for (int A = 0; A < 3; ++A) {
#pragma unroll
    for (int B = 0; B < 3; ++B) {
      double sacc = 0.0;
#pragma unroll
      for (int C = 0; C < 3; ++C) sacc += (((A == C) ? 1.0 : 0.0) - 2.0 * n[A] * n[C]) * ds[C][B];
      J[A][B] = ((A == B) ? 1.0 : 0.0) + x[3] * sacc * 0.5 * iq;
    }
    J[A][3] = n[A] + etab * (1.0 / 3.0);
  }
#pragma unroll
  for (int B = 0; B < 3; ++B) {
    double sacc = 0.0;
#pragma unroll
    for (int C = 0; C < 3; ++C) sacc += n[C] * ds[C][B];
    J[3][B] = (sacc + eta * dpB[B]) / mu;
  }
  J[3][3] = 0.0;
}

// Modified Cam-Clay return (associative) in principal log strain.  Unknowns
// (eps_1..3, y = dgamma |pc_n|); f = q^2/M^2 + p (p - pc),
// pc = pc_n exp(-sum(eps^tr - eps)/(lambda - kappa)).  mcc_eval gives R and,
// optionally, J = dR/dx and Je = dR/d eps^tr.
__device__ inline void mcc_eval(double mu, double lam, double M, double lmk, double pcn, const double etr[3],
                                const double x[4], double R[4], double (*J)[4], double (*Je)[3],
                                double& pc_out) {
  double E[3], tau[3];
  double th = x[0] + x[1] + x[2];
#pragma unroll
  for (int A = 0; A < 3; ++A) { E[A] = exp(2.0 * x[A]); tau[A] = mu * (E[A] - 1.0) + lam * th; }
  double p = (tau[0] + tau[1] + tau[2]) * (1.0 / 3.0);
  double s[3] = {tau[0] - p, tau[1] - p, tau[2] - p};
  double q2 = 1.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  double dvp = (etr[0] - x[0]) + (etr[1] - x[1]) + (etr[2] - x[2]);
  double pc = pcn * exp(-dvp / lmk);
  pc_out = pc;
  double sc = fabs(pcn), isc = 1.0 / sc, iM2 = 1.0 / (M * M);
  double m[3];
#pragma unroll
  for (int A = 0; A < 3; ++A) m[A] = 3.0 * s[A] * iM2 + (2.0 * p - pc) * (1.0 / 3.0);
#pragma unroll
  for (int A = 0; A < 3; ++A) R[A] = x[A] - etr[A] + x[3] * m[A] * isc;
  R[3] = (q2 * iM2 + p * (p - pc)) * isc * isc;
  if (!J) return;
  double dpB[3], ds[3][3];
#pragma unroll
  for (int B = 0; B < 3; ++B) dpB[B] = (2.0 * mu * E[B] + 3.0 * lam) * (1.0 / 3.0);
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int B = 0; B < 3; ++B) ds[A][B] = ((A == B) ? 2.0 * mu * E[A] : 0.0) + lam - dpB[B];
  double dpc = pc / lmk;   // d pc / d eps_B ( = - d pc / d eps^tr_B)
#pragma unroll
  for (int A = 0; A < 3; ++A) {
#pragma unroll
    for (int B = 0; B < 3; ++B) {
      double dm = 3.0 * iM2 * ds[A][B] + (2.0 * dpB[B] - dpc) * (1.0 / 3.0);
      J[A][B] = ((A == B) ? 1.0 : 0.0) + x[3] * isc * dm;
      Je[A][B] = -((A == B) ? 1.0 : 0.0) + x[3] * isc * dpc * (1.0 / 3.0);
    }
    J[A][3] = m[A] * isc;
  }
#pragma unroll
  for (int B = 0; B < 3; ++B) {
    double dq2 = 3.0 * (s[0] * ds[0][B] + s[1] * ds[1][B] + s[2] * ds[2][B]);
    J[3][B] = (dq2 * iM2 + dpB[B] * (2.0 * p - pc) - p * dpc) * isc * isc;
    Je[3][B] = p * dpc * isc * isc;
  }
  J[3][3] = 0.0;
}

// Safeguarded local Newton shared by both models: from the trial state, a
// Newton step on R(x) = 0, halved while it does not reduce ||R|| (accepting
// any step once ||R|| is at rounding level); converged when a full step is
// below 1e-13 relative.  Then dx/d eps^tr = -J^-1 dR/d eps^tr at the root.
template <int MODEL>
__device__ inline void local_newton(double mu, double lam, double eta, double xi, double etab, double coh,
                                    double M, double lmk, double pcn, const double etr[3], ReturnOut& o) {
  double x[4] = {etr[0], etr[1], etr[2], 0.0};
  double R[4], J[4][4], Je[4][3], pc = pcn;
  bool conv = false;
  for (int it = 0; it < 40 && !conv; ++it) {
    if (MODEL == MODEL_NH_DP) dp_eval(mu, lam, eta, xi, etab, coh, etr, x, R, J);
    else mcc_eval(mu, lam, M, lmk, pcn, etr, x, R, J, Je, pc);
    double n0 = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + R[3] * R[3]);
    double b[4][1] = {{R[0]}, {R[1]}, {R[2]}, {R[3]}};
    if (!solve4<1>(J, b)) { o.ok = false; return; }
    double alpha = 1.0;
    for (int ls = 0; ls < 30; ++ls) {
      double xt[4], Rt[4], pct;
#pragma unroll
      for (int i = 0; i < 4; ++i) xt[i] = x[i] - alpha * b[i][0];
      if (MODEL == MODEL_NH_DP) dp_eval(mu, lam, eta, xi, etab, coh, etr, xt, Rt, nullptr);
      else mcc_eval(mu, lam, M, lmk, pcn, etr, xt, Rt, nullptr, nullptr, pct);
      double n1 = sqrt(Rt[0] * Rt[0] + Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3]);
      if (isfinite(n1) && (n1 <= (1.0 - 1e-4 * alpha) * n0 || n1 <= 1e-12)) break;
      alpha *= 0.5;
    }
    double big = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] -= alpha * b[i][0];
      big = fmax(big, fabs(alpha * b[i][0]) / (1.0 + fabs(x[i])));
    }
    if (!(big < 1e300)) { o.ok = false; return; }
    conv = (alpha == 1.0) && (big <= 1e-13);
  }
  if (!conv) { o.ok = false; return; }
  double rhs[4][3];
  if (MODEL == MODEL_NH_DP) {
    dp_eval(mu, lam, eta, xi, etab, coh, etr, x, R, J);
    // dR/d eps^tr = [-I; 0]
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) rhs[i][j] = (i == j) ? 1.0 : 0.0;
  } else {
    mcc_eval(mu, lam, M, lmk, pcn, etr, x, R, J, Je, pc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) rhs[i][j] = -Je[i][j];
  }
  if (!solve4<3>(J, rhs)) { o.ok = false; return; }
  o.x3 = x[3];
#pragma unroll
  for (int A = 0; A < 3; ++A) {
    o.eps[A] = x[A];
#pragma unroll
    for (int B = 0; B < 3; ++B) o.deps[A][B] = rhs[A][B];
  }
  o.pc = (MODEL == MODEL_NH_MCC) ? pc : pcn;
}

__device__ inline void dp_return(double mu, double lam, double eta, double xi, double etab,
                                 double coh, const double etr[3], ReturnOut& o) {
  o.ok = true;
  o.mode = 1;
  // apex: on the trial volume the isotropic state has the smallest pressure;
  // if it still violates f the return goes to tau = (xi c / eta) 1.
  if (eta > 0.0) {
    double th = etr[0] + etr[1] + etr[2];
    double e = th * (1.0 / 3.0);
    double piso = mu * expm1(2.0 * e) + lam * th;
    if (eta * piso - xi * coh >= 0.0) {
      double pa = xi * coh / eta;
      int it = 0;
      for (; it < 60; ++it) {
        double ex = exp(2.0 * e);
        double g = mu * (ex - 1.0) + 3.0 * lam * e - pa;
        double de = g / (2.0 * mu * ex + 3.0 * lam);
        e -= de;
        if (fabs(de) <= 1e-16 * (1.0 + fabs(e))) break;
      }
      o.ok = it < 60;
      o.x3 = 0.0;
#pragma unroll
      for (int A = 0; A < 3; ++A) {
        o.eps[A] = e;
#pragma unroll
        for (int B = 0; B < 3; ++B) o.deps[A][B] = 0.0;
      }
      o.mode = 2;
      return;
    }
  }
  local_newton<MODEL_NH_DP>(mu, lam, eta, xi, etab, coh, 0.0, 1.0, 0.0, etr, o);
}

__device__ inline void mcc_return(double mu, double lam, double M, double lmk, double pcn,
                                  const double etr[3], ReturnOut& o) {
  o.ok = true;
  o.mode = 1;
  local_newton<MODEL_NH_MCC>(mu, lam, 0.0, 0.0, 0.0, 0.0, M, lmk, pcn, etr, o);
}

// Per-particle constitutive state for one iterate.
struct PState {
  double F[3][3];      // dF (increment of the deformation gradient)
  double Fi[3][3];     // dF^-1
  double bn[3][3];     // elastic left Cauchy-Green at the start of the step
  double b[3][3];      // trial b = dF bn dF^T
  double tau[3][3];    // Kirchhoff stress
  double P[3][3];      // V0 tau dF^-T
  double benew[3][3];  // elastic left Cauchy-Green after the return
  double pc;           // hardening variable after the return
  int mode;            // 0 elastic, 1 plastic, 2 apex
  // principal data of a plastic particle (for the tangent)
  double lam[3], Q[3][3], tp[3], D[3][3];
  double mu, lamL;
  double eps[3], x3;   // converged principal log strains and multiplier unknown
};

// Constitutive update of one particle given dF, bn, material; fills
// tau, P and the principal data.  Returns an ERRF_* bit set (0 = ok).
template <int DIM>
__device__ inline int constitutive(const MatC& mc, double E_p, double phi_p, double pcn, double V0,
                                   PState& st) {
  Lame L = lame(E_p, mc.nu);
  st.mu = L.mu;
  st.lamL = L.lam;
  double detF;
  if (!inv3(st.F, st.Fi, detF) || !(detF > 0.0)) return ERRF_DET;
  // trial b = dF bn dF^T
  double t1[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      t1[i][j] = st.F[i][0] * st.bn[0][j] + st.F[i][1] * st.bn[1][j] + st.F[i][2] * st.bn[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      st.b[i][j] = t1[i][0] * st.F[j][0] + t1[i][1] * st.F[j][1] + t1[i][2] * st.F[j][2];
  double detb = det3(st.b);
  if (!(detb > 0.0)) return ERRF_DET;
  double lnJ = 0.5 * log(detb);
  // elastic trial Kirchhoff stress, written without eigenvectors
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      st.tau[i][j] = L.mu * (st.b[i][j] - ((i == j) ? 1.0 : 0.0)) + ((i == j) ? L.lam * lnJ : 0.0);
  st.mode = 0;
  st.pc = pcn;
  bool plastic = false;
  double eta = 0, xi = 0, etab = 0;
  if (mc.model != MODEL_NH) {
    double p = (st.tau[0][0] + st.tau[1][1] + st.tau[2][2]) * (1.0 / 3.0);
    double s00 = st.tau[0][0] - p, s11 = st.tau[1][1] - p, s22 = st.tau[2][2] - p;
    double ss = s00 * s00 + s11 * s11 + s22 * s22 +
                2.0 * (st.tau[0][1] * st.tau[0][1] + st.tau[1][2] * st.tau[1][2] + st.tau[0][2] * st.tau[0][2]);
    double f, ftol;
    if (mc.model == MODEL_NH_DP) {
      dp_consts(phi_p, eta, xi);
      double xb;
      dp_consts(mc.psi, etab, xb);
      f = sqrt(0.5 * ss) + eta * p - xi * mc.coh;
      ftol = 1e-10 * L.mu;
    } else {
      f = 1.5 * ss / (mc.M * mc.M) + p * (p - pcn);
      ftol = 1e-10 * L.mu * fabs(pcn);
    }
    // within a rounding-level tolerance of the surface the state is elastic
    // (a state committed on the surface, re-evaluated at zero increment)
    plastic = f > ftol;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) st.benew[i][j] = st.b[i][j];
  if (plastic) {
    if (DIM == 2) eig_plane(st.b, st.lam, st.Q);
    else eig_jacobi(st.b, st.lam, st.Q);
    if (!(st.lam[0] > 0.0 && st.lam[1] > 0.0 && st.lam[2] > 0.0)) return ERRF_DET;
    double etr[3] = {0.5 * log(st.lam[0]), 0.5 * log(st.lam[1]), 0.5 * log(st.lam[2])};
    ReturnOut ro;
    if (mc.model == MODEL_NH_DP) dp_return(L.mu, L.lam, eta, xi, etab, mc.coh, etr, ro);
    else {
      mcc_return(L.mu, L.lam, mc.M, mc.lmk, pcn, etr, ro);
    }
    if (!ro.ok) return ERRF_RETURN;
    st.mode = ro.mode;
    st.x3 = ro.x3;
#pragma unroll
    for (int A = 0; A < 3; ++A) st.eps[A] = ro.eps[A];
    if (mc.model == MODEL_NH_MCC) st.pc = ro.pc;
    double th = ro.eps[0] + ro.eps[1] + ro.eps[2];
    double Ex[3];
#pragma unroll
    for (int A = 0; A < 3; ++A) {
      Ex[A] = exp(2.0 * ro.eps[A]);
      st.tp[A] = L.mu * (Ex[A] - 1.0) + L.lam * th;
    }
    // principal tangent D_AB = d tau_A / d lam_B
#pragma unroll
    for (int A = 0; A < 3; ++A)
#pragma unroll
      for (int B = 0; B < 3; ++B) {
        double sacc = 0.0;
#pragma unroll
        for (int C = 0; C < 3; ++C)
          sacc += (((A == C) ? 2.0 * L.mu * Ex[A] : 0.0) + L.lam) * ro.deps[C][B];
        st.D[A][B] = sacc / (2.0 * st.lam[B]);
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double a = 0.0, c = 0.0;
#pragma unroll
        for (int A = 0; A < 3; ++A) {
          double qq = st.Q[i][A] * st.Q[j][A];
          a += st.tp[A] * qq;
          c += Ex[A] * qq;
        }
        st.tau[i][j] = a;
        st.benew[i][j] = c;
      }
  }
  // P = V0 tau dF^-T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      st.P[i][j] = V0 * (st.tau[i][0] * st.Fi[j][0] + st.tau[i][1] * st.Fi[j][1] + st.tau[i][2] * st.Fi[j][2]);
  return 0;
}

// Derivatives of the Kirchhoff stress of `constitutive` (same dF and
// start-of-step state, already evaluated into st) with respect to the
// particle's Young's modulus E and friction angle phi (degrees):
//  * E enters only through mu = E m and lam = E l, so at fixed principal log
//    strains tau is proportional to E: elastic d tau / dE = tau / E;
//  * phi enters only through the Drucker-Prager constants eta(phi), xi(phi);
//  * on a return the converged local unknowns x = (eps_1..3, x3) solve
//    R(x; theta) = 0 (dp_eval / mcc_eval), hence dx/dtheta = -J^-1 dR/dtheta
//    with J = dR/dx at the root, and d tau_A = sum_B C_AB d eps_B +
//    (tau_A / E) dE with C_AB = d tau_A / d eps_B; the principal directions
//    (those of the trial b) do not depend on E or phi;
//  * the DP apex state tau = (xi c / eta) 1 depends on phi alone.
// With t = tan phi and S = sqrt(9 + 12 t^2): d eta/dt = 27/S^3,
// d xi/dt = -36 t/S^3, d(xi/eta)/dt = -1/t^2, dt/dphi = (1 + t^2) pi/180.
// `deps` (may be null) receives the principal log-strain derivatives
// d eps_A / dE and d eps_A / dphi (zero on the elastic branch, where eps is
// the trial strain; at the apex, from mu (e^{2e} - 1) + 3 lam e = xi c / eta).
// Returns false if the local system is singular.
template <int DIM>
__device__ inline bool param_dtau(const MatC& mc, double E_p, double phi_p, double pcn, const PState& st,
                                  double dtE[3][3], double dtP[3][3], double (*deps)[2] = nullptr) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dtE[i][j] = (st.mode == 0) ? st.tau[i][j] / E_p : 0.0;
      dtP[i][j] = 0.0;
    }
  if (deps)
#pragma unroll
    for (int A = 0; A < 3; ++A) deps[A][0] = deps[A][1] = 0.0;
  if (st.mode == 0) return true;
  const double deg = 0.017453292519943295;
  if (st.mode == 2) {
    // apex (Drucker-Prager only, eta > 0)
    const double t = tan(phi_p * deg);
    const double d = -mc.coh / (t * t) * (1.0 + t * t) * deg;
#pragma unroll
    for (int i = 0; i < 3; ++i) dtP[i][i] = d;
    if (deps) {
      const double ex = exp(2.0 * st.eps[0]);
      const double ge = 2.0 * st.mu * ex + 3.0 * st.lamL;
      const double pa = st.tp[0];
#pragma unroll
      for (int A = 0; A < 3; ++A) {
        deps[A][0] = -(pa / E_p) / ge;
        deps[A][1] = d / ge;
      }
    }
    return true;
  }
  const double mu = st.mu, lam = st.lamL;
  const double etr[3] = {0.5 * log(st.lam[0]), 0.5 * log(st.lam[1]), 0.5 * log(st.lam[2])};
  const double x[4] = {st.eps[0], st.eps[1], st.eps[2], st.x3};
  double R[4], J[4][4], b[4][2];
  const double p = (st.tp[0] + st.tp[1] + st.tp[2]) * (1.0 / 3.0);
  if (mc.model == MODEL_NH_DP) {
    double eta, xi, etab, xb;
    dp_consts(phi_p, eta, xi);
    dp_consts(mc.psi, etab, xb);
    dp_eval(mu, lam, eta, xi, etab, mc.coh, etr, x, R, J);
    const double t = tan(phi_p * deg);
    const double S = sqrt(9.0 + 12.0 * t * t), iS3 = 1.0 / (S * S * S);
    const double dt = (1.0 + t * t) * deg;
    const double deta = 27.0 * iS3 * dt, dxi = -36.0 * t * iS3 * dt;
#pragma unroll
    for (int A = 0; A < 3; ++A) { b[A][0] = 0.0; b[A][1] = 0.0; }
    b[3][0] = -(xi * mc.coh) / (E_p * mu);
    b[3][1] = -(deta * p - dxi * mc.coh) / mu;
  } else {
    double Je[4][3], pc;
    mcc_eval(mu, lam, mc.M, mc.lmk, pcn, etr, x, R, J, Je, pc);
    const double iM2 = 1.0 / (mc.M * mc.M), isc = 1.0 / fabs(pcn);
    double q2 = 0.0;
#pragma unroll
    for (int A = 0; A < 3; ++A) q2 += 1.5 * (st.tp[A] - p) * (st.tp[A] - p);
#pragma unroll
    for (int A = 0; A < 3; ++A) {
      // m_A + pc/3 = 3 s_A / M^2 + 2p/3 is proportional to E
      const double mA = 3.0 * (st.tp[A] - p) * iM2 + 2.0 * p * (1.0 / 3.0);
      b[A][0] = -x[3] * isc * mA / E_p;
      b[A][1] = 0.0;
    }
    b[3][0] = -(2.0 * q2 * iM2 + 2.0 * p * p - p * pc) * isc * isc / E_p;
    b[3][1] = 0.0;
  }
  if (!solve4<2>(J, b)) return false;
  if (deps)
#pragma unroll
    for (int A = 0; A < 3; ++A) {
      deps[A][0] = b[A][0];
      deps[A][1] = b[A][1];
    }
  double dA[3][2];
#pragma unroll
  for (int A = 0; A < 3; ++A) {
    double sE = st.tp[A] / E_p, sP = 0.0;
#pragma unroll
    for (int B = 0; B < 3; ++B) {
      const double C = ((A == B) ? 2.0 * mu * exp(2.0 * x[A]) : 0.0) + lam;
      sE += C * b[B][0];
      sP += C * b[B][1];
    }
    dA[A][0] = sE;
    dA[A][1] = sP;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double e = 0.0, f = 0.0;
#pragma unroll
      for (int A = 0; A < 3; ++A) {
        const double qq = st.Q[i][A] * st.Q[j][A];
        e += dA[A][0] * qq;
        f += dA[A][1] * qq;
      }
      dtE[i][j] = e;
      dtP[i][j] = f;
    }
  return true;
}

// Consistent tangent A[a][c][b][e] = dP_ac / d dF_be for a,c,b,e < DIM,
// written to out[(((a*DIM + c)*DIM + b)*DIM + e) * stride].
//  Elastic (Neo-Hookean, closed form):
//    A = V0 mu d_ab bn_ce + (V0 mu (dF bn)_ae - P_ae) dF^-1_cb + V0 lam dF^-1_ca dF^-1_eb
//  Plastic (spectral): d tau = Q dtau' Q^T with, for the direction E_be,
//    db'_AB = Q_bA U_Be + U_Ae Q_bB,  U = Q^T dF bn,
//    dtau'_AA = sum_B D_AB db'_BB,  dtau'_AB = theta_AB db'_AB (A != B),
//    theta_AB = (tau_A - tau_B)/(lam_A - lam_B) (limit D_AA - D_AB if equal);
//    A = V0 (dtau dF^-T)_ac - P_ae dF^-1_cb.
template <int DIM, class T>
__device__ inline void tangent(const PState& st, double V0, T* out, long long stride) {
  if (st.mode == 0) {
    double Fb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Fb[i][j] = st.F[i][0] * st.bn[0][j] + st.F[i][1] * st.bn[1][j] + st.F[i][2] * st.bn[2][j];
    const double vmu = V0 * st.mu, vla = V0 * st.lamL;
    if constexpr (sizeof(T) == 4) {
      // FP32 Jacobian: the three factors are formed in FP64 (the first one
      // holds the difference V0 mu dF bn - P) and rounded once; the 81
      // products and sums, all of the scale of mu, then run in FP32
      float G[3][3], X[3][3], Mb[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          G[i][j] = (float)(vmu * Fb[i][j] - st.P[i][j]);
          X[i][j] = (float)st.Fi[i][j];
          Mb[i][j] = (float)(vmu * st.bn[i][j]);
        }
      const float vlf = (float)vla;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int b = 0; b < DIM; ++b)
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
              float v = G[a][e] * X[c][b] + vlf * X[c][a] * X[e][b];
              if (a == b) v += Mb[c][e];
              out[(long long)(((a * DIM + c) * DIM + b) * DIM + e) * stride] = (T)v;
            }
      return;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int b = 0; b < DIM; ++b)
#pragma unroll
          for (int e = 0; e < DIM; ++e) {
            double v = (vmu * Fb[a][e] - st.P[a][e]) * st.Fi[c][b] + vla * st.Fi[c][a] * st.Fi[e][b];
            if (a == b) v += vmu * st.bn[c][e];
            out[(long long)(((a * DIM + c) * DIM + b) * DIM + e) * stride] = (T)v;
          }
    return;
  }
  // plastic / apex: spectral form
  double U[3][3], Fb[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Fb[i][j] = st.F[i][0] * st.bn[0][j] + st.F[i][1] * st.bn[1][j] + st.F[i][2] * st.bn[2][j];
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int e = 0; e < 3; ++e) U[A][e] = st.Q[0][A] * Fb[0][e] + st.Q[1][A] * Fb[1][e] + st.Q[2][A] * Fb[2][e];
  double th[3][3];
  double lmax = fmax(fabs(st.lam[0]), fmax(fabs(st.lam[1]), fabs(st.lam[2])));
#pragma unroll
  for (int A = 0; A < 3; ++A)
#pragma unroll
    for (int B = 0; B < 3; ++B) {
      if (A == B) { th[A][B] = 0.0; continue; }
      double gap = st.lam[A] - st.lam[B];
      th[A][B] = (fabs(gap) > 1e-8 * lmax) ? (st.tp[A] - st.tp[B]) / gap
                                           : 0.5 * ((st.D[A][A] - st.D[A][B]) + (st.D[B][B] - st.D[B][A]));
    }
#pragma unroll
  for (int b = 0; b < DIM; ++b)
#pragma unroll
    for (int e = 0; e < DIM; ++e) {
      double dbp[3][3], dtp[3][3];
#pragma unroll
      for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) dbp[A][B] = st.Q[b][A] * U[B][e] + U[A][e] * st.Q[b][B];
#pragma unroll
      for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) {
          if (A == B) dtp[A][A] = st.D[A][0] * dbp[0][0] + st.D[A][1] * dbp[1][1] + st.D[A][2] * dbp[2][2];
          else dtp[A][B] = th[A][B] * dbp[A][B];
        }
      // dtau = Q dtp Q^T (only rows a < DIM needed), then (dtau dF^-T)_ac
      double QdT[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int B = 0; B < 3; ++B) QdT[i][B] = st.Q[i][0] * dtp[0][B] + st.Q[i][1] * dtp[1][B] + st.Q[i][2] * dtp[2][B];
      double dtau[3][3];
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) dtau[i][k] = QdT[i][0] * st.Q[k][0] + QdT[i][1] * st.Q[k][1] + QdT[i][2] * st.Q[k][2];
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          double v = V0 * (dtau[a][0] * st.Fi[c][0] + dtau[a][1] * st.Fi[c][1] + dtau[a][2] * st.Fi[c][2])
                     - st.P[a][e] * st.Fi[c][b];
          out[(long long)(((a * DIM + c) * DIM + b) * DIM + e) * stride] = (T)v;
        }
    }
}

}  // namespace mpm
