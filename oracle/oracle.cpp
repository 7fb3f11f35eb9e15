// Plain FP64 CPU oracle for one implicit-MPM Newton step (GeoWarp,
// Zhao, Li, Jiang & Choo, arXiv 2507.09435).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
// reference that the CUDA path is checked against.  Only tests/,
// __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
// load it.  It shares no code, header or table with the CUDA library.
// Compiled with -O2 -ffp-contract=off (no FMA contraction).
//
// What it computes (paper Sec. 2.2, "Implicit MPM discretization"):
//   * quadratic B-spline weights w_ip and gradients grad w_ip (the paper names
//     the family, Table 1; the formula is the textbook one);
//   * G2P of the nodal increment: dF_p = 1 + sum_i du_i (x) grad w_ip;
//   * the constitutive update: Neo-Hookean elasticity, optionally followed by
//     a Drucker-Prager or modified Cam-Clay return map in principal
//     logarithmic strain (the paper defers the models to textbooks, Sec. 2.1);
//   * the internal force f_int,i = sum_p V0_p tau_p dF_p^-T grad w_ip (the
//     paper's f_int,p = (sym grad w_p)^T : sigma_p V_p with sigma V = tau V0)
//     and the external force f_ext,i = sum_p w_ip (m_p g + f_p): gravity plus
//     the force a particle carries (the traction term, read as a traction
//     times the particle's share of the loaded face);
//   * the residual r = f_int - f_ext (paper Eq. for r(u^{n+1}));
//   * the Jacobian J = dr/du (paper Eq. for J^{n+1,k}) as its exact
//     derivative: the per-particle tangent A_p = dP_p/d(dF_p) obtained by
//     forward-mode dual numbers through the principal-space return map plus
//     the implicit-function theorem, and the Daleckii-Krein rule for the
//     spectral (eigenvector) part;
//   * the commit of the particle state after convergence (Sec. 2.2 stage 4);
//   * the coupled u-p residual, its exact Jacobian and commit (Sec. 2.2,
//     remark on poromechanics; the equations are a stated reading).
// The Newton loop and the sparse linear solve live in mpm_oracle.py.
//
// Readings of points the paper leaves open are stated where they are used.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

// ------------------------------------------------------------------------
// forward-mode dual number (one direction)
// ------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
using std::exp;
using std::log;
using std::sqrt;

// ------------------------------------------------------------------------
// small dense helpers
// ------------------------------------------------------------------------
typedef double M3[3][3];

void matmul(const M3 a, const M3 b, M3 c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      c[i][j] = s;
    }
}
void transpose(const M3 a, M3 t) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t[i][j] = a[j][i];
}
double det3(const M3 a) {
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
         a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}
// inverse by the adjugate
int inv3(const M3 a, M3 r) {
  double d = det3(a);
  if (!(std::fabs(d) > 0) || !std::isfinite(d)) return -1;
  r[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / d;
  r[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / d;
  r[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / d;
  r[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / d;
  r[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / d;
  r[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / d;
  r[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / d;
  r[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / d;
  r[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / d;
  return 0;
}
// Gaussian elimination with partial pivoting, n <= 4, solves a x = b in place
int solve_small(int n, double a[4][4], double b[4]) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[i][k]) > std::fabs(a[p][k])) p = i;
    if (!(std::fabs(a[p][k]) > 0)) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(a[k][j], a[p][j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = a[i][k] / a[k][k];
      for (int j = k; j < n; ++j) a[i][j] -= f * a[k][j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= a[k][j] * b[j];
    b[k] = s / a[k][k];
  }
  return 0;
}

// Symmetric eigen-decomposition by the cyclic Jacobi method (Golub & Van
// Loan, "Matrix Computations", Sec. 8.5: the symmetric 2x2 Schur step applied
// to every off-diagonal pair in turn).  a = Q diag(lam) Q^T, eigenvectors are
// the columns of Q.
void jacobi_eig(const M3 a_in, double lam[3], M3 Q) {
  M3 a;
  std::memcpy(a, a_in, sizeof(M3));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Q[i][j] = (i == j) ? 1.0 : 0.0;
  double scale = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) scale = std::max(scale, std::fabs(a[i][j]));
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    if (off <= 1e-60 * scale * scale || off == 0.0) break;
    static const int P[3] = {0, 0, 1}, Qx[3] = {1, 2, 2};
    for (int r = 0; r < 3; ++r) {
      int p = P[r], q = Qx[r];
      if (a[p][q] == 0.0) continue;
      double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
      double t = (tau >= 0) ? 1.0 / (tau + std::sqrt(1.0 + tau * tau))
                            : -1.0 / (-tau + std::sqrt(1.0 + tau * tau));
      double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
      // a <- J^T a J with J the rotation in the (p,q) plane
      for (int k = 0; k < 3; ++k) {
        double akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        double apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double qkp = Q[k][p], qkq = Q[k][q];
        Q[k][p] = c * qkp - s * qkq;
        Q[k][q] = s * qkp + c * qkq;
      }
    }
  }
  for (int i = 0; i < 3; ++i) lam[i] = a[i][i];
}

// ------------------------------------------------------------------------
// quadratic B-spline (textbook form; the paper names the family in Table 1)
// ------------------------------------------------------------------------
double bspline_N(double xi) {
  double a = std::fabs(xi);
  if (a < 0.5) return 0.75 - xi * xi;
  if (a < 1.5) { double t = 1.5 - a; return 0.5 * t * t; }
  return 0.0;
}
double bspline_dN(double xi) {
  double a = std::fabs(xi);
  if (a < 0.5) return -2.0 * xi;
  if (a < 1.5) { double t = 1.5 - a; return xi > 0 ? -t : t; }
  return 0.0;
}

struct Grid {
  int dim;
  int n[3];
  double h;
  double o[3];
  long nnode() const {
    long c = 1;
    for (int a = 0; a < dim; ++a) c *= n[a] + 1;
    return c;
  }
  long node(int ix, int iy, int iz) const {
    return ix + (long)(n[0] + 1) * (iy + (long)(n[1] + 1) * iz);
  }
};

// The 3^dim nodes influencing a particle: base node floor(x/h - 1/2) per axis
// and the two after it.  Returns -1 when the support leaves the grid.
struct Stencil {
  int cnt;
  long node[27];
  double w[27];
  double g[27][3];
};
int make_stencil(const Grid& G, const double* xp, Stencil& S) {
  int base[3] = {0, 0, 0};
  double Nv[3][3], dNv[3][3];
  for (int a = 0; a < 3; ++a) {
    if (a < G.dim) {
      double s = (xp[a] - G.o[a]) / G.h;
      base[a] = (int)std::floor(s - 0.5);
      if (base[a] < 0 || base[a] + 2 > G.n[a]) return -1;
      for (int k = 0; k < 3; ++k) {
        double xi = s - (double)(base[a] + k);
        Nv[a][k] = bspline_N(xi);
        dNv[a][k] = bspline_dN(xi) / G.h;
      }
    } else {
      for (int k = 0; k < 3; ++k) { Nv[a][k] = (k == 0) ? 1.0 : 0.0; dNv[a][k] = 0.0; }
    }
  }
  int kz_n = (G.dim == 3) ? 3 : 1;
  S.cnt = 0;
  for (int kz = 0; kz < kz_n; ++kz)
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx) {
        int l = S.cnt++;
        S.node[l] = G.node(base[0] + kx, base[1] + ky, base[2] + kz);
        S.w[l] = Nv[0][kx] * Nv[1][ky] * Nv[2][kz];
        S.g[l][0] = dNv[0][kx] * Nv[1][ky] * Nv[2][kz];
        S.g[l][1] = Nv[0][kx] * dNv[1][ky] * Nv[2][kz];
        S.g[l][2] = Nv[0][kx] * Nv[1][ky] * dNv[2][kz];
      }
  return 0;
}

// ------------------------------------------------------------------------
// materials
// ------------------------------------------------------------------------
enum { MODEL_NH = 0, MODEL_NH_DP = 1, MODEL_NH_MCC = 2 };

struct Mat {
  int model;
  double mu, lam;           // Lame constants of the Neo-Hookean part
  double eta, xi, etabar;   // Drucker-Prager friction, cohesion, dilation factors
  double coh;               // cohesion
  double M, lmk;            // Cam-Clay slope, lambda - kappa
};

// params: E, nu, phi (deg), psi (deg), c, M, lambda_cc, kappa_cc
Mat make_mat(int model, const double* p) {
  Mat m;
  m.model = model;
  double E = p[0], nu = p[1];
  m.mu = E / (2.0 * (1.0 + nu));
  m.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  // Drucker-Prager matched to Mohr-Coulomb in plane strain (reading: the
  // textbook plane-strain match, eta = 3 tan(phi)/sqrt(9 + 12 tan^2 phi),
  // xi = 3/sqrt(9 + 12 tan^2 phi), the same form with psi for the potential).
  const double d2r = 3.14159265358979323846 / 180.0;
  double tp = std::tan(p[2] * d2r), ts = std::tan(p[3] * d2r);
  m.eta = 3.0 * tp / std::sqrt(9.0 + 12.0 * tp * tp);
  m.xi = 3.0 / std::sqrt(9.0 + 12.0 * tp * tp);
  m.etabar = 3.0 * ts / std::sqrt(9.0 + 12.0 * ts * ts);
  m.coh = p[4];
  m.M = p[5];
  m.lmk = p[6] - p[7];
  return m;
}

// Neo-Hookean Kirchhoff stress in principal log strain (reading of the
// paper's unnamed Neo-Hookean law: psi = mu/2 (tr b - 3) - mu ln J +
// lam/2 (ln J)^2, so tau = mu (b - 1) + lam ln J 1, whose principal values
// are tau_A = mu (exp(2 eps_A) - 1) + lam sum_B eps_B).
template <class T>
void nh_principal(const T e[3], const Mat& m, T tau[3]) {
  T th = e[0] + e[1] + e[2];
  for (int A = 0; A < 3; ++A) tau[A] = T(m.mu) * (exp(e[A] * T(2.0)) - T(1.0)) + T(m.lam) * th;
}

// Drucker-Prager return-map equations in principal space, unknowns
// x = (eps_1, eps_2, eps_3, dgamma):
//   eps_A - eps_A^tr + dgamma dg/dtau_A = 0,   f(tau(eps)) / mu = 0,
// f = sqrt(J2) + eta p - xi c,  g = sqrt(J2) + etabar p,  p = tr(tau)/3.
template <class T>
void dp_res(const T x[4], const T etr[3], const Mat& m, T R[4]) {
  T tau[3];
  nh_principal(x, m, tau);
  T p = (tau[0] + tau[1] + tau[2]) / T(3.0);
  T s[3] = {tau[0] - p, tau[1] - p, tau[2] - p};
  T rJ2 = sqrt((s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) * T(0.5));
  for (int A = 0; A < 3; ++A)
    R[A] = x[A] - etr[A] + x[3] * (s[A] / (rJ2 * T(2.0)) + T(m.etabar / 3.0));
  R[3] = (rJ2 + T(m.eta) * p - T(m.xi * m.coh)) / T(m.mu);
}

// Modified Cam-Clay return-map equations (associative), unknowns
// x = (eps_1..3, dgamma*|pc_n|):
//   f = q^2/M^2 + p (p - pc),  q^2 = 3 J2,
//   pc = pc_n exp(-dev_p / (lambda - kappa)),  dev_p = sum_A (eps_A^tr - eps_A),
// with compression negative, so compaction (dev_p < 0) makes pc more negative.
template <class T>
void mcc_res(const T x[4], const T etr[3], const Mat& m, double pcn, T R[4]) {
  T tau[3];
  nh_principal(x, m, tau);
  T p = (tau[0] + tau[1] + tau[2]) / T(3.0);
  T s[3] = {tau[0] - p, tau[1] - p, tau[2] - p};
  T q2 = (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) * T(1.5);
  T dvp = (etr[0] - x[0]) + (etr[1] - x[1]) + (etr[2] - x[2]);
  T pc = exp(-dvp / T(m.lmk)) * T(pcn);
  double sc = std::fabs(pcn), M2 = m.M * m.M;
  for (int A = 0; A < 3; ++A)
    R[A] = x[A] - etr[A] + x[3] * (s[A] * T(3.0 / M2) + (p * T(2.0) - pc) / T(3.0)) / T(sc);
  R[3] = (q2 / T(M2) + p * (p - pc)) / T(sc * sc);
}

template <class T>
void model_res(const T x[4], const T etr[3], const Mat& m, double pcn, T R[4]) {
  if (m.model == MODEL_NH_DP) dp_res(x, etr, m, R);
  else mcc_res(x, etr, m, pcn, R);
}

// dR/dx (4x4) and dR/d eps^tr (4x3) by forward-mode dual numbers
void res_jacobians(const double x[4], const double etr[3], const Mat& m, double pcn,
                   double Jx[4][4], double Je[4][3]) {
  for (int j = 0; j < 4; ++j) {
    Dual xd[4], ed[3], R[4];
    for (int i = 0; i < 4; ++i) xd[i] = Dual(x[i], i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i) ed[i] = Dual(etr[i], 0.0);
    model_res(xd, ed, m, pcn, R);
    for (int i = 0; i < 4; ++i) Jx[i][j] = R[i].d;
  }
  for (int j = 0; j < 3; ++j) {
    Dual xd[4], ed[3], R[4];
    for (int i = 0; i < 4; ++i) xd[i] = Dual(x[i], 0.0);
    for (int i = 0; i < 3; ++i) ed[i] = Dual(etr[i], i == j ? 1.0 : 0.0);
    model_res(xd, ed, m, pcn, R);
    for (int i = 0; i < 4; ++i) Je[i][j] = R[i].d;
  }
}

// Principal-space return map.  Input: trial principal log strains etr.
// Output: eps (3), pc_new, mode (0 elastic, 1 plastic, 2 DP apex) and
// deps[A][B] = d eps_A / d etr_B.  Returns 0 or -2 when the local Newton
// does not converge.
int return_map(const Mat& m, const double etr[3], double pcn, double eps[3],
               double* pc_new, int* mode, double deps[3][3], double* dgam_out) {
  for (int A = 0; A < 3; ++A) {
    eps[A] = etr[A];
    for (int B = 0; B < 3; ++B) deps[A][B] = (A == B) ? 1.0 : 0.0;
  }
  *pc_new = pcn;
  *mode = 0;
  if (dgam_out) *dgam_out = 0.0;
  if (m.model == MODEL_NH) return 0;

  double tau[3];
  nh_principal(etr, m, tau);
  double p = (tau[0] + tau[1] + tau[2]) / 3.0;
  double s[3] = {tau[0] - p, tau[1] - p, tau[2] - p};
  double J2 = 0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  double f, ftol;
  if (m.model == MODEL_NH_DP) {
    f = std::sqrt(J2) + m.eta * p - m.xi * m.coh;
    ftol = 1e-10 * m.mu;
  } else {
    f = 3.0 * J2 / (m.M * m.M) + p * (p - pcn);
    ftol = 1e-10 * m.mu * std::fabs(pcn);
  }
  // Reading: a trial state within a rounding-level tolerance of the yield
  // surface is elastic (e.g. a state committed on the surface, re-evaluated
  // at zero increment), so the branch does not hang on the last bit of f.
  if (!(f > ftol)) return 0;  // elastic

  if (m.model == MODEL_NH_DP && m.eta > 0.0) {
    // Apex test (reading): the deviatoric return keeps the trial volume
    // theta; on that volume the smallest pressure belongs to the isotropic
    // state (exp is convex), so if even that state violates f the return must
    // go to the apex tau = (xi c / eta) 1.
    double th = etr[0] + etr[1] + etr[2];
    double e0 = th / 3.0;
    double piso = m.mu * (std::exp(2.0 * e0) - 1.0) + m.lam * th;
    if (m.eta * piso - m.xi * m.coh >= 0.0) {
      double papex = m.xi * m.coh / m.eta;
      double e = e0;
      int it;
      for (it = 0; it < 100; ++it) {
        double g = m.mu * (std::exp(2.0 * e) - 1.0) + 3.0 * m.lam * e - papex;
        double dg = 2.0 * m.mu * std::exp(2.0 * e) + 3.0 * m.lam;
        double de = g / dg;
        e -= de;
        if (std::fabs(de) <= 1e-16 * (1.0 + std::fabs(e))) break;
      }
      if (it == 100) return -2;
      for (int A = 0; A < 3; ++A) {
        eps[A] = e;
        for (int B = 0; B < 3; ++B) deps[A][B] = 0.0;  // fixed stress state
      }
      *mode = 2;
      if (dgam_out) *dgam_out = 0.0;
      return 0;
    }
  }

  // local Newton on the four return-map equations from the trial state,
  // with step halving while the step does not reduce ||R|| (a safeguard;
  // the root it converges to is the same)
  double x[4] = {etr[0], etr[1], etr[2], 0.0};
  int conv = 0;
  for (int it = 0; it < 100; ++it) {
    double R[4], Jx[4][4], Je[4][3];
    model_res(x, etr, m, pcn, R);
    double n0 = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + R[3] * R[3]);
    res_jacobians(x, etr, m, pcn, Jx, Je);
    double dx[4] = {R[0], R[1], R[2], R[3]};
    if (solve_small(4, Jx, dx) != 0) return -2;
    double alpha = 1.0;
    for (int ls = 0; ls < 30; ++ls) {
      double xt[4], Rt[4];
      for (int i = 0; i < 4; ++i) xt[i] = x[i] - alpha * dx[i];
      model_res(xt, etr, m, pcn, Rt);
      double n1 = std::sqrt(Rt[0] * Rt[0] + Rt[1] * Rt[1] + Rt[2] * Rt[2] + Rt[3] * Rt[3]);
      // accept a sufficient decrease, or any step once ||R|| is at rounding level
      if (std::isfinite(n1) && (n1 <= (1.0 - 1e-4 * alpha) * n0 || n1 <= 1e-12)) break;
      alpha *= 0.5;
    }
    double big = 0;
    for (int i = 0; i < 4; ++i) {
      x[i] -= alpha * dx[i];
      big = std::max(big, std::fabs(alpha * dx[i]) / (1.0 + std::fabs(x[i])));
    }
    if (!std::isfinite(big)) return -2;
    if (alpha == 1.0 && big <= 1e-13) { conv = 1; break; }  // quadratic: the error left is ~1e-26
  }
  if (!conv) return -2;
  // implicit-function theorem: dx/detr = -(dR/dx)^-1 dR/detr
  double Jx[4][4], Je[4][3];
  res_jacobians(x, etr, m, pcn, Jx, Je);
  for (int B = 0; B < 3; ++B) {
    double a[4][4], b[4];
    std::memcpy(a, Jx, sizeof(a));
    for (int i = 0; i < 4; ++i) b[i] = -Je[i][B];
    if (solve_small(4, a, b) != 0) return -2;
    for (int A = 0; A < 3; ++A) deps[A][B] = b[A];
  }
  for (int A = 0; A < 3; ++A) eps[A] = x[A];
  if (m.model == MODEL_NH_MCC) {
    double dvp = (etr[0] - x[0]) + (etr[1] - x[1]) + (etr[2] - x[2]);
    *pc_new = pcn * std::exp(-dvp / m.lmk);
    if (dgam_out) *dgam_out = x[3] / std::fabs(pcn);
  } else if (dgam_out) {
    *dgam_out = x[3];
  }
  *mode = 1;
  return 0;
}

// ------------------------------------------------------------------------
// particle constitutive update and its exact tangent
// ------------------------------------------------------------------------
struct PartOut {
  M3 tau, be, P;   // Kirchhoff stress, new elastic left Cauchy-Green, V0 tau dF^-T
  double pc;
  int mode;
};

// b^tr = dF b_n dF^T -> spectral decomposition -> return map -> tau.
// A (optional, 81 entries) is dP[a][c]/d dF[b][e] stored A[(3a+c)*9 + 3b+e],
// with P = V0 tau dF^-T.
int particle_update(const Mat& m, const M3 be_n, double pcn, const M3 dF, double V0,
                    PartOut& o, double* A) {
  M3 t1, dFt, btr;
  transpose(dF, dFt);
  matmul(dF, be_n, t1);
  matmul(t1, dFt, btr);
  double lam[3];
  M3 Q;
  jacobi_eig(btr, lam, Q);
  for (int A_ = 0; A_ < 3; ++A_)
    if (!(lam[A_] > 0.0)) return -3;
  double etr[3] = {0.5 * std::log(lam[0]), 0.5 * std::log(lam[1]), 0.5 * std::log(lam[2])};
  double eps[3], deps[3][3], dg;
  int rc = return_map(m, etr, pcn, eps, &o.pc, &o.mode, deps, &dg);
  if (rc) return rc;
  double tp[3];
  nh_principal(eps, m, tp);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double st = 0, sb = 0;
      for (int A_ = 0; A_ < 3; ++A_) {
        st += tp[A_] * Q[i][A_] * Q[j][A_];
        sb += std::exp(2.0 * eps[A_]) * Q[i][A_] * Q[j][A_];
      }
      o.tau[i][j] = st;
      o.be[i][j] = sb;
    }
  M3 Fi, FiT;
  if (inv3(dF, Fi)) return -3;
  transpose(Fi, FiT);
  M3 TP;
  matmul(o.tau, FiT, TP);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o.P[i][j] = V0 * TP[i][j];
  if (!A) return 0;

  // principal tangent D[A][B] = d tau_A / d lam_B, lam the eigenvalues of b^tr:
  // d tau_A/d eps_C = 2 mu exp(2 eps_A) delta_AC + lam; d eps^tr_B/d lam_B = 1/(2 lam_B)
  double D[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0;
      for (int c = 0; c < 3; ++c) {
        double dtde = m.lam + ((a == c) ? 2.0 * m.mu * std::exp(2.0 * eps[a]) : 0.0);
        s += dtde * deps[c][b];
      }
      D[a][b] = s / (2.0 * lam[b]);
    }
  // Daleckii-Krein rule for the isotropic tensor function tau(b^tr):
  //   (Q^T dtau Q)_AA = sum_B D_AB (Q^T db Q)_BB,
  //   (Q^T dtau Q)_AB = theta_AB (Q^T db Q)_AB, A != B,
  // theta_AB = (tau_A - tau_B)/(lam_A - lam_B), or its limit
  // D_AA - D_AB when the eigenvalues coincide (relative gap below 1e-8).
  double lmax = std::max(std::fabs(lam[0]), std::max(std::fabs(lam[1]), std::fabs(lam[2])));
  double th[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a == b) { th[a][b] = 0; continue; }
      double gap = lam[a] - lam[b];
      if (std::fabs(gap) > 1e-8 * lmax) th[a][b] = (tp[a] - tp[b]) / gap;
      else th[a][b] = 0.5 * ((D[a][a] - D[a][b]) + (D[b][b] - D[b][a]));
    }
  M3 bnFt, Fbn;
  matmul(be_n, dFt, bnFt);  // b_n dF^T
  matmul(dF, be_n, Fbn);    // dF b_n
  for (int b = 0; b < 3; ++b)
    for (int e = 0; e < 3; ++e) {
      // direction d(dF) = E_be
      M3 db;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          // (E_be b_n dF^T)_ij = delta_ib (b_n dF^T)_ej ; (dF b_n E_be^T)_ij = (dF b_n)_ie delta_jb
          db[i][j] = ((i == b) ? bnFt[e][j] : 0.0) + ((j == b) ? Fbn[i][e] : 0.0);
        }
      M3 dbp, tmp, QT;
      transpose(Q, QT);
      matmul(QT, db, tmp);
      matmul(tmp, Q, dbp);
      M3 dtp;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          if (a == c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += D[a][k] * dbp[k][k];
            dtp[a][c] = s;
          } else {
            dtp[a][c] = th[a][c] * dbp[a][c];
          }
        }
      M3 dtau;
      matmul(Q, dtp, tmp);
      matmul(tmp, QT, dtau);
      // d(dF^-T) = -dF^-T E_be^T dF^-T  ->  (.)_ij = -FiT[i][e] FiT[b][j]
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          double s = 0;
          for (int k = 0; k < 3; ++k) s += dtau[a][k] * FiT[k][c];
          double s2 = 0;
          for (int k = 0; k < 3; ++k) s2 += o.tau[a][k] * (-FiT[k][e] * FiT[b][c]);
          A[(3 * a + c) * 9 + 3 * b + e] = V0 * (s + s2);
        }
    }
  return 0;
}

void sym6_to_m3(const double* s, M3 m) {
  // order xx, yy, zz, xy, yz, xz
  m[0][0] = s[0]; m[1][1] = s[1]; m[2][2] = s[2];
  m[0][1] = m[1][0] = s[3];
  m[1][2] = m[2][1] = s[4];
  m[0][2] = m[2][0] = s[5];
}
void m3_to_sym6(const M3 m, double* s) {
  s[0] = m[0][0]; s[1] = m[1][1]; s[2] = m[2][2];
  s[3] = 0.5 * (m[0][1] + m[1][0]);
  s[4] = 0.5 * (m[1][2] + m[2][1]);
  s[5] = 0.5 * (m[0][2] + m[2][0]);
}

Grid make_grid(const int* gi, const double* gd) {
  Grid G;
  G.dim = gi[0];
  G.n[0] = gi[1]; G.n[1] = gi[2]; G.n[2] = gi[3];
  G.h = gd[0];
  G.o[0] = gd[1]; G.o[1] = gd[2]; G.o[2] = gd[3];
  return G;
}

// G2P: dF = 1 + sum_i du_i (x) grad w_ip  (paper Sec. 2.2, stage 3)
void g2p_dF(const Grid& G, const Stencil& S, const double* du, M3 dF) {
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) dF[a][c] = (a == c) ? 1.0 : 0.0;
  for (int l = 0; l < S.cnt; ++l)
    for (int a = 0; a < G.dim; ++a)
      for (int c = 0; c < G.dim; ++c) dF[a][c] += du[S.node[l] * G.dim + a] * S.g[l][c];
}


// ------------------------------------------------------------------------
// u-p poromechanics (paper Sec. 2.2, remark on the coupled formulation; the
// paper defers the equations to the stabilised MPM u-p literature, so the
// form here is the reading: mixture momentum with total stress
// sigma = sigma' - p 1, fluid mass balance with incompressible constituents
// (J^{n+1} - J^n)/(dt J^{n+1}) + div q = 0, Darcy q = -kappa grad p, backward
// Euler in time, no stabilisation, the same quadratic B-splines for u and p).
// Per particle, with dF the step's deformation gradient, V^n = V0 det F^n,
// p_p = sum_j w_jp p_j and G_p = sum_j p_j grad w_jp (start-of-step
// gradients), multiplied through by dt:
//   pressure part of P:  Pp = -p_p V^n det(dF) dF^-T
//   volume term:         vol = V^n (det dF - 1)         (tested with w_ip)
//   flux term:           fl = kdt V^n det(dF) dF^-1 dF^-T G_p  (with grad w_ip)
// kdt = kappa dt.  Written once for plain doubles and once for dual numbers,
// whose derivative parts give the exact Jacobian of these terms.
// ------------------------------------------------------------------------
template <class S>
void up_terms(const S dF[3][3], S pp, const S G[3], double Vn, double kdt, S Pp[3][3], S& vol, S fl[3]) {
  S det = dF[0][0] * (dF[1][1] * dF[2][2] - dF[1][2] * dF[2][1]) -
          dF[0][1] * (dF[1][0] * dF[2][2] - dF[1][2] * dF[2][0]) +
          dF[0][2] * (dF[1][0] * dF[2][1] - dF[1][1] * dF[2][0]);
  // inverse by the adjugate
  S inv[3][3];
  inv[0][0] = (dF[1][1] * dF[2][2] - dF[1][2] * dF[2][1]) / det;
  inv[0][1] = (dF[0][2] * dF[2][1] - dF[0][1] * dF[2][2]) / det;
  inv[0][2] = (dF[0][1] * dF[1][2] - dF[0][2] * dF[1][1]) / det;
  inv[1][0] = (dF[1][2] * dF[2][0] - dF[1][0] * dF[2][2]) / det;
  inv[1][1] = (dF[0][0] * dF[2][2] - dF[0][2] * dF[2][0]) / det;
  inv[1][2] = (dF[0][2] * dF[1][0] - dF[0][0] * dF[1][2]) / det;
  inv[2][0] = (dF[1][0] * dF[2][1] - dF[1][1] * dF[2][0]) / det;
  inv[2][1] = (dF[0][1] * dF[2][0] - dF[0][0] * dF[2][1]) / det;
  inv[2][2] = (dF[0][0] * dF[1][1] - dF[0][1] * dF[1][0]) / det;
  const S Vnew = S(Vn) * det;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) Pp[a][c] = S(0.0) - pp * Vnew * inv[c][a];
  vol = S(Vn) * (det - S(1.0));
  // t = dF^-T G, fl = kdt V^{n+1} dF^-1 t
  S t[3];
  for (int k = 0; k < 3; ++k) t[k] = inv[0][k] * G[0] + inv[1][k] * G[1] + inv[2][k] * G[2];
  for (int c = 0; c < 3; ++c) fl[c] = S(kdt) * Vnew * (inv[c][0] * t[0] + inv[c][1] * t[1] + inv[c][2] * t[2]);
}

// G2P of the u-p nodal vector U (stride B = dim + 1): dF, p_p and G_p.
void g2p_up(const Grid& G, const Stencil& S, const double* U, M3 dF, double& pp, double Gp[3]) {
  const int B = G.dim + 1;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) dF[a][c] = (a == c) ? 1.0 : 0.0;
  pp = 0.0;
  Gp[0] = Gp[1] = Gp[2] = 0.0;
  for (int l = 0; l < S.cnt; ++l) {
    const double* u = U + S.node[l] * B;
    for (int a = 0; a < G.dim; ++a)
      for (int c = 0; c < G.dim; ++c) dF[a][c] += u[a] * S.g[l][c];
    pp += S.w[l] * u[G.dim];
    for (int c = 0; c < G.dim; ++c) Gp[c] += u[G.dim] * S.g[l][c];
  }
}

}  // namespace

extern "C" {

// gi = {dim, nx, ny, nz}; gd = {h, ox, oy, oz}
// Shape functions of one particle: up to 27 nodes, weights, gradients.
int orc_stencil(const int* gi, const double* gd, const double* xp, long* node, double* w,
                double* g) {
  Grid G = make_grid(gi, gd);
  Stencil S;
  if (make_stencil(G, xp, S)) return -1;
  for (int l = 0; l < S.cnt; ++l) {
    node[l] = S.node[l];
    w[l] = S.w[l];
    for (int a = 0; a < 3; ++a) g[3 * l + a] = S.g[l][a];
  }
  return S.cnt;
}

int orc_eig(const double* a9, double* lam, double* Q9) {
  M3 a, Q;
  std::memcpy(a, a9, sizeof(M3));
  jacobi_eig(a, lam, Q);
  std::memcpy(Q9, Q, sizeof(M3));
  return 0;
}

// Principal return map alone (for pins): model, params8, etr (3), pcn.
int orc_return_map(int model, const double* params, const double* etr, double pcn, double* eps,
                   double* pc_new, int* mode, double* deps9, double* dgam) {
  Mat m = make_mat(model, params);
  double d[3][3];
  int rc = return_map(m, etr, pcn, eps, pc_new, mode, d, dgam);
  std::memcpy(deps9, d, sizeof(d));
  return rc;
}

// One particle: dF (9, row-major), be_n (6), pcn, V0 -> tau (9), be (6), pc,
// mode, P = V0 tau dF^-T (9) and optionally A = dP/d dF (81).
int orc_particle(int model, const double* params, const double* be6, double pcn,
                 const double* dF9, double V0, double* tau9, double* be6_out, double* pc_out,
                 int* mode, double* P9, double* A81) {
  Mat m = make_mat(model, params);
  M3 be, dF;
  sym6_to_m3(be6, be);
  std::memcpy(dF, dF9, sizeof(M3));
  PartOut o;
  int rc = particle_update(m, be, pcn, dF, V0, o, A81);
  if (rc) return rc;
  std::memcpy(tau9, o.tau, sizeof(M3));
  m3_to_sym6(o.be, be6_out);
  *pc_out = o.pc;
  *mode = o.mode;
  std::memcpy(P9, o.P, sizeof(M3));
  return 0;
}

// Global residual r = f_int - f_ext on the dense node grid (nnode*dim) and
// nodal mass M_i = sum_p w_ip m_p (paper's mapping equation).  f_ext spreads
// each particle's weight m_p g and the force it carries, fext (3 per
// particle, nullable: the traction term of the paper's discrete external
// force, read as a traction times the particle's share of the loaded face),
// with w_ip.  Returns 0, -1 (particle outside the grid) or a constitutive
// failure code.  When `mode_out` is given the per-particle mode is written
// there; when `rabs` is given it receives sum_p |contribution| per DOF (the
// scale against which the rounding of r is judged).
int orc_residual(const int* gi, const double* gd, const double* grav, int np, const double* x,
                 const double* V0, const double* m, const int* model, const double* params,
                 const double* be, const double* pc, const double* fext, const double* du, double* r,
                 double* mass, int* mode_out, double* rabs) {
  Grid G = make_grid(gi, gd);
  long nn = G.nnode();
  std::fill(r, r + nn * G.dim, 0.0);
  std::fill(mass, mass + nn, 0.0);
  if (rabs) std::fill(rabs, rabs + nn * G.dim, 0.0);
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben;
    g2p_dF(G, S, du, dF);
    sym6_to_m3(be + 6 * p, ben);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, nullptr);
    if (rc) return rc;
    if (mode_out) mode_out[p] = o.mode;
    for (int l = 0; l < S.cnt; ++l) {
      long i = S.node[l];
      mass[i] += S.w[l] * m[p];
      for (int a = 0; a < G.dim; ++a) {
        double f = 0;
        for (int c = 0; c < G.dim; ++c) f += o.P[a][c] * S.g[l][c];
        const double fe = S.w[l] * (m[p] * grav[a] + (fext ? fext[3 * p + a] : 0.0));
        r[i * G.dim + a] += f - fe;
        if (rabs) rabs[i * G.dim + a] += std::fabs(f) + std::fabs(fe);
      }
    }
  }
  return 0;
}

// Global Jacobian K_ij[a][b] = sum_p sum_{c,e} gw_ip[c] A_p[a c b e] gw_jp[e]
// as node-pair blocks (dim x dim, row-major), summed over particles.
// Writes at most `cap` blocks; returns the number of blocks (or <0 on error).
int orc_jacobian(const int* gi, const double* gd, int np, const double* x, const double* V0,
                 const int* model, const double* params, const double* be, const double* pc,
                 const double* du, long cap, long* bi, long* bj, double* bval) {
  Grid G = make_grid(gi, gd);
  const int d = G.dim;
  std::map<std::pair<long, long>, std::array<double, 9>> K;
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben;
    g2p_dF(G, S, du, dF);
    sym6_to_m3(be + 6 * p, ben);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    double A[81];
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, A);
    if (rc) return rc;
    for (int li = 0; li < S.cnt; ++li)
      for (int lj = 0; lj < S.cnt; ++lj) {
        auto& blk = K[std::make_pair(S.node[li], S.node[lj])];
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) {
            double s = 0;
            for (int c = 0; c < d; ++c)
              for (int e = 0; e < d; ++e)
                s += S.g[li][c] * A[(3 * a + c) * 9 + 3 * b + e] * S.g[lj][e];
            blk[a * d + b] += s;
          }
      }
  }
  long k = 0;
  for (auto& kv : K) {
    if (k >= cap) return -4;
    bi[k] = kv.first.first;
    bj[k] = kv.first.second;
    for (int t = 0; t < d * d; ++t) bval[k * d * d + t] = kv.second[t];
    ++k;
  }
  return (int)k;
}

// Commit after convergence (paper Sec. 2.2, stage 4): x += sum_i w_ip du_i,
// F <- dF F, be and pc from the return map.
int orc_commit(const int* gi, const double* gd, int np, double* x, const double* V0,
               const int* model, const double* params, double* be, double* pc, double* F,
               const double* du) {
  Grid G = make_grid(gi, gd);
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben;
    g2p_dF(G, S, du, dF);
    sym6_to_m3(be + 6 * p, ben);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, nullptr);
    if (rc) return rc;
    double dx[3] = {0, 0, 0};
    for (int l = 0; l < S.cnt; ++l)
      for (int a = 0; a < G.dim; ++a) dx[a] += S.w[l] * du[S.node[l] * G.dim + a];
    for (int a = 0; a < G.dim; ++a) x[3 * p + a] += dx[a];
    m3_to_sym6(o.be, be + 6 * p);
    pc[p] = o.pc;
    M3 Fo, Fn;
    std::memcpy(Fo, F + 9 * p, sizeof(M3));
    matmul(dF, Fo, Fn);
    std::memcpy(F + 9 * p, Fn, sizeof(M3));
  }
  return 0;
}

// ---- u-p formulation --------------------------------------------------
// U and r hold B = dim + 1 values per node: (du_0 .. du_{dim-1}, p), with p
// the pore pressure at the end of the step (positive in compression) and
// r_p the fluid mass balance multiplied by dt.  F (9 per particle) is the
// start-of-step deformation gradient (V^n = V0 det F); kdt = kappa dt per
// particle; fext (3 per particle, nullable) is an external force carried by
// the particle (a surface traction times the particle's face area), spread
// to the nodes with w_ip like gravity.
int orc_residual_up(const int* gi, const double* gd, const double* grav, int np, const double* x,
                    const double* V0, const double* F, const double* m, const int* model,
                    const double* params, const double* be, const double* pc, const double* kdt,
                    const double* fext, const double* U, double* r, double* mass, int* mode_out,
                    double* rabs) {
  Grid G = make_grid(gi, gd);
  const int d = G.dim, B = d + 1;
  long nn = G.nnode();
  std::fill(r, r + nn * B, 0.0);
  std::fill(mass, mass + nn, 0.0);
  if (rabs) std::fill(rabs, rabs + nn * B, 0.0);
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben, Fn;
    double pp, Gp[3];
    g2p_up(G, S, U, dF, pp, Gp);
    sym6_to_m3(be + 6 * p, ben);
    std::memcpy(Fn, F + 9 * p, sizeof(M3));
    const double Vn = V0[p] * det3(Fn);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, nullptr);
    if (rc) return rc;
    if (mode_out) mode_out[p] = o.mode;
    double Pp[3][3], vol, fl[3];
    up_terms<double>(dF, pp, Gp, Vn, kdt[p], Pp, vol, fl);
    for (int l = 0; l < S.cnt; ++l) {
      long i = S.node[l];
      mass[i] += S.w[l] * m[p];
      for (int a = 0; a < d; ++a) {
        double f = 0, fa = 0;
        for (int c = 0; c < d; ++c) {
          f += (o.P[a][c] + Pp[a][c]) * S.g[l][c];
          fa += std::fabs(o.P[a][c] * S.g[l][c]) + std::fabs(Pp[a][c] * S.g[l][c]);
        }
        const double fe = S.w[l] * (m[p] * grav[a] + (fext ? fext[3 * p + a] : 0.0));
        r[i * B + a] += f - fe;
        if (rabs) rabs[i * B + a] += fa + std::fabs(fe);
      }
      double q = S.w[l] * vol, qa = std::fabs(S.w[l] * vol);
      for (int c = 0; c < d; ++c) {
        q += fl[c] * S.g[l][c];
        qa += std::fabs(fl[c] * S.g[l][c]);
      }
      r[i * B + d] += q;
      if (rabs) rabs[i * B + d] += qa;
    }
  }
  return 0;
}

// Exact Jacobian of the u-p residual as (B x B) node-pair blocks: the
// effective-stress part through the tangent A_p of the solid oracle, the
// pressure, volume and flux terms through forward-mode dual numbers seeded
// on dF_be, p_p and G_p,e.
int orc_jacobian_up(const int* gi, const double* gd, int np, const double* x, const double* V0,
                    const double* F, const int* model, const double* params, const double* be,
                    const double* pc, const double* kdt, const double* U, long cap, long* bi, long* bj,
                    double* bval) {
  Grid G = make_grid(gi, gd);
  const int d = G.dim, B = d + 1;
  std::map<std::pair<long, long>, std::array<double, 16>> K;
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben, Fn;
    double pp, Gp[3];
    g2p_up(G, S, U, dF, pp, Gp);
    sym6_to_m3(be + 6 * p, ben);
    std::memcpy(Fn, F + 9 * p, sizeof(M3));
    const double Vn = V0[p] * det3(Fn);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    double A[81];
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, A);
    if (rc) return rc;
    // derivatives of (Pp, vol, fl): seeds 0..8 = dF_be (b*3+e), 9 = p_p, 10..12 = G_e
    double dPp[13][3][3], dvol[13], dfl[13][3];
    for (int sd = 0; sd < 13; ++sd) {
      Dual dFd[3][3], ppd(pp, sd == 9 ? 1.0 : 0.0), Gd[3];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) dFd[a][c] = Dual(dF[a][c], (sd < 9 && sd == 3 * a + c) ? 1.0 : 0.0);
      for (int c = 0; c < 3; ++c) Gd[c] = Dual(Gp[c], (sd == 10 + c) ? 1.0 : 0.0);
      Dual Ppd[3][3], vold, fld[3];
      up_terms<Dual>(dFd, ppd, Gd, Vn, kdt[p], Ppd, vold, fld);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) dPp[sd][a][c] = Ppd[a][c].d;
      dvol[sd] = vold.d;
      for (int c = 0; c < 3; ++c) dfl[sd][c] = fld[c].d;
    }
    for (int li = 0; li < S.cnt; ++li)
      for (int lj = 0; lj < S.cnt; ++lj) {
        auto& blk = K[std::make_pair(S.node[li], S.node[lj])];
        const double* gi_ = S.g[li];
        const double* gj_ = S.g[lj];
        const double wi = S.w[li], wj = S.w[lj];
        // momentum rows a, displacement columns b
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) {
            double s = 0;
            for (int c = 0; c < d; ++c)
              for (int e = 0; e < d; ++e)
                s += gi_[c] * (A[(3 * a + c) * 9 + 3 * b + e] + dPp[3 * b + e][a][c]) * gj_[e];
            blk[a * B + b] += s;
          }
        // momentum rows a, pressure column: through p_p (w_j) and G_p (g_j)
        for (int a = 0; a < d; ++a) {
          double s = 0;
          for (int c = 0; c < d; ++c) {
            s += gi_[c] * dPp[9][a][c] * wj;
            for (int e = 0; e < d; ++e) s += gi_[c] * dPp[10 + e][a][c] * gj_[e];
          }
          blk[a * B + d] += s;
        }
        // mass-balance row, displacement columns b
        for (int b = 0; b < d; ++b) {
          double s = 0;
          for (int e = 0; e < d; ++e) {
            double t = wi * dvol[3 * b + e];
            for (int c = 0; c < d; ++c) t += gi_[c] * dfl[3 * b + e][c];
            s += t * gj_[e];
          }
          blk[d * B + b] += s;
        }
        // mass-balance row, pressure column
        {
          double s = wi * dvol[9] * wj;
          for (int e = 0; e < d; ++e) s += wi * dvol[10 + e] * gj_[e];
          for (int c = 0; c < d; ++c) {
            s += gi_[c] * dfl[9][c] * wj;
            for (int e = 0; e < d; ++e) s += gi_[c] * dfl[10 + e][c] * gj_[e];
          }
          blk[d * B + d] += s;
        }
      }
  }
  long k = 0;
  for (auto& kv : K) {
    if (k >= cap) return -4;
    bi[k] = kv.first.first;
    bj[k] = kv.first.second;
    for (int t = 0; t < B * B; ++t) bval[k * B * B + t] = kv.second[t];
    ++k;
  }
  return (int)k;
}

// Commit of a u-p step: as orc_commit with the displacement part of U, and
// the particle pore pressure p_p = sum_i w_ip p_i written to pp.
int orc_commit_up(const int* gi, const double* gd, int np, double* x, const double* V0,
                  const int* model, const double* params, double* be, double* pc, double* F,
                  const double* U, double* pp) {
  Grid G = make_grid(gi, gd);
  const int d = G.dim, B = d + 1;
  for (int p = 0; p < np; ++p) {
    Stencil S;
    if (make_stencil(G, x + 3 * p, S)) return -1;
    M3 dF, ben;
    double ppv, Gp[3];
    g2p_up(G, S, U, dF, ppv, Gp);
    sym6_to_m3(be + 6 * p, ben);
    Mat mt = make_mat(model[p], params + 8 * p);
    PartOut o;
    int rc = particle_update(mt, ben, pc[p], dF, V0[p], o, nullptr);
    if (rc) return rc;
    double dx[3] = {0, 0, 0};
    for (int l = 0; l < S.cnt; ++l)
      for (int a = 0; a < d; ++a) dx[a] += S.w[l] * U[S.node[l] * B + a];
    for (int a = 0; a < d; ++a) x[3 * p + a] += dx[a];
    m3_to_sym6(o.be, be + 6 * p);
    pc[p] = o.pc;
    M3 Fo, Fnew;
    std::memcpy(Fo, F + 9 * p, sizeof(M3));
    matmul(dF, Fo, Fnew);
    std::memcpy(F + 9 * p, Fnew, sizeof(M3));
    pp[p] = ppv;
  }
  return 0;
}

}  // extern "C"
