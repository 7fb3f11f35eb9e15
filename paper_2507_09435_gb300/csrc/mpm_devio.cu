// Device-pointer variants of the scene's getters and of the Dirichlet setter:
// the caller passes device buffers it owns (for example the data pointers of
// CUDA tensors); the work is issued on the scene's stream and the getters do
// not synchronise the host.  Units and layouts are those of the host getters:
// the u-p pressure unknowns and mass-balance rows are returned in physical
// units (the solver holds p / psc and rows scaled by psc).
#include "mpm_internal.h"

namespace mpm {

namespace {
constexpr int DTPB = 256;
inline unsigned nblk(long long n) { return (unsigned)((n + DTPB - 1) / DTPB); }

__global__ void k_du_out(const double* __restrict__ du, double* out, long long ndof, int B, int D, double psc) {
  const long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (d >= ndof) return;
  const double v = du[d];
  out[d] = (B > D && d % B == D) ? v * psc : v;
}

__global__ void k_residual_out(const double* __restrict__ r, const uint8_t* __restrict__ fixed,
                               const int* __restrict__ node2row, double* out, long long ndof, int B, int D,
                               double psc) {
  const long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (d >= ndof) return;
  double v = (fixed[d] || node2row[d / B] < 0) ? 0.0 : r[d];
  if (B > D && d % B == D) v /= psc;
  out[d] = v;
}

// positions in the caller's particle order, 3 per particle (z = 0 in 2D)
__global__ void k_positions_out(DevParticles P, int D, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const long long o = (long long)P.orig[p] * 3;
#pragma unroll
  for (int a = 0; a < 3; ++a) out[o + a] = (a < D) ? P.x[a][p] : 0.0;
}

// prescribed DOFs from device arrays; an index outside [0, ndof) is skipped
// and counted in *bad
__global__ void k_dirichlet_in(int n, const long long* __restrict__ dof, const double* __restrict__ value,
                               uint8_t* fixed, double* bcval, long long ndof, int B, int D, double psc, int* bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long d = dof[k];
  if (d < 0 || d >= ndof) {
    atomicAdd(bad, 1);
    return;
  }
  fixed[d] = 1;
  bcval[d] = (B > D && d % B == D) ? value[k] / psc : value[k];
}
}  // namespace

cudaError_t launch_du_out(const double* du, double* out, long long ndof, int B, int D, double psc,
                          cudaStream_t st) {
  if (ndof == 0) return cudaSuccess;
  k_du_out<<<nblk(ndof), DTPB, 0, st>>>(du, out, ndof, B, D, psc);
  return cudaGetLastError();
}

cudaError_t launch_residual_out(const double* r, const uint8_t* fixed, const int* node2row, double* out,
                                long long ndof, int B, int D, double psc, cudaStream_t st) {
  if (ndof == 0) return cudaSuccess;
  k_residual_out<<<nblk(ndof), DTPB, 0, st>>>(r, fixed, node2row, out, ndof, B, D, psc);
  return cudaGetLastError();
}

cudaError_t launch_positions_out(const DevParticles& P, int D, double* out, cudaStream_t st) {
  if (P.np == 0) return cudaSuccess;
  k_positions_out<<<nblk(P.np), DTPB, 0, st>>>(P, D, out);
  return cudaGetLastError();
}

cudaError_t launch_dirichlet_in(int n, const long long* dof, const double* value, uint8_t* fixed, double* bcval,
                                long long ndof, int B, int D, double psc, int* bad, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_dirichlet_in<<<nblk(n), DTPB, 0, st>>>(n, dof, value, fixed, bcval, ndof, B, D, psc, bad);
  return cudaGetLastError();
}

}  // namespace mpm
