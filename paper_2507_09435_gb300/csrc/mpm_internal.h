// Internal declarations shared by the CUDA translation units of libmpm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_device.cuh"

namespace mpm {

constexpr int MAX_BE = 6;
constexpr int MAX_F = 9;

// Particle state on the device, structure of arrays, kept sorted by base cell.
struct DevParticles {
  int np;
  double* x[3];
  double* vol0;
  double* mass;
  int* mat;
  double* Ep;        // per-particle Young's modulus (always filled)
  double* phip;      // per-particle friction angle (always filled)
  double* be[MAX_BE];  // xx, yy, zz, xy (2D) / xx, yy, zz, xy, yz, xz (3D)
  double* pc;
  double* F[MAX_F];  // dim*dim row-major
  int* orig;         // caller's index of each sorted particle
  double* kdt;       // u-p: mobility times time step (null for the solid formulation)
  double* pp;        // u-p: pore pressure at the particle after the last commit
  double* fext[3];   // external force carried by the particle (null: none)
  // first constitutive failure of a pass: [claimed, caller index, trial b
  // eigenvalues (3), E, phi, pc, model, return-map mode]
  double* fail_rec;
};
constexpr int FAIL_REC = 10;

struct DevGrid {
  int dim;
  int n[3];
  int nx1, ny1, nz1;
  long long nnode;
  double h, ih;
  double o[3];
};

// Stencil-BSR Jacobian: for every active node (row) the 5^dim neighbour
// blocks at fixed slots, one plane per slot, blocks contiguous within a plane:
// val[(slot*cap + row)*B*B + a*B + b] with B values per node (a 2x2 FP32
// block is one 16-byte load).
template <class T>
struct DevMatrix {
  T* val;
  const unsigned* pmask;  // per row PMASK_WORDS(D) words, bit s set when slot s can be
                          // nonzero (the node pair shares an occupied cell); null: read
                          // every slot (absent slots hold zeros either way)
  T* dinv;          // block-Jacobi inverse: seg == 1: dinv[row*B*B + a*B + b], the
                    // node's diagonal block; seg == 4: dinv[(s*4B + i)*4B + j], the
                    // inverse of the 4B x 4B diagonal block of rows 4s..4s+3
  int cap;          // row capacity (row stride of the SoA planes)
  const int* rows;  // node index of each row
  const int* nrow;  // device scalar: active row count
  int seg;          // rows per preconditioner block: 1 (node) or 4 (row segment)
};

// One D x D block of the matrix (contiguous), through the read-only path:
// a single 16-byte load for 2x2 FP32, two for 2x2 FP64.  GENERIC: ordinary
// loads through a generic pointer (the block may sit in shared memory).
template <int D, class T, bool GENERIC = false>
__device__ __forceinline__ void ld_block(const T* p, T b[D * D]) {
  if constexpr (D == 2 && sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 v = GENERIC ? *q : __ldg(q);
    b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
  } else if constexpr (D == 2 && sizeof(T) == 8) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 u = GENERIC ? q[0] : __ldg(q);
    const double2 w = GENERIC ? q[1] : __ldg(q + 1);
    b[0] = u.x; b[1] = u.y; b[2] = w.x; b[3] = w.y;
  } else {
#pragma unroll
    for (int k = 0; k < D * D; ++k) b[k] = GENERIC ? p[k] : __ldg(p + k);
  }
}

// The D entries of node j of a vector.  WEAK = true issues ordinary (weak,
// L1-cacheable) loads, for data written earlier in the same kernel and made
// visible by a release/acquire grid barrier; otherwise the read-only path,
// for data constant over the kernel.
template <int D, class T, bool WEAK>
__device__ __forceinline__ void ld_node(const T* x, long long j, T v[D]) {
  if constexpr (D == 2 && sizeof(T) == 4) {
    const float2* q = reinterpret_cast<const float2*>(x + j * 2);
    const float2 u = WEAK ? *q : __ldg(q);
    v[0] = u.x; v[1] = u.y;
  } else if constexpr (D == 2 && sizeof(T) == 8) {
    const double2* q = reinterpret_cast<const double2*>(x + j * 2);
    const double2 u = WEAK ? *q : __ldg(q);
    v[0] = u.x; v[1] = u.y;
  } else {
#pragma unroll
    for (int b = 0; b < D; ++b) v[b] = WEAK ? x[j * D + b] : __ldg(x + j * D + b);
  }
}

// z = M^-1 v for one row, M the block-Jacobi preconditioner.  With row
// segments (K.seg == 4) the four rows of a segment sit on four consecutive
// lanes of one warp (one thread per row, blockDim a multiple of 32, rows
// aligned to 4), which exchange their values by shuffles.  `live` is the
// ballot of the lanes that call this (exactly the lanes executing it).
// GENERIC: the inverses may sit in shared memory (ordinary loads).
template <int B, class T, bool GENERIC = false>
__device__ __forceinline__ void precond_apply(const DevMatrix<T>& K, int row, const T v[B], T z[B],
                                              unsigned live) {
  if (K.seg <= 1) {
    T m[B * B];
    ld_block<B, T, GENERIC>(&K.dinv[(long long)row * (B * B)], m);
#pragma unroll
    for (int a = 0; a < B; ++a) {
      T s = (T)0;
#pragma unroll
      for (int b = 0; b < B; ++b) s += m[a * B + b] * v[b];
      z[a] = s;
    }
    return;
  }
  constexpr int W = 4 * B;
  const int lane = threadIdx.x & 31, base = lane & ~3, r = lane & 3;
  const T* M = K.dinv + ((long long)(row >> 2) * W + r * B) * W;
#pragma unroll
  for (int a = 0; a < B; ++a) z[a] = (T)0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool src = (live >> (base + q)) & 1u;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const T t = __shfl_sync(live, v[b], base + q);
      const T vb = src ? t : (T)0;
#pragma unroll
      for (int a = 0; a < B; ++a) z[a] += (GENERIC ? M[a * W + q * B + b] : __ldg(M + a * W + q * B + b)) * vb;
    }
  }
}

// Words of the per-row slot-presence mask.
constexpr int pmask_words(int D) { return D == 2 ? 1 : 4; }

// The row's slot-presence words (all ones without a mask).
template <int D, bool GENERIC = false>
__device__ __forceinline__ void load_pmask(const unsigned* pmask, int row, unsigned pm[pmask_words(D)]) {
  constexpr int PW = pmask_words(D);
  if (pmask) {
    if constexpr (PW == 4) {
      const uint4* q = reinterpret_cast<const uint4*>(pmask) + row;
      const uint4 v = GENERIC ? *q : __ldg(q);
      pm[0] = v.x; pm[1] = v.y; pm[2] = v.z; pm[3] = v.w;
    } else {
      pm[0] = GENERIC ? pmask[row] : __ldg(pmask + row);
    }
  } else {
#pragma unroll
    for (int w = 0; w < PW; ++w) pm[w] = ~0u;
  }
}

// y = K x for one row (node i) of a stencil-BSR matrix: the 5^D neighbour
// blocks of the row against the neighbours' values of x (x on the padded
// dense node grid of the matrix's level); slots absent from the row's
// presence mask are not read.  COHERENT: x was written earlier in the same
// kernel (ordinary loads instead of the read-only path).  GENERIC: the matrix
// may sit in shared memory (ordinary loads for it as well).
template <int D, class T, int B, bool COHERENT = false, bool GENERIC = false>
__device__ __forceinline__ void stencil_row_product(const DevMatrix<T>& K, int row, long long i, int nx1, int ny1,
                                                    const T* x, T y[B]) {
#pragma unroll
  for (int a = 0; a < B; ++a) y[a] = (T)0;
  constexpr int ZR = (D == 3) ? 2 : 0;
  const long long cap = K.cap;
  unsigned pm[pmask_words(D)];
  load_pmask<D, GENERIC>(K.pmask, row, pm);
#pragma unroll
  for (int dz = -ZR; dz <= ZR; ++dz)
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
      for (int dx = -2; dx <= 2; ++dx) {
        const int slot = (D == 2) ? (dx + 2) + 5 * (dy + 2) : (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
        // absent slots: predicated off (no load is issued), not branched
        // around, so that the loads of all slots stay in flight together
        const bool on = (pm[slot >> 5] >> (slot & 31)) & 1u;
        const long long j = i + dx + (long long)nx1 * (dy + (long long)ny1 * dz);
        T xj[B], kb[B * B];
        if (on) {
          ld_node<B, T, COHERENT || GENERIC>(x, j, xj);
          ld_block<B, T, GENERIC>(&K.val[((long long)slot * cap + row) * (B * B)], kb);
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) xj[b] = (T)0;
#pragma unroll
          for (int b = 0; b < B * B; ++b) kb[b] = (T)0;
        }
#pragma unroll
        for (int a = 0; a < B; ++a)
#pragma unroll
          for (int b = 0; b < B; ++b) y[a] += kb[a * B + b] * xj[b];
      }
}

// Threads per block of the row-parallel Krylov kernels (one thread per
// active row; the grids are ceil(rows / KRYLOV_TPB) blocks).
constexpr int KRYLOV_TPB = 128;

struct KrylovScalars {
  double rho, alpha, omega;
  double acc_rv, acc_ts, acc_tt, acc_rho, acc_rr;
  double tol2, bnorm2, rr_last;
  int iter, done, status, maxit;
  // merged-reduction BiCGStab: rho of the previous iteration and the extra
  // dot products (s,s), (rhat,s), (rhat,t), (v,v); (rhat,rhat) of the start
  double rho_old, acc_ss, acc_rs, acc_rt, acc_vv, rhat2;
  // blocks of the current kernel that have stored their partial sums (the
  // last one adds them up and resets it)
  unsigned int ticket;
  // merged BiCGStab, set once per kernel by the last block of the grid sum:
  // beta and the FP32 copies of alpha, omega and beta; the stop decision
  // for the next iteration (0: go on, else 1 + status) and the breakdown
  // flag of the (rhat, v) test
  double beta;
  float alpha_f, omega_f, beta_f;
  int next_stop, c_break;
};

// ---- host launchers (stream-ordered, no synchronisation) ----------------
cudaError_t scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st);
size_t scan_tmp_ints(int n);

template <int D>
cudaError_t launch_cell_keys(const DevParticles& P, const DevGrid& G, int* key, int* count, int* rank,
                             int* err, cudaStream_t st);
cudaError_t launch_sort_scatter(int np, const int* key, const int* rank, const int* cstart, int* perm,
                                cudaStream_t st);
struct GatherArrays {
  int nd, ni;
  const double* dsrc[24];
  double* ddst[24];
  const int* isrc[4];
  int* idst[4];
};
cudaError_t launch_gather(int np, const int* perm, const GatherArrays& g, cudaStream_t st);
cudaError_t launch_flag_positive(const int* count, int* flag, long long n, cudaStream_t st);
cudaError_t launch_compact(const int* flag, const int* pos, int* list, long long n, cudaStream_t st);
template <int D>
cudaError_t launch_mass(const DevParticles& P, const DevGrid& G, const int* cstart, double* fp, double* M,
                        long long nnode, cudaStream_t st);
cudaError_t launch_active(const double* M, double thr, int* flag, long long nnode, cudaStream_t st);
cudaError_t launch_node2row(const int* flag, const int* pos, int* node2row, int* rows, long long nnode,
                            cudaStream_t st);
cudaError_t launch_apply_bc(const uint8_t* fixed, const double* bcval, const int* node2row, double* du,
                            long long ndof, int D, cudaStream_t st);

// particle pass: mode 0 residual, 1 residual + tangent, 2 commit
template <int D, class T>
cudaError_t launch_particles(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* du,
                             double* r, const double* grav, T* A, int mode, int* err, int* nplastic,
                             cudaStream_t st);
// u-p particle pass (B = D + 1 values per node, the last the scaled pore
// pressure p / psc; the mass-balance rows of r are scaled by psc, and so are
// the pressure rows and columns of the tangent)
template <int D, class T>
cudaError_t launch_particles_up(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* U,
                                double* r, const double* grav, T* A, int mode, double psc, int* err,
                                int* nplastic, cudaStream_t st);
template <int D>
cudaError_t launch_stress_out(const DevParticles& P, const DevGrid& G, const MatC* mats, double* tau9,
                              cudaStream_t st);

// Values per cell block of the 3D assembly: 27 x 27 node pairs x 9, padded
// to a multiple of 16 bytes.
constexpr int CELL_BLOCK_VALUES = 6564;
// Occupied cells and their block buffer for the 3D two-phase assembly:
// cells[0..ncell) the occupied cells (base nodes) in index order, count the
// particles per cell, cellpos[cell] the cell's position in that list, blk
// room for ncell x CELL_BLOCK_VALUES values.
template <class T>
struct Asm3 {
  const int* cells;
  int ncell;
  const int* count;
  const int* cellpos;
  T* blk;
};
// a3: the 3D cell data (unused in 2D, may be null there)
template <int D, class T, int B = D>
cudaError_t launch_assemble(const DevParticles& P, const DevGrid& G, const int* cstart, const int* node2row,
                            const T* A, DevMatrix<T> K, int nrow_host, const Asm3<T>* a3, cudaStream_t st);
// 3D single-phase rows: cell block products, then a gather per row
// (mpm_assemble_cells.cu)
template <class T>
cudaError_t launch_assemble_cells3(const DevParticles& P, const DevGrid& G, const Asm3<T>& a3, const int* cstart,
                                   const int* node2row, const T* A, DevMatrix<T> K, int nrow_host,
                                   cudaStream_t st);
template <int D, class T, int B = D>
cudaError_t launch_bc_matrix(const DevGrid& G, DevMatrix<T> K, const uint8_t* fixed, const int* node2row,
                             int nrow_host, cudaStream_t st);
template <int D, class T, int B = D>
cudaError_t launch_block_jacobi(const DevGrid& G, DevMatrix<T> K, int nrow_host, int* err, cudaStream_t st);
template <int D>
cudaError_t launch_pattern_count(const DevGrid& G, const int* rows, int nrow_host, const int* node2row,
                                 const int* count, int* mask, cudaStream_t st);
// the same pattern as per-row slot-presence bits (pmask_words(D) per row)
template <int D>
cudaError_t launch_pattern_bits(const DevGrid& G, const int* rows, int nrow_host, const int* node2row,
                                const int* count, unsigned* bits, cudaStream_t st);

// free-DOF residual norm^2 into *out (device double, written; the sum in an
// order fixed by the grid, through part and ticket: ticket zero on entry,
// left zero)
template <int D>
cudaError_t launch_norm_free(const double* r, const int* rows, int nrow_host, const uint8_t* fixed,
                             double* out, double* part, unsigned* ticket, cudaStream_t st);
// scratch of launch_norm_free: one double per block of 256 rows
inline long long norm_part_slots(long long rows) { return (rows + 255) / 256 + 1; }
// r on every grid node from the particles' contributions fp (B values per
// node, the k_particles / k_particles_up layout), in a fixed order
template <int D, int B>
cudaError_t launch_gather_residual(const DevGrid& G, const int* cstart, const double* fp, int np, double* r,
                                   long long nn, cudaStream_t st);
// the particles of every cell in increasing source index (after the scatter)
cudaError_t launch_sort_cells(const int* cstart, int* perm, long long ncells, cudaStream_t st);

// Geometric multigrid preconditioner (mpm_mg.cu).  One level of the
// hierarchy: the level's grid (nz1 = 1 in 2D), its stencil-BSR matrix (seg 1
// on the coarse levels; the block inverses pre-multiplied by the smoother's
// damping), node -> row map, prescribed-DOF flags and three padded vectors.
template <class T>
struct MgLevel {
  int nx1, ny1, nz1;
  DevMatrix<T> K;
  const int* node2row;
  const uint8_t* fixed;
  T *b, *z, *r;
};
constexpr int MG_MAX_LEVELS = 12;
constexpr int MG_DENSE_MAX = 128;   // unknowns of the coarsest (dense) level
constexpr int MG_POWER_IT = 8;      // power iterations for lambda_max(D^-1 A)
constexpr int MG_TAIL_ROWS = 16384; // coarse levels this small run inside one cluster
constexpr int MG_NU0 = 2;           // smoothing sweeps per side on the finest level
constexpr int MG_TAIL_TPB = 512;
// Threads per block of the cluster tail: 1024 for 2D FP32 node blocks (one
// row per thread for levels of up to 16,384 rows on 16 blocks), else
// MG_TAIL_TPB (the register budget of the wider blocks).
constexpr int MG_TAIL_TPB_WIDE = 1024;
template <class T, int B>
constexpr int mg_tail_tpb() {
  return (sizeof(T) == 4 && B == 2) ? MG_TAIL_TPB_WIDE : MG_TAIL_TPB;
}
// Dynamic shared memory the cluster tail may take per block for the levels it
// stages (one block per SM at this size).
constexpr int MG_TAIL_SMEM_MAX = 200 * 1024;
// Where one staged level sits in the tail's dynamic shared memory: byte
// offsets of its row list, matrix blocks, block inverses, node-to-row map,
// prescribed flags and vectors b, z, r (-1: not staged; the dense level
// stages only its rows, b and z), the bytes copied or zeroed for each, and
// the vectors' padding in elements.
struct MgStage {
  int off[8];
  int len[8];
  int vpad;
};
// A built hierarchy, for the V-cycle launches: levels 0..L-1 (the last
// dense); levels tail..L-1 (tail >= 1) run inside one kernel of one
// thread-block cluster of `cluster` blocks, the levels above it one launch
// per step.  Levels staged..L-1 (tail < staged; staged == L: none) are small
// enough for every block of the cluster to copy them into its shared memory
// (`smem` bytes, the dense inverse's `inv_len` bytes at `inv_off`) and run
// them in full by itself, between block barriers.
template <class T>
struct MgApply {
  MgLevel<T> lev[MG_MAX_LEVELS];
  int caps[MG_MAX_LEVELS];
  int L, tail, cluster;
  const float* invT;
  int staged, smem, inv_off, inv_len;
  MgStage stg[MG_MAX_LEVELS];
  // 2D levels above the tail: residual + restriction and prolongation +
  // first post-sweep as one tiled launch each (node-block smoother)
  int fused;
};
template <int D, class T, int B>
int mg_tail_cluster(bool* staging);
template <int D>
cudaError_t launch_mg_flags(int fx, int fy, int fz, const int* n2r_f, int cx, int cy, long long nc, int* flag,
                            cudaStream_t st);
template <int D, int B>
cudaError_t launch_mg_fixed(int fx, int fy, int fz, const int* n2r_f, const uint8_t* fix_f, int cx, int cy,
                            long long nc, uint8_t* fix_c, cudaStream_t st);
template <int D, class T, int B>
cudaError_t launch_mg_galerkin(MgLevel<T> f, MgLevel<T> c, int nrow_c, cudaStream_t st);
// power iteration on D^-1 A of a level: nrm[k] = ||v_k||^2 (v_k of unit
// predecessor), so sqrt(nrm[iters]) estimates lambda_max; va, vb scratch
// The power iterations for lambda_max(D^-1 A) of levels 0..n-1 at once
// (one launch per step): start vectors in va, scratch vb; start[] is filled
// by the launcher from the row capacities.
template <class T>
struct MgPowerSet {
  MgLevel<T> lev[MG_MAX_LEVELS];
  T* va[MG_MAX_LEVELS];
  T* vb[MG_MAX_LEVELS];
  int start[MG_MAX_LEVELS + 1];
  int n;
};
// blocks of one power-iteration launch over levels with row capacities caps[0..n-1]
int mg_power_blocks(const int* caps, int n);
// nrm: (iters + 1) norms per level; part: mg_power_blocks(caps, n) doubles;
// tickets: n counters, zero on entry and left zero
template <int D, class T, int B>
cudaError_t launch_mg_power(MgPowerSet<T> ps, const int* caps, double* nrm, int iters, double* part,
                            unsigned* tickets, cudaStream_t st);
template <class T>
cudaError_t launch_mg_scale(T* dinv, long long n, const double* nrm, double c, cudaStream_t st);
template <int D, class T, int B>
cudaError_t launch_mg_dense_inverse(MgLevel<T> c, float* invT, cudaStream_t st);
// z0 = V-cycle(b0) given the first smoothing sweep already in z0; levels
// 0..L-1, the last dense; kernels return at once while *done is set
template <int D, class T, int B>
cudaError_t launch_mg_vcycle(const MgApply<T>& mg, const T* b0, T* z0, const int* done, cudaStream_t st);
int mg_vcycle_launches(int L, int tail, int fused);
// z0 = M^-1 b0 outside a Krylov solve: the first finest-level sweep from the
// zero vector `zero` (padded, all zero), then the V-cycle
template <int D, class T, int B>
cudaError_t launch_mg_apply(const MgApply<T>& mg, const T* b0, const T* zero, T* z0, cudaStream_t st);

// device-pointer getters and Dirichlet setter (mpm_devio.cu)
cudaError_t launch_du_out(const double* du, double* out, long long ndof, int B, int D, double psc,
                          cudaStream_t st);
cudaError_t launch_residual_out(const double* r, const uint8_t* fixed, const int* node2row, double* out,
                                long long ndof, int B, int D, double psc, cudaStream_t st);
cudaError_t launch_positions_out(const DevParticles& P, int D, double* out, cudaStream_t st);
cudaError_t launch_dirichlet_in(int n, const long long* dof, const double* value, uint8_t* fixed, double* bcval,
                                long long ndof, int B, int D, double psc, int* bad, cudaStream_t st);

// Krylov
template <int D, class T>
struct KrylovVecs {
  T *x, *r, *rhat, *p, *phat, *v, *s, *shat, *t;
  double* red;   // reduction slots: 5 per block of the row grid (krylov_red_slots)
};
// slots of KrylovVecs::red for a matrix of row capacity cap
inline long long krylov_red_slots(long long cap) { return 5 * ((cap + KRYLOV_TPB - 1) / KRYLOV_TPB); }
template <int D, class T, int B = D>
cudaError_t launch_bicgstab_init(DevMatrix<T> K, const double* res, const uint8_t* fixed, KrylovVecs<D, T> v,
                                 KrylovScalars* S, double tol2, int maxit, int nblk, cudaStream_t st);
// one BiCGStab iteration; with `mg`, each preconditioner application is the
// V-cycle (the fused block-Jacobi step being its first smoothing sweep)
template <int D, class T, int B = D>
cudaError_t launch_bicgstab_iter(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                 int nblk, cudaStream_t st, const MgApply<T>* mg = nullptr);
template <int D, class T, int B = D>
cudaError_t launch_bicgstab_restart(const DevGrid& G, DevMatrix<T> K, const double* res, const uint8_t* fixed,
                                    KrylovVecs<D, T> v, KrylovScalars* S, double tol2, int maxit, int nblk,
                                    cudaStream_t st);
template <int D, class T, int B = D>
cudaError_t launch_update_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, double* du, int nblk,
                             cudaStream_t st);
template <int D, class T, int B = D>
cudaError_t launch_spmv(const DevGrid& G, DevMatrix<T> K, const T* x, T* y, int nblk, cudaStream_t st);
template <int D, class T, int B = D>
cudaError_t launch_step_du(DevMatrix<T> K, const T* x, const uint8_t* fixed, const double* base, double* du,
                           double alpha, int nblk, cudaStream_t st, const unsigned long long* absmax = nullptr,
                           double hlim = 0.0);
template <int D, class T, int B = D>
cudaError_t launch_absmax(DevMatrix<T> K, const T* x, const uint8_t* fixed, unsigned long long* out, int nblk,
                          cudaStream_t st);
// kernels launched by one scan_exclusive call of n elements
int scan_launches(long long n);
// persistent cooperative BiCGStab (one launch per solve); 0 blocks = unsupported
constexpr int PERSIST_MAX_BLOCKS = 1024;   // partial-sum slots per reduction
constexpr int PERSIST_BAR_WORDS = 1024;    // barrier tree counters (128-byte lines)
template <int D, class T>
int persistent_blocks(int device);
template <int D, class T>
cudaError_t launch_bicgstab_persistent(const DevGrid& G, DevMatrix<T> K, KrylovVecs<D, T> v, KrylovScalars* S,
                                       double* part, unsigned int* bar, int* err, int nblocks, cudaStream_t st);

// adjoint of a converged step (mpm_adjoint.cu)
template <int D, class T, int B>
cudaError_t launch_transpose_blocks(const DevGrid& G, DevMatrix<T> K, const int* node2row, T* out, int nrow,
                                    cudaStream_t st);
template <int D, int B>
cudaError_t launch_loss_p2g(const DevParticles& P, const DevGrid& G, const double* dLdx, double* g, int* err,
                            cudaStream_t st);
template <int D, int B>
cudaError_t launch_adjoint_rhs(const double* g, double* b, long long ndof, double psc, cudaStream_t st);
template <int D, int B>
cudaError_t launch_particle_increment(const DevParticles& P, const DevGrid& G, const double* U, double* out,
                                      int* err, cudaStream_t st);
template <int D, class T, int B>
cudaError_t launch_param_grad(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* U,
                              const T* mu, double psc, double* gE, double* gPhi, double* gK, int* err,
                              cudaStream_t st);

// reverse chain through load steps (mpm_adjoint_steps.cu); sbar: 19 per
// particle in caller order (x 3, b_e 6, p_c 1, F 9)
template <int D, class T, int B>
cudaError_t launch_adj_commit_vjp(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* grav,
                                  const double* U, double psc, const double* sbar, double* g, int* err,
                                  cudaStream_t st);
template <int D, class T, int B>
cudaError_t launch_adj_state_vjp(const DevParticles& P, const DevGrid& G, const MatC* mats, const double* grav,
                                 const double* U, const T* mu, double psc, const double* sbar, double* sbar_out,
                                 double* gE, double* gPhi, double* gK, int* err, cudaStream_t st);

// GMRES(m) with classical Gram-Schmidt applied twice
constexpr int GMRES_MMAX = 64;
struct GmresState {
  double H[(GMRES_MMAX + 1) * GMRES_MMAX];   // Hessenberg, column-major, leading dim MMAX+1
  double cs[GMRES_MMAX], sn[GMRES_MMAX], gv[GMRES_MMAX + 1], y[GMRES_MMAX];
  double h1[GMRES_MMAX + 1], h2[GMRES_MMAX + 1];  // projection accumulators of one step
  double wn2, wn2b, res, tol;
  int jdone, done, finished, status, iter, maxit;
};
template <class T>
struct GmresVecs {
  T* base;           // m+1 basis vectors, each `stride` elements, padded by `pad`
  long long stride, pad;
  T* w;              // Arnoldi work vector
  T* z;              // preconditioned basis vector
};
template <int D, class T, int B = D>
cudaError_t launch_gmres_begin(const DevGrid& G, DevMatrix<T> K, const double* res, const uint8_t* fixed,
                               GmresVecs<T> g, T* x, GmresState* st, int first, double tol, int maxit,
                               int nblk, cudaStream_t s);
template <int D, class T, int B = D>
cudaError_t launch_gmres_cycle(const DevGrid& G, DevMatrix<T> K, GmresVecs<T> g, T* x, GmresState* st, int m,
                               int nblk, cudaStream_t s);

}  // namespace mpm
