// C ABI of the implicit-MPM Newton step (declared in include/mpm.h): scene
// lifetime, the staged load step and its Newton loop (paper Sec. 2.2), and
// the getters used by tests and callers.  All device memory is owned by the
// scene; all work is stream-ordered on the scene's stream, with host
// synchronisation only where a scalar decides the control flow (active-row
// count, residual norm, Krylov done flag between graph chunks).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mpm.h"
#include "mpm_internal.h"

using namespace mpm;

namespace {
struct Fail {
  mpm_status st;
  std::string msg;
};
[[noreturn]] void fail(mpm_status st, const std::string& m) { throw Fail{st, m}; }
void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}
// Active nodes: nodal mass above this fraction of the largest particle mass
// (a node reached only by the far tail of a particle's B-spline, a distance t
// inside its support edge, has mass ~ t^2 m / 2 and stiffness ~ t^2 but moves
// the particle's dF at O(1): below t of about 0.014 such a node makes J
// nearly singular and stalls Newton; it is left out of the step instead).
constexpr double ACTIVE_REL = 1e-4;
constexpr int KTPB = KRYLOV_TPB;
constexpr int GRAPH_CHUNK = 8;   // Krylov iterations per graph launch
thread_local std::string g_create_err;  // message of the last failed mpm_create_scene
}  // namespace

struct mpm_scene {
  mpm_scene_desc desc{};
  int D = 2, B = 2, np = 0, nmat = 0, nbe = 4, nF = 4;
  bool mixed = false;
  bool up = false;          // coupled u-p: B = D + 1 values per node
  double psc = 1.0;         // u-p: pressure unknown / mass-balance row scale
  int seg = 1;              // rows per block-Jacobi block (1 node, 4 row segment)
  DevGrid G{};
  long long nnode = 0, ndof = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  MatC* d_mats = nullptr;
  std::vector<MatC> hmats;
  DevParticles P{}, Q{};   // live particle arrays and the gather target of the sort
  int *d_key = nullptr, *d_rank = nullptr, *d_perm = nullptr;
  int *d_count = nullptr, *d_cstart = nullptr, *d_flag = nullptr, *d_pos = nullptr;
  int *d_cells = nullptr, *d_node2row = nullptr, *d_rows = nullptr, *d_scan_tmp = nullptr;
  int *d_nrow = nullptr, *d_err = nullptr, *d_nplastic = nullptr;
  double *d_M = nullptr, *d_du = nullptr, *d_r = nullptr, *d_bcval = nullptr, *d_grav = nullptr,
         *d_norm = nullptr;
  const double* krhs = nullptr;   // right-hand side source of the Krylov solve (d_r or the adjoint's)
  uint8_t* d_fixed = nullptr;
  void* d_A = nullptr;
  // matrix (stencil-BSR), grown on demand
  void* d_K = nullptr;
  void* d_dinv = nullptr;
  int cap = 0;
  // Krylov vectors (BiCGStab: 9), padded
  void* d_vec = nullptr;
  long long vpad = 0, vlen = 0;   // padding and padded length in elements
  KrylovScalars* d_S = nullptr;
  KrylovScalars* h_S = nullptr;
  int* h_int = nullptr;           // pinned: ncell, nrow, err, nplastic
  double* h_dbl = nullptr;        // pinned: norm
  cudaGraphExec_t gexec = nullptr;
  bool use_graph = true;
  cudaEvent_t ev[6]{};
  // step state
  int nrow = 0, ncell = 0;
  bool staged = false;
  int k = 0;
  double r0 = 0, rk = 0, rprev = 0, eta_prev = 0.1;
  double grav[3] = {0, 0, 0};
  double mmax = 0;
  float t_asm = 0, t_kry = 0, t_res = 0;
  long long launches = 0;   // kernels launched by this scene
  long long halvings = 0;   // Newton steps halved after a return-map failure
  long long restarts = 0;   // BiCGStab restarts after a breakdown or the limit
  long long limited = 0;    // Newton corrections scaled by the step-length limit
  unsigned long long* d_absmax = nullptr;
  // GMRES(m)
  int gm = 0;
  void* d_gvec = nullptr;
  GmresState* d_gst = nullptr;
  char* h_gst = nullptr;              // pinned copy of the scalar tail of GmresState
  cudaGraphExec_t gexec_gm = nullptr;
  int gm_graph_cap = -1;
  double* d_duprev = nullptr;
  int pblocks = 0;          // co-resident blocks for the persistent Krylov kernel (0 = use graphs)
  unsigned int* d_bar = nullptr;   // barrier counter of the persistent kernel
  double* d_fail = nullptr;        // first constitutive failure record of a pass
  double* d_part = nullptr;        // per-block partial sums of its reductions
  void* d_KT = nullptr;            // adjoint: transposed Jacobian scratch
  unsigned* d_pmask = nullptr;     // per-row slot-presence bits of the Jacobian pattern
  double* d_red = nullptr;         // Krylov reduction slots (krylov_red_slots(cap))
  double* d_fp = nullptr;          // per-particle residual contributions (3^dim nodes x B per particle)
  double* d_norm_part = nullptr;   // residual-norm block sums (norm_part_slots(cap))
  unsigned* d_norm_ticket = nullptr;
  int* d_cellpos = nullptr;        // position of each occupied cell in d_cells (exclusive scan)
  void* d_cblk = nullptr;          // 3D assembly: 27 x 27 x 9 block values per occupied cell
  long long cblk_cap = 0;          // cells d_cblk has room for
  int kt_cap = -1;
  int adj_kit = 0;                 // Krylov iterations of the last adjoint solve
  // geometric multigrid preconditioner (MPM_PC_MG): levels 1.. of the
  // hierarchy (entry 0 unused: level 0 is the scene's own matrix)
  struct MgHost {
    int nx1 = 0, ny1 = 0, nz1 = 0;
    long long nnode = 0, vpad = 0, vlen = 0;
    int *node2row = nullptr, *rows = nullptr, *flag = nullptr, *pos = nullptr, *nrow_d = nullptr;
    uint8_t* fixed = nullptr;
    void *val = nullptr, *dinv = nullptr, *vec = nullptr;
    int cap = 0, nrow = 0;
  };
  bool mg = false;
  int mg_L = 0;                    // levels in use for the staged step (the last dense)
  std::vector<MgHost> mgl;
  void* d_mg_v0 = nullptr;         // level 0: residual and power-iteration scratch (2 vectors)
  float* d_mg_inv = nullptr;       // coarsest-level dense inverse, transposed
  double* d_mg_nrm = nullptr;      // power-iteration norms, MG_POWER_IT + 1 per level
  double* d_mg_part = nullptr;     // power-iteration partial sums, one per block of a launch
  int mg_part_n = 0;
  unsigned* d_mg_tickets = nullptr;   // power-iteration sums: one ticket per level
  int* d_mg_err = nullptr;         // singular coarse diagonal blocks (identity used)
  int* h_mgn = nullptr;            // pinned: active rows per level
  bool mg_lam = false;             // smoother damping estimated for the staged step
  std::vector<int> graph_sig;      // capacities the BiCGStab graph was captured with
  std::string err;

  // Device memory comes from the stream-ordered pool on the scene's stream:
  // unlike cudaMalloc/cudaFree it does not synchronise the device, so scenes
  // created and destroyed while others run (a serving loop) do not stall
  // them.  The stream is synchronised after each allocation so that the
  // memory is ready for copies issued on other streams.
  template <class T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    ck(cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st), "cudaMallocAsync");
    ck(cudaStreamSynchronize(st), "sync");
    allocs.push_back(p);
    return (T*)p;
  }
  void dfree(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) allocs.erase(it);
    cudaFreeAsync(p, st);
  }
};

namespace {

template <int D>
void pattern_mask(mpm_scene* s, std::vector<int>& mask);

size_t tsize(const mpm_scene* s) { return s->mixed ? 4 : 8; }

int stencil_slots(int D) { return D == 2 ? 25 : 125; }

mpm_status map_err_bits(int bits, std::string& msg) {
  if (bits & ERRF_BOUNDS) { msg = "a particle's B-spline support left the grid"; return MPM_ERR_BOUNDS; }
  if (bits & ERRF_RETURN) { msg = "return-map local Newton did not converge"; return MPM_ERR_RETURN_MAP; }
  if (bits & (ERRF_NONFINITE | ERRF_DET)) { msg = "non-finite value or non-positive det(F)"; return MPM_ERR_NONFINITE; }
  if (bits & ERRF_BARRIER) { msg = "grid barrier of the persistent Krylov kernel timed out"; return MPM_ERR_TIMEOUT; }
  return MPM_OK;
}

void validate_desc(const mpm_scene_desc* d) {
  if (!d) fail(MPM_ERR_INVALID_ARG, "desc is NULL");
  if (d->dim != 2 && d->dim != 3) fail(MPM_ERR_INVALID_ARG, "dim must be 2 or 3");
  for (int a = 0; a < d->dim; ++a)
    if (d->n[a] < 3) fail(MPM_ERR_INVALID_ARG, "need at least 3 cells per axis");
  if (!(d->h > 0)) fail(MPM_ERR_INVALID_ARG, "h must be positive");
  if (d->precision != MPM_FP64 && d->precision != MPM_MIXED) fail(MPM_ERR_INVALID_ARG, "bad precision");
  if (d->krylov != MPM_BICGSTAB && d->krylov != MPM_GMRES) fail(MPM_ERR_INVALID_ARG, "bad krylov");
  if (!(d->newton_tol > 0) || d->newton_maxit < 1 || d->newton_maxit > 32)
    fail(MPM_ERR_INVALID_ARG, "newton_tol > 0 and 1 <= newton_maxit <= 32 required");
  if (!(d->krylov_rtol > 0) || d->krylov_maxit < 1) fail(MPM_ERR_INVALID_ARG, "bad Krylov settings");
  if (d->formulation != MPM_SOLID && d->formulation != MPM_UP) fail(MPM_ERR_INVALID_ARG, "bad formulation");
  if (d->precond != MPM_PC_AUTO && d->precond != MPM_PC_NODE && d->precond != MPM_PC_SEG4 &&
      d->precond != MPM_PC_MG)
    fail(MPM_ERR_INVALID_ARG, "bad precond");
  if (d->precond == MPM_PC_MG && d->krylov != MPM_BICGSTAB)
    fail(MPM_ERR_INVALID_ARG, "the multigrid preconditioner is built for BiCGStab");
  if (d->jacobian_reuse < 0) fail(MPM_ERR_INVALID_ARG, "jacobian_reuse must be >= 0");
  if (d->formulation == MPM_UP) {
    if (d->dim != 2) fail(MPM_ERR_INVALID_ARG, "the u-p formulation is built for dim 2");
    if (!(d->dt > 0)) fail(MPM_ERR_INVALID_ARG, "u-p needs dt > 0");
    if (!(d->p_scale >= 0)) fail(MPM_ERR_INVALID_ARG, "p_scale must be >= 0");
  }
}

int dofs_per_node(const mpm_scene_desc* d) { return d->dim + (d->formulation == MPM_UP ? 1 : 0); }

long long nnode_of(const mpm_scene_desc* d) {
  long long c = 1;
  for (int a = 0; a < d->dim; ++a) c *= d->n[a] + 1;
  return c;
}

// Device bytes of a scene, excluding the matrix capacity growth margin.
size_t footprint(const mpm_scene_desc* d, int np) {
  const int D = d->dim, B = dofs_per_node(d), NPHI = D + (B > D ? 1 : 0);
  const size_t T = d->precision == MPM_MIXED ? 4 : 8;
  const long long nn = nnode_of(d), ndof = nn * B;
  const int nbe = D == 2 ? 4 : 6, nF = D * D;
  const int up_extra = (B > D) ? 2 : 0;   // kdt, pp
  size_t part = (size_t)np * (2 * (D + 2 + 2 + nbe + 1 + nF + up_extra) * 8 + 2 * 2 * 4 + 3 * 4 +
                              (D == 3 ? 27 : 9) * B * 8);   // + the residual contributions
  size_t grid = (size_t)nn * (7 * 4 + 8) + (size_t)ndof * (4 * 8 + 1);
  size_t tang = (size_t)np * B * NPHI * B * NPHI * T;
  long long pad = 2 + 2LL * (d->n[0] + 1) + (D == 3 ? 2LL * (d->n[0] + 1) * (d->n[1] + 1) : 0);
  size_t vec = 9 * (size_t)(nn + 2 * pad) * B * T;
  // GMRES(m): the m + 3 basis and work vectors beside the nine BiCGStab ones
  if (d->krylov == MPM_GMRES) {
    const int m = d->gmres_restart > 0 ? std::min(std::max(d->gmres_restart, 2), GMRES_MMAX) : 30;
    vec += (size_t)(m + 3) * (size_t)(nn + 2 * pad) * B * T;
  }
  // active rows are bounded by the nodes the particles can reach; the
  // block-Jacobi inverses take one B x B block per row, or four for the
  // 4-row segments (the u-p default); per row also the presence mask and
  // (under a byte) the Krylov reduction slots; in 3D the blocks of the
  // occupied cells (at most one per particle, 27 x 27 x 9 values each)
  long long rows = std::min<long long>(nn, (long long)np * (D == 2 ? 9 : 27));
  const int seg = (d->precond == MPM_PC_SEG4 || (d->precond == MPM_PC_AUTO && B > D)) ? 4 : 1;
  size_t mat = (size_t)rows * ((stencil_slots(D) + seg) * B * B * T + pmask_words(D) * 4 + 1);
  if (D == 3) mat += (size_t)std::min<long long>(nn, np) * CELL_BLOCK_VALUES * T + (size_t)nn * 4;
  // multigrid: coarse matrices (a quarter per level in 2D, an eighth in 3D),
  // coarse grids and vectors, two level-0 scratch vectors
  size_t mg = 0;
  if (d->precond == MPM_PC_MG) mg = mat / (D == 2 ? 3 : 7) + (size_t)nn * 12 + vec / 3 + (1 << 20);
  return part + grid + tang + vec + mat + mg + (1 << 20);
}

template <class T>
DevMatrix<T> matview(mpm_scene* s) {
  DevMatrix<T> K;
  K.val = (T*)s->d_K;
  K.pmask = s->d_pmask;
  K.dinv = (T*)s->d_dinv;
  K.cap = s->cap;
  K.rows = s->d_rows;
  K.nrow = s->d_nrow;
  K.seg = s->seg;
  return K;
}

template <int D, class T>
KrylovVecs<D, T> vecview(mpm_scene* s) {
  T* b = (T*)s->d_vec;
  KrylovVecs<D, T> v;
  T** f[9] = {&v.x, &v.r, &v.rhat, &v.p, &v.phat, &v.v, &v.s, &v.shat, &v.t};
  for (int k = 0; k < 9; ++k) *f[k] = b + k * s->vlen + s->vpad;
  v.red = s->d_red;
  return v;
}

void ensure_capacity(mpm_scene* s, int nrow) {
  if (nrow <= s->cap) return;
  int cap = std::max<int>(1024, (int)std::min<long long>(s->nnode, (long long)(nrow * 1.25) + 64));
  s->dfree(s->d_K);
  s->dfree(s->d_dinv);
  s->dfree(s->d_pmask);
  s->dfree(s->d_red);
  s->dfree(s->d_norm_part);
  s->d_K = nullptr;
  s->d_dinv = nullptr;
  s->d_pmask = nullptr;
  s->d_red = nullptr;
  s->d_norm_part = nullptr;
  const size_t S = stencil_slots(s->D), DD = (size_t)s->B * s->B;
  s->d_pmask = s->dalloc<unsigned>((size_t)cap * pmask_words(s->D));
  s->d_red = s->dalloc<double>((size_t)krylov_red_slots(cap));
  s->d_norm_part = s->dalloc<double>((size_t)norm_part_slots(cap));
  if (s->mixed) {
    s->d_K = s->dalloc<float>((size_t)cap * S * DD);
    s->d_dinv = s->dalloc<float>((size_t)(cap + 4) * DD * s->seg);
  } else {
    s->d_K = s->dalloc<double>((size_t)cap * S * DD);
    s->d_dinv = s->dalloc<double>((size_t)(cap + 4) * DD * s->seg);
  }
  s->cap = cap;
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  s->graph_sig.clear();
}

template <int D>
DevParticles make_particles(mpm_scene* s) {
  DevParticles P{};
  P.np = s->np;
  for (int a = 0; a < 3; ++a) P.x[a] = (a < D) ? s->dalloc<double>(s->np) : nullptr;
  P.vol0 = s->dalloc<double>(s->np);
  P.mass = s->dalloc<double>(s->np);
  P.mat = s->dalloc<int>(s->np);
  P.Ep = s->dalloc<double>(s->np);
  P.phip = s->dalloc<double>(s->np);
  for (int k = 0; k < MAX_BE; ++k) P.be[k] = (k < s->nbe) ? s->dalloc<double>(s->np) : nullptr;
  P.pc = s->dalloc<double>(s->np);
  for (int k = 0; k < MAX_F; ++k) P.F[k] = (k < s->nF) ? s->dalloc<double>(s->np) : nullptr;
  P.orig = s->dalloc<int>(s->np);
  P.kdt = s->up ? s->dalloc<double>(s->np) : nullptr;
  P.pp = s->up ? s->dalloc<double>(s->np) : nullptr;
  for (int a = 0; a < 3; ++a) P.fext[a] = nullptr;
  return P;
}

GatherArrays gather_list(mpm_scene* s, const DevParticles& src, DevParticles& dst) {
  GatherArrays g{};
  int nd = 0;
  for (int a = 0; a < s->D; ++a) { g.dsrc[nd] = src.x[a]; g.ddst[nd++] = dst.x[a]; }
  g.dsrc[nd] = src.vol0; g.ddst[nd++] = dst.vol0;
  g.dsrc[nd] = src.mass; g.ddst[nd++] = dst.mass;
  g.dsrc[nd] = src.Ep; g.ddst[nd++] = dst.Ep;
  g.dsrc[nd] = src.phip; g.ddst[nd++] = dst.phip;
  for (int k = 0; k < s->nbe; ++k) { g.dsrc[nd] = src.be[k]; g.ddst[nd++] = dst.be[k]; }
  g.dsrc[nd] = src.pc; g.ddst[nd++] = dst.pc;
  for (int k = 0; k < s->nF; ++k) { g.dsrc[nd] = src.F[k]; g.ddst[nd++] = dst.F[k]; }
  if (src.kdt) { g.dsrc[nd] = src.kdt; g.ddst[nd++] = dst.kdt; }
  if (src.pp) { g.dsrc[nd] = src.pp; g.ddst[nd++] = dst.pp; }
  for (int a = 0; a < s->D; ++a)
    if (src.fext[a]) { g.dsrc[nd] = src.fext[a]; g.ddst[nd++] = dst.fext[a]; }
  g.nd = nd;
  g.isrc[0] = src.mat; g.idst[0] = dst.mat;
  g.isrc[1] = src.orig; g.idst[1] = dst.orig;
  g.ni = 2;
  return g;
}

template <int D, class T, int B>
void launch_particle_pass(mpm_scene* s, int mode, int* nplastic) {
  if constexpr (B > D)
    ck(launch_particles_up<D, T>(s->P, s->G, s->d_mats, s->d_du, s->d_fp, s->d_grav, (T*)s->d_A, mode, s->psc,
                                 s->d_err, nplastic, s->st),
       "u-p particle kernel");
  else
    ck(launch_particles<D, T>(s->P, s->G, s->d_mats, s->d_du, s->d_fp, s->d_grav, (T*)s->d_A, mode, s->d_err,
                              nplastic, s->st),
       "particle kernel");
}

template <int D, class T, int B>
void residual_pass(mpm_scene* s, int mode) {
  ck(cudaMemsetAsync(s->d_nplastic, 0, sizeof(int), s->st), "memset");
  ck(cudaMemsetAsync(s->d_fail, 0, sizeof(double), s->st), "memset");
  launch_particle_pass<D, T, B>(s, mode, s->d_nplastic);
  // the residual of every node, added in a fixed order from the particles'
  // contributions
  ck(launch_gather_residual<D, B>(s->G, s->d_cstart, s->d_fp, s->np, s->d_r, s->nnode, s->st), "gather r");
  ck(launch_norm_free<B>(s->d_r, s->d_rows, s->nrow, s->d_fixed, s->d_norm, s->d_norm_part, s->d_norm_ticket,
                         s->st),
     "norm kernel");
  ck(cudaMemcpyAsync(s->h_dbl, s->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s->st), "copy norm");
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->st), "copy err");
  s->launches += 2;
}

void check_err_bits(mpm_scene* s) {
  std::string m;
  mpm_status st = map_err_bits(s->h_int[2], m);
  if (st == MPM_OK) return;
  if (s->h_int[2] & (ERRF_RETURN | ERRF_DET)) {
    double rec[FAIL_REC];
    if (cudaMemcpy(rec, s->d_fail, sizeof(rec), cudaMemcpyDeviceToHost) == cudaSuccess && rec[0] != 0.0) {
      char buf[320];
      snprintf(buf, sizeof(buf),
               " (first at particle %.0f: trial b eigenvalues %.17g %.17g %.17g, E %.17g, phi %.17g, pc %.17g, "
               "model %.0f)",
               rec[1], rec[2], rec[3], rec[4], rec[5], rec[6], rec[7], rec[8]);
      m += buf;
    }
  }
  fail(st, m);
}

template <int D, int B>
void mg_structure(mpm_scene* s);

template <int D, class T, int B>
void begin_step_impl(mpm_scene* s, mpm_newton_report* rep) {
  cudaStream_t st = s->st;
  const long long nn = s->nnode;
  s->staged = false;
  ck(cudaMemsetAsync(s->d_err, 0, sizeof(int), st), "memset");
  // a0: counting sort of particles by base cell
  ck(cudaMemsetAsync(s->d_count, 0, (nn + 1) * sizeof(int), st), "memset");
  ck(launch_cell_keys<D>(s->P, s->G, s->d_key, s->d_count, s->d_rank, s->d_err, st), "cell keys");
  ck(scan_exclusive(s->d_count, s->d_cstart, (int)(nn + 1), s->d_scan_tmp, st), "scan");
  ck(launch_sort_scatter(s->np, s->d_key, s->d_rank, s->d_cstart, s->d_perm, st), "scatter");
  ck(launch_sort_cells(s->d_cstart, s->d_perm, nn, st), "sort cells");
  GatherArrays g = gather_list(s, s->P, s->Q);
  ck(launch_gather(s->np, s->d_perm, g, st), "gather");
  std::swap(s->P, s->Q);
  // occupied cells
  ck(launch_flag_positive(s->d_count, s->d_flag, nn + 1, st), "flags");
  ck(scan_exclusive(s->d_flag, s->d_cellpos, (int)(nn + 1), s->d_scan_tmp, st), "scan");
  ck(launch_compact(s->d_flag, s->d_cellpos, s->d_cells, nn, st), "compact");
  ck(cudaMemcpyAsync(s->h_int + 0, s->d_cellpos + nn, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
  // nodal mass and active rows
  ck(launch_mass<D>(s->P, s->G, s->d_cstart, s->d_fp, s->d_M, nn, st), "mass");
  ck(cudaMemsetAsync(s->d_flag + nn, 0, sizeof(int), st), "memset");
  ck(launch_active(s->d_M, ACTIVE_REL * s->mmax, s->d_flag, nn, st), "active");
  ck(scan_exclusive(s->d_flag, s->d_pos, (int)(nn + 1), s->d_scan_tmp, st), "scan");
  ck(launch_node2row(s->d_flag, s->d_pos, s->d_node2row, s->d_rows, nn, st), "node2row");
  ck(cudaMemcpyAsync(s->d_nrow, s->d_pos + nn, sizeof(int), cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemcpyAsync(s->h_int + 1, s->d_pos + nn, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaStreamSynchronize(st), "sync");
  s->launches += 10 + 3LL * scan_launches(nn + 1);
  check_err_bits(s);
  s->ncell = s->h_int[0];
  s->nrow = s->h_int[1];
  ensure_capacity(s, s->nrow);
  ck(launch_pattern_bits<D>(s->G, s->d_rows, s->nrow, s->d_node2row, s->d_count, s->d_pmask, st),
     "pattern bits");
  s->launches += 1;
  if (D == 3 && s->ncell > s->cblk_cap) {
    s->dfree(s->d_cblk);
    s->d_cblk = nullptr;
    const long long cap = (long long)(s->ncell * 1.1) + 64;
    s->d_cblk = s->dalloc<unsigned char>((size_t)cap * CELL_BLOCK_VALUES * (s->mixed ? 4 : 8));
    s->cblk_cap = cap;
  }
  if (s->mg) mg_structure<D, B>(s);
  // prescribed increments and r^0 (with the tangent for the first iteration)
  ck(cudaMemcpyAsync(s->d_grav, s->grav, 3 * sizeof(double), cudaMemcpyHostToDevice, st), "grav");
  ck(launch_apply_bc(s->d_fixed, s->d_bcval, s->d_node2row, s->d_du, s->ndof, B, st), "bc");
  cudaEventRecord(s->ev[2], st);
  residual_pass<D, T, B>(s, 1);
  cudaEventRecord(s->ev[3], st);
  ck(cudaStreamSynchronize(st), "sync");
  check_err_bits(s);
  s->r0 = std::sqrt(s->h_dbl[0]);
  s->rk = s->r0;
  s->rprev = s->r0;
  s->eta_prev = 0.1;
  s->k = 0;
  s->staged = true;
  if (!std::isfinite(s->r0)) fail(MPM_ERR_NONFINITE, "non-finite initial residual");
  cudaEventElapsedTime(&s->t_res, s->ev[2], s->ev[3]);
  if (rep) {
    rep->status = MPM_OK;
    rep->krylov_iters = 0;
    rep->krylov_rel = 0;
    rep->krylov_rtol = 0;
    rep->r_norm = s->r0;
    rep->rel_residual = 1.0;
    rep->n_plastic = s->h_int[3];
  }
}

// ---- geometric multigrid hierarchy (csrc/mpm_mg.cu) ----------------------
// Grids of every coarse level, allocated with the scene (each level has about
// a quarter (2D) or an eighth (3D) of the nodes of the one above; coarsening
// stops when every axis has at most 2 nodes, at most 8 nodes in all).
void mg_create(mpm_scene* s) {
  s->mgl.assign(1, mpm_scene::MgHost{});
  int nx = s->G.nx1, ny = s->G.ny1, nz = s->G.nz1;
  const size_t T = tsize(s);
  while ((int)s->mgl.size() < MG_MAX_LEVELS && (nx > 2 || ny > 2 || (s->D == 3 && nz > 2))) {
    mpm_scene::MgHost m;
    m.nx1 = nx / 2 + 1;
    m.ny1 = ny / 2 + 1;
    m.nz1 = s->D == 3 ? nz / 2 + 1 : 1;
    m.nnode = (long long)m.nx1 * m.ny1 * m.nz1;
    m.node2row = s->dalloc<int>(m.nnode);
    m.rows = s->dalloc<int>(m.nnode);
    m.flag = s->dalloc<int>(m.nnode + 1);
    m.pos = s->dalloc<int>(m.nnode + 1);
    m.nrow_d = s->dalloc<int>(1);
    m.fixed = s->dalloc<uint8_t>((m.nnode * s->B + 15) & ~15LL);   // whole 16-byte units (tail staging)
    m.vpad = (2 + 2LL * m.nx1 + (s->D == 3 ? 2LL * m.nx1 * m.ny1 : 0)) * s->B;
    m.vlen = m.nnode * s->B + 2 * m.vpad;
    m.vec = s->mixed ? (void*)s->dalloc<float>(3 * m.vlen) : (void*)s->dalloc<double>(3 * m.vlen);
    ck(cudaMemsetAsync(m.vec, 0, 3 * m.vlen * T, s->st), "memset");
    ck(cudaMemsetAsync(m.nrow_d, 0, sizeof(int), s->st), "memset");
    s->mgl.push_back(m);
    nx = m.nx1;
    ny = m.ny1;
    nz = m.nz1;
  }
  s->d_mg_v0 = s->mixed ? (void*)s->dalloc<float>(2 * s->vlen) : (void*)s->dalloc<double>(2 * s->vlen);
  ck(cudaMemsetAsync(s->d_mg_v0, 0, 2 * s->vlen * T, s->st), "memset");
  s->d_mg_inv = s->dalloc<float>((size_t)MG_DENSE_MAX * MG_DENSE_MAX);
  s->d_mg_nrm = s->dalloc<double>((size_t)MG_MAX_LEVELS * (MG_POWER_IT + 1));
  s->d_mg_tickets = s->dalloc<unsigned>(MG_MAX_LEVELS);
  ck(cudaMemsetAsync(s->d_mg_tickets, 0, MG_MAX_LEVELS * sizeof(unsigned), s->st), "memset");
  s->d_mg_err = s->dalloc<int>(1);
  ck(cudaMallocHost(&s->h_mgn, MG_MAX_LEVELS * sizeof(int)), "host alloc");
}

// Active nodes and prescribed DOFs of every coarse level for the staged step
// (after the fine rows and prescribed DOFs are set); the hierarchy in use ends
// at the first level with at most MG_DENSE_MAX unknowns.
template <int D, int B>
void mg_structure(mpm_scene* s) {
  cudaStream_t st = s->st;
  const int Lmax = (int)s->mgl.size();
  int fx = s->G.nx1, fy = s->G.ny1, fz = s->G.nz1;
  const int* n2r = s->d_node2row;
  const uint8_t* fix = s->d_fixed;
  for (int l = 1; l < Lmax; ++l) {
    auto& m = s->mgl[l];
    ck(launch_mg_flags<D>(fx, fy, fz, n2r, m.nx1, m.ny1, m.nnode, m.flag, st), "mg flags");
    ck(scan_exclusive(m.flag, m.pos, (int)(m.nnode + 1), s->d_scan_tmp, st), "mg scan");
    ck(launch_node2row(m.flag, m.pos, m.node2row, m.rows, m.nnode, st), "mg rows");
    ck(cudaMemcpyAsync(m.nrow_d, m.pos + m.nnode, sizeof(int), cudaMemcpyDeviceToDevice, st), "copy");
    ck(cudaMemcpyAsync(s->h_mgn + l, m.pos + m.nnode, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    ck(launch_mg_fixed<D, B>(fx, fy, fz, n2r, fix, m.nx1, m.ny1, m.nnode, m.fixed, st), "mg fixed");
    s->launches += 3 + scan_launches(m.nnode + 1);
    fx = m.nx1;
    fy = m.ny1;
    fz = m.nz1;
    n2r = m.node2row;
    fix = m.fixed;
  }
  ck(cudaStreamSynchronize(st), "sync");
  s->h_mgn[0] = s->nrow;
  int L = 0;
  for (int l = 0; l < Lmax && L == 0; ++l)
    if ((long long)s->h_mgn[l] * B <= MG_DENSE_MAX) L = l + 1;
  if (L == 0) fail(MPM_ERR_INVALID_ARG, "grid too large for the multigrid hierarchy");
  const size_t S = stencil_slots(D), BB = (size_t)B * B;
  for (int l = 1; l < L; ++l) {
    auto& m = s->mgl[l];
    m.nrow = s->h_mgn[l];
    if (m.nrow > m.cap || !m.val) {
      const int cap = (int)std::min<long long>(m.nnode, std::max<long long>(64, (long long)(m.nrow * 1.25) + 32));
      s->dfree(m.val);
      s->dfree(m.dinv);
      if (s->mixed) {
        m.val = s->dalloc<float>((size_t)cap * S * BB);
        m.dinv = s->dalloc<float>((size_t)(cap + 4) * BB);
      } else {
        m.val = s->dalloc<double>((size_t)cap * S * BB);
        m.dinv = s->dalloc<double>((size_t)(cap + 4) * BB);
      }
      m.cap = cap;
    }
  }
  s->mg_L = L;
  s->mg_lam = false;
}

template <class T>
MgApply<T> mg_view(mpm_scene* s) {
  MgApply<T> a{};
  a.L = s->mg_L;
  a.invT = s->d_mg_inv;
  MgLevel<T>& f = a.lev[0];
  f.nx1 = s->G.nx1;
  f.ny1 = s->G.ny1;
  f.nz1 = s->G.nz1;
  f.K = matview<T>(s);
  f.node2row = s->d_node2row;
  f.fixed = s->d_fixed;
  f.b = nullptr;
  f.z = (T*)s->d_mg_v0 + s->vlen + s->vpad;   // smoothing scratch
  f.r = (T*)s->d_mg_v0 + s->vpad;
  a.caps[0] = s->cap;
  // cluster tail: from the first coarse level with at most MG_TAIL_ROWS rows
  a.tail = std::max(a.L - 1, 1);
  for (int l = 1; l < a.L; ++l)
    if (s->h_mgn[l] <= MG_TAIL_ROWS) {
      a.tail = l;
      break;
    }
  for (int l = 1; l < a.L; ++l) {
    const auto& m = s->mgl[l];
    MgLevel<T>& c = a.lev[l];
    c.nx1 = m.nx1;
    c.ny1 = m.ny1;
    c.nz1 = m.nz1;
    c.K.val = (T*)m.val;
    c.K.pmask = nullptr;   // coarse levels: every slot read
    c.K.dinv = (T*)m.dinv;
    c.K.cap = m.cap;
    c.K.rows = m.rows;
    c.K.nrow = m.nrow_d;
    c.K.seg = 1;
    c.node2row = m.node2row;
    c.fixed = m.fixed;
    T* v = (T*)m.vec;
    c.b = v + m.vpad;
    c.z = v + m.vlen + m.vpad;
    c.r = v + 2 * m.vlen + m.vpad;
    a.caps[l] = m.cap;
  }
  a.fused = (s->D == 2 && a.lev[0].K.seg == 1 && MG_NU0 >= 2) ? 1 : 0;
  // coarse levels the tail stages in shared memory: from the first level
  // below the tail from which all levels down to the dense one fit
  a.staged = a.L;
  a.smem = a.inv_off = a.inv_len = 0;
  const int l0 = std::min(std::max(a.tail, 1), a.L - 1);
  const size_t TS = sizeof(T), BB = (size_t)s->B * s->B, S = stencil_slots(s->D);
  const auto al16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  for (int ls = l0 + 1; ls <= a.L - 1; ++ls) {
    MgStage stg[MG_MAX_LEVELS] = {};
    size_t off = 0;
    for (int l = ls; l < a.L && off <= (size_t)MG_TAIL_SMEM_MAX; ++l) {
      const auto& m = s->mgl[l];
      const bool dense = (l == a.L - 1);
      const size_t vb = (size_t)m.vlen * TS;
      // rows, blocks, block inverses, node-to-row map, prescribed flags, b, z, r
      const size_t len[8] = {(size_t)m.cap * 4,
                             dense ? 0 : S * (size_t)m.cap * BB * TS,
                             dense ? 0 : (size_t)m.cap * BB * TS,
                             dense ? 0 : (size_t)m.nnode * 4,
                             dense ? 0 : al16((size_t)m.nnode * s->B),
                             vb,
                             vb,
                             dense ? 0 : vb};
      for (int k = 0; k < 8; ++k) {
        stg[l].off[k] = len[k] ? (int)std::min(off, (size_t)MG_TAIL_SMEM_MAX) : -1;
        stg[l].len[k] = (int)std::min(len[k], (size_t)MG_TAIL_SMEM_MAX);
        off += al16(len[k]);
      }
      stg[l].vpad = (int)m.vpad;
    }
    const size_t nd = (size_t)std::min(s->mgl[a.L - 1].cap * s->B, MG_DENSE_MAX);
    const size_t inv = nd * nd * sizeof(float);
    if (off + al16(inv) <= (size_t)MG_TAIL_SMEM_MAX) {
      a.staged = ls;
      a.inv_off = (int)off;
      a.inv_len = (int)inv;
      a.smem = (int)(off + al16(inv));
      for (int l = ls; l < a.L; ++l) a.stg[l] = stg[l];
      break;
    }
  }
  return a;
}

// smoother damping w = MG_DAMP / lambda_max(D^-1 A), per level
constexpr double MG_DAMP = 1.2;
// BiCGStab iterations per graph launch with the V-cycle (a few iterations
// per solve: a long chunk would launch many early-returning kernels)
constexpr int MG_CHUNK = 2;

// Coarse operators, their block inverses, the smoother damping (estimated at
// the first assembly of a load step) and the coarsest dense inverse, from the
// assembled level-0 matrix and its block-Jacobi inverse.
template <int D, class T, int B>
void mg_setup(mpm_scene* s) {
  if (!s->mg || s->mg_L == 0 || s->nrow == 0) return;
  cudaStream_t st = s->st;
  MgApply<T> a = mg_view<T>(s);
  const int L = a.L;
  for (int l = 1; l < L; ++l) {
    ck(launch_mg_galerkin<D, T, B>(a.lev[l - 1], a.lev[l], s->h_mgn[l], st), "galerkin");
    s->launches += 1;
    if (l + 1 < L) {
      ck(launch_block_jacobi<D, T, B>(s->G, a.lev[l].K, s->h_mgn[l], s->d_mg_err, st), "coarse block jacobi");
      s->launches += 1;
    }
  }
  const int P1 = MG_POWER_IT + 1;
  if (!s->mg_lam) {
    MgPowerSet<T> ps{};
    ps.n = L - 1;
    for (int l = 0; l + 1 < L; ++l) {
      ps.lev[l] = a.lev[l];
      ps.va[l] = (l == 0) ? (T*)s->d_mg_v0 + s->vpad : a.lev[l].b;
      ps.vb[l] = (l == 0) ? (T*)s->d_mg_v0 + s->vlen + s->vpad : a.lev[l].z;
    }
    const int nb = mg_power_blocks(a.caps, ps.n);
    if (nb > s->mg_part_n) {
      s->dfree(s->d_mg_part);
      s->d_mg_part = s->dalloc<double>((size_t)nb);
      s->mg_part_n = nb;
    }
    ck(launch_mg_power<D, T, B>(ps, a.caps, s->d_mg_nrm, MG_POWER_IT, s->d_mg_part, s->d_mg_tickets, st), "power");
    if (ps.n > 0) s->launches += 1 + MG_POWER_IT;
    s->mg_lam = true;
  }
  for (int l = 0; l + 1 < L; ++l) {
    const long long n = (long long)(a.caps[l] + 4) * B * B * (l == 0 ? s->seg : 1);
    ck(launch_mg_scale<T>(a.lev[l].K.dinv, n, s->d_mg_nrm + l * P1 + MG_POWER_IT, MG_DAMP, st), "scale");
    s->launches += 1;
  }
  ck(launch_mg_dense_inverse<D, T, B>(a.lev[L - 1], s->d_mg_inv, st), "dense inverse");
  s->launches += 1;
}

// z = M^-1 b with the hierarchy of the last assembly (host vectors of ndof
// doubles, rounded to T on the way in); scratch vectors of the padded
// level-0 layout are allocated for the call
template <int D, class T, int B>
void mg_apply_impl(mpm_scene* s, const double* b, double* z) {
  if (!s->mg || s->mg_L == 0 || s->nrow == 0)
    fail(MPM_ERR_STATE, "no multigrid hierarchy (MPM_PC_MG, after an assembly)");
  cudaStream_t st = s->st;
  MgApply<T> mga = mg_view<T>(s);
  bool staging = false;
  mga.cluster = mg_tail_cluster<D, T, B>(&staging);
  if (!staging) mga.staged = mga.L;
  std::vector<T> h((size_t)s->ndof);
  for (long long d = 0; d < s->ndof; ++d) h[d] = (T)b[d];
  T* v = s->dalloc<T>(3 * (size_t)s->vlen);
  ck(cudaMemsetAsync(v, 0, 3 * (size_t)s->vlen * sizeof(T), st), "memset");
  T* vb = v + s->vpad;
  T* vzero = v + s->vlen + s->vpad;
  T* vz = v + 2 * s->vlen + s->vpad;
  ck(cudaMemcpyAsync(vb, h.data(), (size_t)s->ndof * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
  ck(launch_mg_apply<D, T, B>(mga, vb, vzero, vz, st), "v-cycle");
  s->launches += (mga.L >= 2 ? 1 : 0) + mg_vcycle_launches(mga.L, mga.tail, mga.fused);
  ck(cudaMemcpyAsync(h.data(), vz, (size_t)s->ndof * sizeof(T), cudaMemcpyDeviceToHost, st), "download");
  ck(cudaStreamSynchronize(st), "sync");
  s->dfree(v);
  for (long long d = 0; d < s->ndof; ++d) z[d] = (double)h[d];
}

template <int D, class T, int B>
void build_graph(mpm_scene* s, int nblk, const MgApply<T>* mg, int chunk, const std::vector<int>& sig) {
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  cudaGraph_t g;
  ck(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal), "capture");
  DevMatrix<T> K = matview<T>(s);
  KrylovVecs<D, T> v = vecview<D, T>(s);
  for (int c = 0; c < chunk; ++c) launch_bicgstab_iter<D, T, B>(s->G, K, v, s->d_S, nblk, s->st, mg);
  ck(cudaStreamEndCapture(s->st, &g), "end capture");
  ck(cudaGraphInstantiate(&s->gexec, g, 0), "instantiate");
  cudaGraphDestroy(g);
  s->graph_sig = sig;
}


// Assembly of the per-particle consistent tangents (written by the last
// residual pass) into the stencil-BSR Jacobian, prescribed rows/columns set
// to the identity, block-Jacobi inverse.
template <int D, class T, int B>
void assemble_impl(mpm_scene* s, bool with_mg = true) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged (call mpm_begin_step)");
  cudaStream_t st = s->st;
  DevMatrix<T> K = matview<T>(s);
  // every block of every active row is stored by the assembly (no zero fill)
  const Asm3<T> a3{s->d_cells, s->ncell, s->d_count, s->d_cellpos, (T*)s->d_cblk};
  ck(launch_assemble<D, T, B>(s->P, s->G, s->d_cstart, s->d_node2row, (const T*)s->d_A, K, s->nrow, &a3, st),
     "assemble");
  ck(launch_bc_matrix<D, T, B>(s->G, K, s->d_fixed, s->d_node2row, s->nrow, st), "bc matrix");
  ck(launch_block_jacobi<D, T, B>(s->G, K, s->nrow, s->d_err, st), "block jacobi");
  s->launches += 3;
  if (with_mg) mg_setup<D, T, B>(s);
}

// Restarted GMRES(m) on J d = -r to an absolute residual `tol`: cycles of m
// Arnoldi steps (one CUDA graph per cycle), polled once per cycle.
template <int D, class T, int B>
void gmres_solve(mpm_scene* s, DevMatrix<T> K, T* x, double tol, int nblk, int& kit, int& kstat, double& kres2) {
  cudaStream_t st = s->st;
  T* base = (T*)s->d_gvec;
  GmresVecs<T> g;
  g.base = base;
  g.stride = s->vlen;
  g.pad = s->vpad;
  g.w = base + (long long)(s->gm + 1) * s->vlen + s->vpad;
  g.z = base + (long long)(s->gm + 2) * s->vlen + s->vpad;
  if (s->use_graph && s->gm_graph_cap != s->cap) {
    if (s->gexec_gm) {
      cudaGraphExecDestroy(s->gexec_gm);
      s->gexec_gm = nullptr;
    }
    cudaGraph_t gr;
    ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture");
    launch_gmres_cycle<D, T, B>(s->G, K, g, x, s->d_gst, s->gm, nblk, st);
    ck(cudaStreamEndCapture(st, &gr), "end capture");
    ck(cudaGraphInstantiate(&s->gexec_gm, gr, 0), "instantiate");
    cudaGraphDestroy(gr);
    s->gm_graph_cap = s->cap;
  }
  const size_t tail = offsetof(GmresState, wn2);
  const size_t tail_bytes = sizeof(GmresState) - tail;
  GmresState* h = (GmresState*)(s->h_gst - tail);   // fields from wn2 on are valid
  for (int cycle = 0;; ++cycle) {
    ck(launch_gmres_begin<D, T, B>(s->G, K, s->krhs, s->d_fixed, g, x, s->d_gst, cycle == 0 ? 1 : 0, tol,
                                s->desc.krylov_maxit, nblk, st),
       "gmres begin");
    s->launches += 3;
    if (s->use_graph) ck(cudaGraphLaunch(s->gexec_gm, st), "graph launch");
    else ck(launch_gmres_cycle<D, T, B>(s->G, K, g, x, s->d_gst, s->gm, nblk, st), "gmres cycle");
    s->launches += 4LL * s->gm + 2;
    ck(cudaMemcpyAsync(s->h_gst, (char*)s->d_gst + tail, tail_bytes, cudaMemcpyDeviceToHost, st), "copy");
    ck(cudaStreamSynchronize(st), "sync");
    if (h->finished || h->iter >= s->desc.krylov_maxit || cycle > s->desc.krylov_maxit) break;
  }
  kit = h->iter;
  kstat = h->status;
  kres2 = h->res * h->res;
}

// Krylov solve of J x = -b on the free DOFs (b = s->krhs, by default the
// residual) to the absolute tolerance eta * rnorm; x is left in the Krylov
// vector x.  BiCGStab (graph chunks or the persistent kernel) or GMRES(m).
template <int D, class T, int B>
void krylov_solve(mpm_scene* s, double eta, double rnorm, int& kit, int& kstat, double& kres2) {
  cudaStream_t st = s->st;
  DevMatrix<T> K = matview<T>(s);
  const int nblk = (s->cap + KTPB - 1) / KTPB;
  KrylovVecs<D, T> v = vecview<D, T>(s);
  double tol2 = eta * eta * rnorm * rnorm;
  kit = 0;
  kstat = 0;
  kres2 = 0.0;
  if (s->gm > 0) {
    gmres_solve<D, T, B>(s, K, v.x, eta * rnorm, nblk, kit, kstat, kres2);
  } else {
  const bool use_mg = s->mg && s->mg_L > 0;
  MgApply<T> mga{};
  if (use_mg) {
    mga = mg_view<T>(s);
    bool staging = false;
    mga.cluster = mg_tail_cluster<D, T, B>(&staging);
    if (!staging) mga.staged = mga.L;
  }
  const MgApply<T>* mgp = use_mg ? &mga : nullptr;
  int* d_done = &s->d_S->done;
  const int chunk = use_mg ? MG_CHUNK : GRAPH_CHUNK;
  const int per_iter = 4 + (use_mg ? 2 * mg_vcycle_launches(mga.L, mga.tail, mga.fused) : 0);
  ck(launch_bicgstab_init<D, T, B>(K, s->krhs, s->d_fixed, v, s->d_S, tol2, s->desc.krylov_maxit, nblk, st),
     "krylov init");
  if (use_mg) {
    ck(launch_mg_vcycle<D, T, B>(mga, v.p, v.phat, d_done, st), "v-cycle");
    s->launches += mg_vcycle_launches(mga.L, mga.tail, mga.fused);
  }
  const int pblk = std::min(s->pblocks, std::max(1, (s->nrow * 4 + 511) / 512));
  if (s->pblocks > 0) {
    // whole solve in one cooperative launch
    if constexpr (B == D)
      ck(launch_bicgstab_persistent<D, T>(s->G, K, v, s->d_S, s->d_part, s->d_bar, s->d_err, pblk, st),
         "persistent krylov");
    s->launches += 1;
    ck(cudaMemcpyAsync(s->h_S, s->d_S, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st), "copy S");
    ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
    ck(cudaStreamSynchronize(st), "sync");
    check_err_bits(s);
  }
  std::vector<int> sig = {s->cap, use_mg ? s->mg_L : 0, use_mg ? mga.tail : 0, use_mg ? mga.cluster : 0};
  if (use_mg)
    for (int l = 1; l < s->mg_L; ++l) sig.push_back(s->mgl[l].cap);
  if (s->pblocks == 0 && s->use_graph && sig != s->graph_sig) build_graph<D, T, B>(s, nblk, mgp, chunk, sig);
  if (s->pblocks == 0) {
    // graph chunks of GRAPH_CHUNK iterations until the done flag; on a
    // (near) breakdown or the iteration limit, restart from the current x
    // with the true residual b - J x (at most 3 restarts)
    for (int restart = 0;; ++restart) {
      int launched = 0;
      for (;;) {
        if (s->use_graph) {
          ck(cudaGraphLaunch(s->gexec, st), "graph launch");
        } else {
          for (int c = 0; c < chunk; ++c)
            ck(launch_bicgstab_iter<D, T, B>(s->G, K, v, s->d_S, nblk, st, mgp), "krylov");
        }
        launched += chunk;
        s->launches += (long long)per_iter * chunk;
        ck(cudaMemcpyAsync(s->h_S, s->d_S, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st), "copy S");
        ck(cudaStreamSynchronize(st), "sync");
        if (s->h_S->done) break;
        if (launched > s->desc.krylov_maxit + 2 * chunk) break;   // belt and braces
      }
      kit += s->h_S->iter;
      kstat = s->h_S->status;
      if (restart >= 3 || kit >= s->desc.krylov_maxit) break;
      // restart from the true residual b - J x; when the recurrence reported
      // convergence this also checks it (the recurrence residual can drift
      // from the true one on ill-conditioned systems such as u-p)
      ck(launch_bicgstab_restart<D, T, B>(s->G, K, s->krhs, s->d_fixed, v, s->d_S, tol2,
                                       s->desc.krylov_maxit - kit, nblk, st),
         "krylov restart");
      s->launches += 1;
      ck(cudaMemcpyAsync(s->h_S, s->d_S, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st), "copy S");
      ck(cudaStreamSynchronize(st), "sync");
      if (kstat == 0 && s->h_S->rr_last <= 4.0 * tol2) break;   // true residual within 2x of the tolerance
      kstat = 0;
      s->restarts += 1;
      // the restart's search direction, preconditioned by the V-cycle (the
      // restart kernel applied only its first smoothing sweep)
      if (use_mg) {
        ck(launch_mg_vcycle<D, T, B>(mga, v.p, v.phat, d_done, st), "v-cycle");
        s->launches += mg_vcycle_launches(mga.L, mga.tail, mga.fused);
      }
    }
  } else {
    kit = s->h_S->iter;
    kstat = s->h_S->status;
  }
  kres2 = s->h_S->rr_last;
  }
}

template <int D, class T, int B>
void newton_impl(mpm_scene* s, mpm_newton_report* rep) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged (call mpm_begin_step)");
  cudaStream_t st = s->st;
  DevMatrix<T> K = matview<T>(s);
  cudaEventRecord(s->ev[0], st);
  // modified Newton (jacobian_reuse = k > 1): the Jacobian of the load
  // step's iteration 0, k, 2k, ... serves the iterations after it
  const int reuse = s->desc.jacobian_reuse;
  if (reuse <= 1 || s->k % reuse == 0) assemble_impl<D, T, B>(s);
  // linear tolerance: fixed, or Eisenstat-Walker choice 2 (gamma 0.9,
  // alpha 2) capped at ETA_MAX = 1e-2: with the classical cap of 0.1 loose
  // steps through the plastic zone made Newton diverge on footing problems.
  double eta = s->desc.krylov_rtol;
  if (s->desc.forcing == MPM_FORCING_EW) {
    constexpr double ETA_MAX = 1e-2;
    if (s->k == 0) {
      eta = ETA_MAX;
    } else {
      double ratio = s->rk / s->rprev;
      eta = 0.9 * ratio * ratio;
      double safe = 0.9 * s->eta_prev * s->eta_prev;
      if (safe > 0.1) eta = std::max(eta, safe);
    }
    // no need to solve below what the Newton tolerance asks of this step
    eta = std::max(eta, 0.5 * s->desc.newton_tol * s->r0 / std::max(s->rk, 1e-300));
    eta = std::min(std::max(eta, s->desc.krylov_rtol), ETA_MAX);
  }
  s->eta_prev = eta;
  const int nblk = (s->cap + KTPB - 1) / KTPB;
  cudaEventRecord(s->ev[1], st);
  KrylovVecs<D, T> v = vecview<D, T>(s);
  int kit = 0, kstat = 0;
  double kres2 = 0.0;
  krylov_solve<D, T, B>(s, eta, s->rk, kit, kstat, kres2);
  const double krel = (s->rk > 0) ? std::sqrt(std::max(kres2, 0.0)) / s->rk : 0.0;
  // step-length limit (reading): a Newton correction that would move a node
  // by more than one cell width h is scaled down to h (a near-singular J, as
  // at the onset of a mechanism, otherwise yields astronomically large steps)
  // (the limit is applied on the device by the update kernel; the host reads
  // max |d| back with the new residual norm, without a synchronisation of its own)
  ck(launch_absmax<D, T, B>(K, v.x, s->d_fixed, s->d_absmax, nblk, st), "absmax");
  ck(cudaMemcpyAsync(s->d_duprev, s->d_du, s->ndof * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy du");
  ck(launch_step_du<D, T, B>(K, v.x, s->d_fixed, s->d_duprev, s->d_du, 1.0, nblk, st, s->d_absmax, s->G.h),
     "update");
  ck(cudaMemcpyAsync(s->h_dbl + 2, s->d_absmax, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
  s->launches += 3;   // Krylov init + absmax + update
  cudaEventRecord(s->ev[2], st);
  residual_pass<D, T, B>(s, 1);
  cudaEventRecord(s->ev[3], st);
  ck(cudaStreamSynchronize(st), "sync");
  const double xmax = s->h_dbl[2];
  const bool limited = !std::isfinite(xmax) || xmax > s->G.h;
  if (limited) s->limited += 1;
  // a full step that drives a return map out of its domain (or to a
  // non-finite state), or that does not decrease ||r|| while ||r|| is still
  // well above the tolerance (a backtracking line search on the residual
  // norm, for the non-smooth plastic branches), is halved, at most four times;
  // the last halving is taken whatever its residual
  auto need_halving = [&]() {
    if (s->h_int[2] & (ERRF_RETURN | ERRF_NONFINITE | ERRF_DET)) return true;
    const double rnew = std::sqrt(s->h_dbl[0]);
    return !(rnew < (1.0 - 1e-4) * s->rk) && s->rk > 10.0 * s->desc.newton_tol * s->r0;
  };
  for (int half = 1; half <= 4 && need_halving(); ++half) {
    ck(cudaMemsetAsync(s->d_err, 0, sizeof(int), st), "memset");
    ck(launch_step_du<D, T, B>(K, v.x, s->d_fixed, s->d_duprev, s->d_du, std::ldexp(1.0, -half), nblk, st,
                               s->d_absmax, s->G.h),
       "step");
    s->launches += 1;
    residual_pass<D, T, B>(s, 1);
    cudaEventRecord(s->ev[3], st);
    ck(cudaStreamSynchronize(st), "sync");
    s->halvings += 1;
  }
  check_err_bits(s);
  cudaEventElapsedTime(&s->t_asm, s->ev[0], s->ev[1]);
  cudaEventElapsedTime(&s->t_kry, s->ev[1], s->ev[2]);
  cudaEventElapsedTime(&s->t_res, s->ev[2], s->ev[3]);
  s->rprev = s->rk;
  s->rk = std::sqrt(s->h_dbl[0]);
  s->k += 1;
  if (!std::isfinite(s->rk)) fail(MPM_ERR_NONFINITE, "non-finite residual");
  if (rep) {
    rep->status = kstat == 0 ? MPM_OK : (kstat == 1 ? MPM_ERR_KRYLOV_MAXIT : MPM_ERR_KRYLOV_BREAKDOWN);
    rep->krylov_iters = kit;
    rep->krylov_rel = krel;
    rep->krylov_rtol = eta;
    rep->r_norm = s->rk;
    rep->rel_residual = (s->r0 > 0) ? s->rk / s->r0 : 0.0;
    rep->n_plastic = s->h_int[3];
  }
}

template <int D, class T, int B>
void set_du_impl(mpm_scene* s, const double* du) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged (call mpm_begin_step)");
  std::vector<double> h(du, du + s->ndof);
  if (B > D)
    for (long long d = D; d < s->ndof; d += B) h[d] /= s->psc;
  std::vector<uint8_t> f(s->ndof);
  std::vector<double> bc(s->ndof);
  std::vector<int> n2r(s->nnode);
  ck(cudaStreamSynchronize(s->st), "sync");
  ck(cudaMemcpy(f.data(), s->d_fixed, s->ndof, cudaMemcpyDeviceToHost), "download");
  ck(cudaMemcpy(bc.data(), s->d_bcval, s->ndof * sizeof(double), cudaMemcpyDeviceToHost), "download");
  ck(cudaMemcpy(n2r.data(), s->d_node2row, s->nnode * sizeof(int), cudaMemcpyDeviceToHost), "download");
  for (long long d = 0; d < s->ndof; ++d)
    if (f[d] && n2r[d / B] >= 0) h[d] = bc[d];
  ck(cudaMemcpy(s->d_du, h.data(), s->ndof * sizeof(double), cudaMemcpyHostToDevice), "upload");
  residual_pass<D, T, B>(s, 1);
  ck(cudaStreamSynchronize(s->st), "sync");
  check_err_bits(s);
  s->rk = std::sqrt(s->h_dbl[0]);
}

template <int D, class T, int B>
void commit_impl(mpm_scene* s) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged");
  launch_particle_pass<D, T, B>(s, 2, nullptr);
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st), "copy");
  ck(cudaStreamSynchronize(s->st), "sync");
  s->launches += 1;
  check_err_bits(s);
  s->staged = false;
}

template <int D, class T, int B>
void time_spmv_impl(mpm_scene* s, int reps, double* ms, double* bytes) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged");
  if (reps < 1) fail(MPM_ERR_INVALID_ARG, "reps must be positive");
  DevMatrix<T> K = matview<T>(s);
  KrylovVecs<D, T> v = vecview<D, T>(s);
  const int nblk = (s->cap + KTPB - 1) / KTPB;
  ck(launch_spmv<D, T, B>(s->G, K, v.phat, v.v, nblk, s->st), "spmv");   // warm-up
  ck(cudaEventRecord(s->ev[4], s->st), "event");
  for (int k = 0; k < reps; ++k) ck(launch_spmv<D, T, B>(s->G, K, v.phat, v.v, nblk, s->st), "spmv");
  ck(cudaEventRecord(s->ev[5], s->st), "event");
  ck(cudaEventSynchronize(s->ev[5]), "sync");
  float t = 0;
  ck(cudaEventElapsedTime(&t, s->ev[4], s->ev[5]), "elapsed");
  s->launches += reps + 1;
  *ms = t / reps;
  long long nnzb = 0;
  {
    std::vector<int> mask;
    pattern_mask<D>(s, mask);
    for (int m : mask) nnzb += m;
  }
  const double ts = sizeof(T);
  *bytes = (double)nnzb * B * B * ts + (double)s->nrow * B * ts * 2.0 + (double)s->nrow * 4.0;
}

// Adjoint of the staged step at its current (converged) iterate; see
// mpm_adjoint.cu for the equations.  K is left holding J^T.
template <int D, class T, int B>
void adjoint_impl(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* gE, double* gPhi,
                  double* gK) {
  if (!s->staged) fail(MPM_ERR_STATE, "no converged step staged (run the Newton iterations, then the adjoint)");
  cudaStream_t st = s->st;
  ck(cudaMemsetAsync(s->d_err, 0, sizeof(int), st), "memset");
  assemble_impl<D, T, B>(s, false);
  DevMatrix<T> K = matview<T>(s);
  const int S = stencil_slots(D);
  const size_t nval = (size_t)s->cap * S * B * B;
  if (s->kt_cap != s->cap) {
    s->dfree(s->d_KT);
    s->d_KT = s->dalloc<T>(nval);
    s->kt_cap = s->cap;
  }
  ck(launch_transpose_blocks<D, T, B>(s->G, K, s->d_node2row, (T*)s->d_KT, s->nrow, st), "transpose");
  ck(cudaMemcpyAsync(s->d_K, s->d_KT, nval * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy");
  ck(launch_block_jacobi<D, T, B>(s->G, K, s->nrow, s->d_err, st), "block jacobi");
  // multigrid on the transposed operator (P^T J^T P is the transpose of the
  // Galerkin operator of J); the smoother damping is estimated again
  s->mg_lam = false;
  mg_setup<D, T, B>(s);
  s->launches += 2;
  // right-hand side: dL/du on the nodes, plus a particle-displacement
  // gradient mapped with the weights; b = -S g
  double* d_g = s->dalloc<double>(s->ndof);
  double* d_b = s->dalloc<double>(s->ndof);
  if (dL_dU) ck(cudaMemcpyAsync(d_g, dL_dU, s->ndof * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
  else ck(cudaMemsetAsync(d_g, 0, s->ndof * sizeof(double), st), "memset");
  double* d_x = nullptr;
  if (dL_dx && s->np > 0) {
    d_x = s->dalloc<double>((size_t)s->np * 3);
    ck(cudaMemcpyAsync(d_x, dL_dx, (size_t)s->np * 3 * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
    ck(launch_loss_p2g<D, B>(s->P, s->G, d_x, d_g, s->d_err, st), "loss p2g");
    s->launches += 1;
  }
  ck(launch_adjoint_rhs<D, B>(d_g, d_b, s->ndof, s->up ? s->psc : 1.0, st), "rhs");
  ck(cudaMemsetAsync(s->d_norm, 0, sizeof(double), st), "memset");
  ck(launch_norm_free<B>(d_b, s->d_rows, s->nrow, s->d_fixed, s->d_norm, s->d_norm_part, s->d_norm_ticket, st),
     "norm");
  ck(cudaMemcpyAsync(s->h_dbl + 4, s->d_norm, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaStreamSynchronize(st), "sync");
  s->launches += 2;
  const double bnorm = std::sqrt(s->h_dbl[4]);
  KrylovVecs<D, T> v = vecview<D, T>(s);
  int kit = 0, kstat = 0;
  double kres2 = 0.0;
  if (bnorm > 0) {
    s->krhs = d_b;
    try {
      krylov_solve<D, T, B>(s, s->mixed ? 1e-6 : 1e-12, bnorm, kit, kstat, kres2);
    } catch (...) {
      s->krhs = s->d_r;
      throw;
    }
    s->krhs = s->d_r;
  } else {
    ck(cudaMemsetAsync((T*)s->d_vec + s->vpad, 0, s->ndof * sizeof(T), st), "memset");
  }
  s->adj_kit = kit;
  double *d_gE = gE ? s->dalloc<double>(std::max(s->np, 1)) : nullptr;
  double *d_gP = gPhi ? s->dalloc<double>(std::max(s->np, 1)) : nullptr;
  double *d_gK = gK ? s->dalloc<double>(s->nmat) : nullptr;
  if (d_gK) ck(cudaMemsetAsync(d_gK, 0, s->nmat * sizeof(double), st), "memset");
  ck(launch_param_grad<D, T, B>(s->P, s->G, s->d_mats, s->d_du, v.x, s->up ? s->psc : 1.0, d_gE, d_gP, d_gK,
                                s->d_err, st),
     "parameter gradient");
  s->launches += 1;
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaStreamSynchronize(st), "sync");
  if (gE && s->np) ck(cudaMemcpy(gE, d_gE, s->np * sizeof(double), cudaMemcpyDeviceToHost), "download");
  if (gPhi && s->np) ck(cudaMemcpy(gPhi, d_gP, s->np * sizeof(double), cudaMemcpyDeviceToHost), "download");
  if (gK) ck(cudaMemcpy(gK, d_gK, s->nmat * sizeof(double), cudaMemcpyDeviceToHost), "download");
  s->dfree(d_g);
  s->dfree(d_b);
  s->dfree(d_x);
  s->dfree(d_gE);
  s->dfree(d_gP);
  s->dfree(d_gK);
  check_err_bits(s);
  // a solve that stopped early (breakdown near convergence, the iteration
  // limit) is accepted when its residual is within a loose bound of the target
  const double accept = s->mixed ? 1e-5 : 1e-8;
  if (kstat != 0 && !(std::sqrt(std::max(kres2, 0.0)) <= accept * bnorm))
    fail(kstat == 1 ? MPM_ERR_KRYLOV_MAXIT : MPM_ERR_KRYLOV_BREAKDOWN, "adjoint Krylov solve failed");
}

// One step of the reverse chain (see mpm_adjoint_steps.cu): on entry sb
// holds the adjoint of the end-of-step state (19 per particle, caller order),
// on exit that of the start-of-step state; the parameter gradients are added
// to gE, gPhi (np) and gK (nmat).
template <int D, class T, int B>
void adjoint_step_impl(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* sb, double* gE, double* gPhi,
                       double* gK) {
  if (!s->staged) fail(MPM_ERR_STATE, "no converged step staged (restore the state, stage the step, set du)");
  cudaStream_t st = s->st;
  ck(cudaMemsetAsync(s->d_err, 0, sizeof(int), st), "memset");
  assemble_impl<D, T, B>(s, false);
  DevMatrix<T> K = matview<T>(s);
  const int S = stencil_slots(D);
  const size_t nval = (size_t)s->cap * S * B * B;
  if (s->kt_cap != s->cap) {
    s->dfree(s->d_KT);
    s->d_KT = s->dalloc<T>(nval);
    s->kt_cap = s->cap;
  }
  ck(launch_transpose_blocks<D, T, B>(s->G, K, s->d_node2row, (T*)s->d_KT, s->nrow, st), "transpose");
  ck(cudaMemcpyAsync(s->d_K, s->d_KT, nval * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy");
  ck(launch_block_jacobi<D, T, B>(s->G, K, s->nrow, s->d_err, st), "block jacobi");
  // multigrid on the transposed operator (P^T J^T P is the transpose of the
  // Galerkin operator of J); the smoother damping is estimated again
  s->mg_lam = false;
  mg_setup<D, T, B>(s);
  const size_t np = (size_t)std::max(s->np, 1);
  double* d_g = s->dalloc<double>(s->ndof);
  double* d_b = s->dalloc<double>(s->ndof);
  double* d_sb = s->dalloc<double>(np * 19);
  double* d_so = s->dalloc<double>(np * 19);
  double* d_gE = s->dalloc<double>(np);
  double* d_gP = s->dalloc<double>(np);
  double* d_gK = s->dalloc<double>(s->nmat);
  if (dL_dU) ck(cudaMemcpyAsync(d_g, dL_dU, s->ndof * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
  else ck(cudaMemsetAsync(d_g, 0, s->ndof * sizeof(double), st), "memset");
  if (s->np > 0) ck(cudaMemcpyAsync(d_sb, sb, (size_t)s->np * 19 * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
  ck(cudaMemsetAsync(d_gE, 0, np * sizeof(double), st), "memset");
  ck(cudaMemsetAsync(d_gP, 0, np * sizeof(double), st), "memset");
  ck(cudaMemsetAsync(d_gK, 0, s->nmat * sizeof(double), st), "memset");
  double* d_x = nullptr;
  if (dL_dx && s->np > 0) {
    d_x = s->dalloc<double>(np * 3);
    ck(cudaMemcpyAsync(d_x, dL_dx, (size_t)s->np * 3 * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
    ck(launch_loss_p2g<D, B>(s->P, s->G, d_x, d_g, s->d_err, st), "loss p2g");
  }
  const double psc = s->up ? s->psc : 1.0;
  ck(launch_adj_commit_vjp<D, T, B>(s->P, s->G, s->d_mats, s->d_grav, s->d_du, psc, d_sb, d_g, s->d_err, st),
     "commit vjp");
  ck(launch_adjoint_rhs<D, B>(d_g, d_b, s->ndof, psc, st), "rhs");
  ck(cudaMemsetAsync(s->d_norm, 0, sizeof(double), st), "memset");
  ck(launch_norm_free<B>(d_b, s->d_rows, s->nrow, s->d_fixed, s->d_norm, s->d_norm_part, s->d_norm_ticket, st),
     "norm");
  ck(cudaMemcpyAsync(s->h_dbl + 4, s->d_norm, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaStreamSynchronize(st), "sync");
  s->launches += 6;
  const double bnorm = std::sqrt(s->h_dbl[4]);
  KrylovVecs<D, T> v = vecview<D, T>(s);
  int kit = 0, kstat = 0;
  double kres2 = 0.0;
  if (bnorm > 0) {
    s->krhs = d_b;
    try {
      krylov_solve<D, T, B>(s, s->mixed ? 1e-6 : 1e-12, bnorm, kit, kstat, kres2);
    } catch (...) {
      s->krhs = s->d_r;
      throw;
    }
    s->krhs = s->d_r;
  } else {
    ck(cudaMemsetAsync((T*)s->d_vec + s->vpad, 0, s->ndof * sizeof(T), st), "memset");
  }
  s->adj_kit = kit;
  ck(launch_adj_state_vjp<D, T, B>(s->P, s->G, s->d_mats, s->d_grav, s->d_du, v.x, psc, d_sb, d_so, d_gE, d_gP,
                                   d_gK, s->d_err, st),
     "state vjp");
  s->launches += 1;
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
  ck(cudaStreamSynchronize(st), "sync");
  std::vector<double> h(np);
  if (s->np > 0) {
    ck(cudaMemcpy(sb, d_so, (size_t)s->np * 19 * sizeof(double), cudaMemcpyDeviceToHost), "download");
    if (gE) {
      ck(cudaMemcpy(h.data(), d_gE, s->np * sizeof(double), cudaMemcpyDeviceToHost), "download");
      for (int p = 0; p < s->np; ++p) gE[p] += h[p];
    }
    if (gPhi) {
      ck(cudaMemcpy(h.data(), d_gP, s->np * sizeof(double), cudaMemcpyDeviceToHost), "download");
      for (int p = 0; p < s->np; ++p) gPhi[p] += h[p];
    }
  }
  if (gK) {
    std::vector<double> hk(s->nmat);
    ck(cudaMemcpy(hk.data(), d_gK, s->nmat * sizeof(double), cudaMemcpyDeviceToHost), "download");
    for (int m = 0; m < s->nmat; ++m) gK[m] += hk[m];
  }
  for (double* d : {d_g, d_b, d_sb, d_so, d_gE, d_gP, d_gK, d_x}) s->dfree(d);
  check_err_bits(s);
  const double accept = s->mixed ? 1e-5 : 1e-8;
  if (kstat != 0 && !(std::sqrt(std::max(kres2, 0.0)) <= accept * bnorm))
    fail(kstat == 1 ? MPM_ERR_KRYLOV_MAXIT : MPM_ERR_KRYLOV_BREAKDOWN, "adjoint Krylov solve failed");
}

template <int D, class T, int B>
void particle_increment_impl(mpm_scene* s, double* out) {
  if (!s->staged) fail(MPM_ERR_STATE, "no load step staged");
  double* d_o = s->dalloc<double>((size_t)std::max(s->np, 1) * 3);
  ck(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->st), "memset");
  ck(launch_particle_increment<D, B>(s->P, s->G, s->d_du, d_o, s->d_err, s->st), "increment");
  s->launches += 1;
  ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st), "copy");
  ck(cudaStreamSynchronize(s->st), "sync");
  if (s->np) ck(cudaMemcpy(out, d_o, (size_t)s->np * 3 * sizeof(double), cudaMemcpyDeviceToHost), "download");
  s->dfree(d_o);
  check_err_bits(s);
}

// dispatch on (dim, precision, values per node)
template <template <int, class, int> class F, class... Args>
void dispatch(mpm_scene* s, Args... args) {
  if (s->up) {
    if (s->mixed) F<2, float, 3>::run(s, args...);
    else F<2, double, 3>::run(s, args...);
  } else if (s->D == 2) {
    if (s->mixed) F<2, float, 2>::run(s, args...);
    else F<2, double, 2>::run(s, args...);
  } else {
    if (s->mixed) F<3, float, 3>::run(s, args...);
    else F<3, double, 3>::run(s, args...);
  }
}
template <int D, class T, int B> struct BeginF { static void run(mpm_scene* s, mpm_newton_report* r) { begin_step_impl<D, T, B>(s, r); } };
template <int D, class T, int B> struct NewtonF { static void run(mpm_scene* s, mpm_newton_report* r) { newton_impl<D, T, B>(s, r); } };
template <int D, class T, int B> struct CommitF { static void run(mpm_scene* s) { commit_impl<D, T, B>(s); } };
template <int D, class T, int B> struct SetDuF { static void run(mpm_scene* s, const double* du) { set_du_impl<D, T, B>(s, du); } };
template <int D, class T, int B> struct TimeSpmvF {
  static void run(mpm_scene* s, int reps, double* ms, double* bytes) { time_spmv_impl<D, T, B>(s, reps, ms, bytes); }
};
template <int D, class T, int B> struct AdjointF {
  static void run(mpm_scene* s, const double* a, const double* b, double* c, double* d, double* e) {
    adjoint_impl<D, T, B>(s, a, b, c, d, e);
  }
};
template <int D, class T, int B> struct AdjointStepF {
  static void run(mpm_scene* s, const double* a, const double* b, double* sb, double* c, double* d, double* e) {
    adjoint_step_impl<D, T, B>(s, a, b, sb, c, d, e);
  }
};
template <int D, class T, int B> struct MgApplyF {
  static void run(mpm_scene* s, const double* b, double* z) { mg_apply_impl<D, T, B>(s, b, z); }
};
template <int D, class T, int B> struct IncrementF {
  static void run(mpm_scene* s, double* o) { particle_increment_impl<D, T, B>(s, o); }
};
template <int D, class T, int B> struct AssembleF {
  static void run(mpm_scene* s) {
    assemble_impl<D, T, B>(s);
    ck(cudaMemcpyAsync(s->h_int + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st), "copy");
    ck(cudaStreamSynchronize(s->st), "sync");
    check_err_bits(s);
  }
};

template <class Fn>
mpm_status guarded(mpm_scene* s, Fn&& fn) {
  try {
    fn();
    return MPM_OK;
  } catch (const Fail& f) {
    if (s) s->err = f.msg;
    return f.st;
  } catch (const std::exception& e) {
    if (s) s->err = e.what();
    return MPM_ERR_INVALID_ARG;
  } catch (...) {
    if (s) s->err = "unknown failure";
    return MPM_ERR_INVALID_ARG;
  }
}

void destroy(mpm_scene* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  for (void* p : s->allocs) cudaFreeAsync(p, s->st);
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->gexec_gm) cudaGraphExecDestroy(s->gexec_gm);
  if (s->h_gst) cudaFreeHost(s->h_gst);
  if (s->h_S) cudaFreeHost(s->h_S);
  if (s->h_int) cudaFreeHost(s->h_int);
  if (s->h_dbl) cudaFreeHost(s->h_dbl);
  if (s->h_mgn) cudaFreeHost(s->h_mgn);
  for (auto& e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  delete s;
}

}  // namespace

extern "C" {

mpm_status mpm_create_scene(const mpm_scene_desc* desc, int np, const double* x, const double* vol0,
                            const double* mass, const int* mat_id, const double* E_p, const double* phi_p,
                            const double* pc0_p, const mpm_material* mats, int nmat, void* stream,
                            mpm_scene** out) {
  if (!out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  mpm_scene* s = new (std::nothrow) mpm_scene();
  if (!s) return MPM_ERR_OOM;
  mpm_status rc = guarded(s, [&] {
    validate_desc(desc);
    if (np < 0 || (np > 0 && (!x || !vol0 || !mass || !mat_id))) fail(MPM_ERR_INVALID_ARG, "particle arrays");
    if (!mats || nmat < 1) fail(MPM_ERR_INVALID_ARG, "need at least one material");
    s->desc = *desc;
    s->D = desc->dim;
    s->up = desc->formulation == MPM_UP;
    s->B = dofs_per_node(desc);
    // preconditioner blocks: the u-p default is the row segment, whose exact
    // 4-node solves take in the lateral pressure modes that only the small
    // Darcy term controls (node blocks leave them to the Krylov method)
    s->seg = (desc->precond == MPM_PC_SEG4 || (desc->precond == MPM_PC_AUTO && s->up)) ? 4 : 1;
    s->mg = desc->precond == MPM_PC_MG;
    s->np = np;
    s->nmat = nmat;
    s->nbe = s->D == 2 ? 4 : 6;
    s->nF = s->D * s->D;
    s->mixed = desc->precision == MPM_MIXED;
    DevGrid& G = s->G;
    G.dim = s->D;
    for (int a = 0; a < 3; ++a) {
      G.n[a] = (a < s->D) ? desc->n[a] : 0;
      G.o[a] = desc->origin[a];
    }
    G.nx1 = G.n[0] + 1;
    G.ny1 = G.n[1] + 1;
    G.nz1 = s->D == 3 ? G.n[2] + 1 : 1;
    G.h = desc->h;
    G.ih = 1.0 / desc->h;
    s->nnode = (long long)G.nx1 * G.ny1 * G.nz1;
    G.nnode = s->nnode;
    s->ndof = s->nnode * s->B;
    if (s->nnode + 1 > 2000000000LL) fail(MPM_ERR_INVALID_ARG, "grid too large");
    // materials
    for (int m = 0; m < nmat; ++m) {
      const mpm_material& q = mats[m];
      if (q.model < MPM_NH || q.model > MPM_NH_MCC) fail(MPM_ERR_INVALID_ARG, "bad material model");
      if (!(q.E > 0) || !(q.nu > -1 && q.nu < 0.5)) fail(MPM_ERR_INVALID_ARG, "bad elastic constants");
      if (q.model == MPM_NH_MCC && !(q.lambda_cc > q.kappa_cc && q.M > 0))
        fail(MPM_ERR_INVALID_ARG, "bad Cam-Clay constants");
      MatC c{};
      c.model = q.model;
      c.E = q.E;
      c.nu = q.nu;
      c.rho = q.rho;
      c.phi = q.phi;
      c.psi = q.psi;
      c.coh = q.c;
      c.M = q.M;
      c.lmk = q.lambda_cc - q.kappa_cc;
      c.pc0 = q.pc0;
      c.dkdt_dk = (s->up && q.gamma_w > 0) ? desc->dt / q.gamma_w : 0.0;
      s->hmats.push_back(c);
      if (s->up && (!(q.k_hyd >= 0) || !(q.gamma_w > 0)))
        fail(MPM_ERR_INVALID_ARG, "u-p materials need k_hyd >= 0 and gamma_w > 0");
    }
    if (s->up) {
      // pressure scale: the largest shear modulus over the grid spacing
      // (p / psc is then a length, psc * (mass balance) a force)
      double mu_max = 0.0;
      for (int m = 0; m < nmat; ++m) mu_max = std::max(mu_max, mats[m].E / (2.0 * (1.0 + mats[m].nu)));
      s->psc = desc->p_scale > 0 ? desc->p_scale : mu_max / desc->h;
    }
    // host-side validation of particles
    for (int p = 0; p < np; ++p) {
      if (mat_id[p] < 0 || mat_id[p] >= nmat) fail(MPM_ERR_INVALID_ARG, "mat_id out of range");
      if (!(mass[p] > 0) || !(vol0[p] > 0)) fail(MPM_ERR_INVALID_ARG, "mass and vol0 must be positive");
      for (int a = 0; a < s->D; ++a) {
        double sg = (x[3 * p + a] - G.o[a]) / G.h;
        double fb = std::floor(sg - 0.5);
        if (!(fb >= 0 && fb <= G.n[a] - 2)) fail(MPM_ERR_INVALID_ARG, "particle outside the grid interior");
      }
      if (E_p && !(E_p[p] > 0)) fail(MPM_ERR_INVALID_ARG, "E_p must be positive");
      if (pc0_p && s->hmats[mat_id[p]].model == MPM_NH_MCC && !(pc0_p[p] < 0))
        fail(MPM_ERR_INVALID_ARG, "pc0 must be negative");
      s->mmax = std::max(s->mmax, mass[p]);
    }
    if (stream) {
      s->st = (cudaStream_t)stream;
    } else {
      ck(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking), "stream");
      s->own_stream = true;
    }
    s->use_graph = s->st != nullptr && s->st != cudaStreamLegacy && s->st != cudaStreamPerThread;
    for (auto& e : s->ev) ck(cudaEventCreate(&e), "event");
    ck(cudaMallocHost(&s->h_S, sizeof(KrylovScalars)), "host alloc");
    ck(cudaMallocHost(&s->h_int, 16 * sizeof(int)), "host alloc");
    ck(cudaMallocHost(&s->h_dbl, 16 * sizeof(double)), "host alloc");
    s->d_mats = s->dalloc<MatC>(nmat);
    ck(cudaMemcpyAsync(s->d_mats, s->hmats.data(), nmat * sizeof(MatC), cudaMemcpyHostToDevice, s->st), "copy");
    // particles: staging on the host in SoA order
    auto mk = [&](DevParticles& P) {
      if (s->D == 2) P = make_particles<2>(s);
      else P = make_particles<3>(s);
    };
    mk(s->P);
    mk(s->Q);
    s->d_fail = s->dalloc<double>(FAIL_REC);
    ck(cudaMemsetAsync(s->d_fail, 0, FAIL_REC * sizeof(double), s->st), "memset");
    s->P.fail_rec = s->d_fail;
    s->Q.fail_rec = s->d_fail;
    std::vector<double> h(np);
    auto up = [&](double* d) {
      ck(cudaMemcpy(d, h.data(), np * sizeof(double), cudaMemcpyHostToDevice), "upload");
    };
    if (np > 0) {
      for (int a = 0; a < s->D; ++a) {
        for (int p = 0; p < np; ++p) h[p] = x[3 * p + a];
        up(s->P.x[a]);
      }
      std::copy(vol0, vol0 + np, h.begin()); up(s->P.vol0);
      std::copy(mass, mass + np, h.begin()); up(s->P.mass);
      for (int p = 0; p < np; ++p) h[p] = E_p ? E_p[p] : mats[mat_id[p]].E;
      up(s->P.Ep);
      for (int p = 0; p < np; ++p) h[p] = phi_p ? phi_p[p] : mats[mat_id[p]].phi;
      up(s->P.phip);
      for (int p = 0; p < np; ++p) h[p] = pc0_p ? pc0_p[p] : mats[mat_id[p]].pc0;
      up(s->P.pc);
      for (int k = 0; k < s->nbe; ++k) {
        std::fill(h.begin(), h.end(), k < 3 ? 1.0 : 0.0);
        up(s->P.be[k]);
      }
      for (int k = 0; k < s->nF; ++k) {
        std::fill(h.begin(), h.end(), (k % (s->D + 1) == 0) ? 1.0 : 0.0);
        up(s->P.F[k]);
      }
      ck(cudaMemcpy(s->P.mat, mat_id, np * sizeof(int), cudaMemcpyHostToDevice), "upload");
      if (s->up) {
        for (int p = 0; p < np; ++p) h[p] = mats[mat_id[p]].k_hyd / mats[mat_id[p]].gamma_w * desc->dt;
        up(s->P.kdt);
        std::fill(h.begin(), h.end(), 0.0);
        up(s->P.pp);
      }
      std::vector<int> o(np);
      for (int p = 0; p < np; ++p) o[p] = p;
      ck(cudaMemcpy(s->P.orig, o.data(), np * sizeof(int), cudaMemcpyHostToDevice), "upload");
    }
    // sort scratch and grid arrays
    const long long nn = s->nnode;
    s->d_key = s->dalloc<int>(np);
    s->d_rank = s->dalloc<int>(np);
    s->d_perm = s->dalloc<int>(np);
    s->d_count = s->dalloc<int>(nn + 1);
    s->d_cstart = s->dalloc<int>(nn + 1);
    s->d_flag = s->dalloc<int>(nn + 1);
    s->d_pos = s->dalloc<int>(nn + 1);
    s->d_cells = s->dalloc<int>(nn);
    s->d_cellpos = s->dalloc<int>(nn + 1);
    s->d_node2row = s->dalloc<int>(nn);
    s->d_rows = s->dalloc<int>(nn);
    s->d_scan_tmp = s->dalloc<int>(scan_tmp_ints((int)(nn + 1)));
    s->d_nrow = s->dalloc<int>(1);
    s->d_err = s->dalloc<int>(2);
    s->d_nplastic = s->d_err + 1;
    s->d_M = s->dalloc<double>(nn);
    s->d_du = s->dalloc<double>(s->ndof);
    s->d_duprev = s->dalloc<double>(s->ndof);
    s->d_absmax = s->dalloc<unsigned long long>(1);
    s->d_r = s->dalloc<double>(s->ndof);
    s->krhs = s->d_r;
    s->d_bcval = s->dalloc<double>(s->ndof);
    s->d_grav = s->dalloc<double>(3);
    s->d_norm = s->dalloc<double>(1);
    s->d_fixed = s->dalloc<uint8_t>(s->ndof);
    ck(cudaMemsetAsync(s->d_du, 0, s->ndof * sizeof(double), s->st), "memset");
    ck(cudaMemsetAsync(s->d_r, 0, s->ndof * sizeof(double), s->st), "memset");
    ck(cudaMemsetAsync(s->d_bcval, 0, s->ndof * sizeof(double), s->st), "memset");
    ck(cudaMemsetAsync(s->d_fixed, 0, s->ndof, s->st), "memset");
    ck(cudaMemsetAsync(s->d_nrow, 0, sizeof(int), s->st), "memset");
    const size_t T = tsize(s);
    const size_t NPHI = s->D + (s->up ? 1 : 0);
    const size_t D4 = (size_t)s->B * NPHI * s->B * NPHI;   // tangent entries per particle
    s->d_A = s->mixed ? (void*)s->dalloc<float>((size_t)np * D4) : (void*)s->dalloc<double>((size_t)np * D4);
    s->vpad = (2 + 2LL * G.nx1 + (s->D == 3 ? 2LL * G.nx1 * G.ny1 : 0)) * s->B;
    s->vlen = s->ndof + 2 * s->vpad;
    if (s->mixed) s->d_vec = s->dalloc<float>(9 * s->vlen);
    else s->d_vec = s->dalloc<double>(9 * s->vlen);
    ck(cudaMemsetAsync(s->d_vec, 0, 9 * s->vlen * T, s->st), "memset");
    s->d_S = s->dalloc<KrylovScalars>(1);
    s->d_norm_ticket = s->dalloc<unsigned>(1);
    ck(cudaMemsetAsync(s->d_norm_ticket, 0, sizeof(unsigned), s->st), "memset");
    s->d_fp = s->dalloc<double>((size_t)np * (s->D == 3 ? 27 : 9) * s->B);
    if (s->mg) mg_create(s);
    if (desc->krylov == MPM_GMRES) {
      s->gm = desc->gmres_restart > 0 ? std::min(std::max(desc->gmres_restart, 2), GMRES_MMAX) : 30;
      const size_t nv = (size_t)(s->gm + 3) * s->vlen;
      if (s->mixed) s->d_gvec = s->dalloc<float>(nv);
      else s->d_gvec = s->dalloc<double>(nv);
      ck(cudaMemsetAsync(s->d_gvec, 0, nv * T, s->st), "memset");
      s->d_gst = s->dalloc<GmresState>(1);
      ck(cudaMallocHost(&s->h_gst, 128), "host alloc");
    }
    s->d_bar = s->dalloc<unsigned int>(PERSIST_BAR_WORDS);
    s->d_part = s->dalloc<double>(5 * PERSIST_MAX_BLOCKS);
    {
      // BiCGStab runs as CUDA-graph chunks of four kernels per iteration;
      // MPM_KRYLOV_PERSISTENT=1 selects the single cooperative kernel instead
      // (measured slower on the 2D footing: 32 vs 25 us per iteration)
      const char* env = getenv("MPM_KRYLOV_PERSISTENT");
      int dev = 0;
      ck(cudaGetDevice(&dev), "device");
      const bool want_persistent = env && env[0] == '1';
      if (want_persistent && desc->krylov == MPM_BICGSTAB && !s->up && s->seg == 1 && !s->mg) {
        if (s->D == 2) s->pblocks = s->mixed ? persistent_blocks<2, float>(dev) : persistent_blocks<2, double>(dev);
        else s->pblocks = s->mixed ? persistent_blocks<3, float>(dev) : persistent_blocks<3, double>(dev);
      }
    }
    ck(cudaStreamSynchronize(s->st), "sync");
  });
  if (rc != MPM_OK) {
    g_create_err = s->err;
    destroy(s);
    return rc;
  }
  *out = s;
  return MPM_OK;
}

mpm_status mpm_set_gravity(mpm_scene* s, const double g[3]) {
  if (!s || !g) return MPM_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) s->grav[a] = g[a];
  return MPM_OK;
}

mpm_status mpm_set_dirichlet(mpm_scene* s, int n, const long long* dof, const double* value) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (n < 0 || (n > 0 && (!dof || !value))) fail(MPM_ERR_INVALID_ARG, "dirichlet arrays");
    std::vector<uint8_t> f(s->ndof, 0);
    std::vector<double> v(s->ndof, 0.0);
    for (int k = 0; k < n; ++k) {
      if (dof[k] < 0 || dof[k] >= s->ndof) fail(MPM_ERR_INVALID_ARG, "dirichlet dof out of range");
      f[dof[k]] = 1;
      // a prescribed pore pressure is held as p / psc inside the solver
      v[dof[k]] = (s->up && dof[k] % s->B == s->D) ? value[k] / s->psc : value[k];
    }
    ck(cudaStreamSynchronize(s->st), "sync");
    ck(cudaMemcpy(s->d_fixed, f.data(), s->ndof, cudaMemcpyHostToDevice), "upload");
    ck(cudaMemcpy(s->d_bcval, v.data(), s->ndof * sizeof(double), cudaMemcpyHostToDevice), "upload");
  });
}

mpm_status mpm_begin_step(mpm_scene* s, mpm_newton_report* rep) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<BeginF>(s, rep); });
}

mpm_status mpm_newton_step(mpm_scene* s, mpm_newton_report* rep) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<NewtonF>(s, rep); });
}

mpm_status mpm_commit_step(mpm_scene* s) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<CommitF>(s); });
}

mpm_status mpm_set_du(mpm_scene* s, const double* du) {
  if (!s || !du) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<SetDuF>(s, du); });
}

mpm_status mpm_assemble(mpm_scene* s) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<AssembleF>(s); });
}

mpm_status mpm_time_spmv(mpm_scene* s, int reps, double* ms_per_launch, double* bytes_per_launch) {
  if (!s || !ms_per_launch || !bytes_per_launch) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<TimeSpmvF>(s, reps, ms_per_launch, bytes_per_launch); });
}

mpm_status mpm_kernel_launches(const mpm_scene* s, long long* out) {
  if (!s || !out) return MPM_ERR_INVALID_ARG;
  *out = s->launches;
  return MPM_OK;
}

mpm_status mpm_get_newton_counters(const mpm_scene* s, long long* limited, long long* halvings) {
  if (!s) return MPM_ERR_INVALID_ARG;
  if (limited) *limited = s->limited;
  if (halvings) *halvings = s->halvings;
  return MPM_OK;
}

mpm_status mpm_solve_step(mpm_scene* s, mpm_step_report* rep) {
  if (!s) return MPM_ERR_INVALID_ARG;
  mpm_step_report local{};
  mpm_step_report& R = rep ? *rep : local;
  std::memset(&R, 0, sizeof(R));
  mpm_status st = guarded(s, [&] {
    auto t0 = std::chrono::steady_clock::now();
    mpm_newton_report nr{};
    dispatch<BeginF>(s, &nr);
    auto t1 = std::chrono::steady_clock::now();
    R.t_setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    R.r0_norm = s->r0;
    R.hist[0] = 1.0;
    R.n_active_nodes = s->nrow;
    R.t_residual_ms += s->t_res;
    bool conv = s->r0 == 0.0;
    while (!conv && s->k < s->desc.newton_maxit) {
      dispatch<NewtonF>(s, &nr);
      R.krylov_iters[s->k - 1] = nr.krylov_iters;
      R.krylov_iters_total += nr.krylov_iters;
      R.hist[s->k] = nr.rel_residual;
      R.t_assembly_ms += s->t_asm;
      R.t_krylov_ms += s->t_kry;
      R.t_residual_ms += s->t_res;
      conv = nr.rel_residual <= s->desc.newton_tol;
    }
    R.newton_iters = s->k;
    R.converged = conv;
    R.rel_residual = s->r0 > 0 ? s->rk / s->r0 : 0.0;
    if (!conv) fail(MPM_ERR_NOT_CONVERGED, "Newton did not reach newton_tol");
    auto t2 = std::chrono::steady_clock::now();
    dispatch<CommitF>(s);
    auto t3 = std::chrono::steady_clock::now();
    R.t_commit_ms = std::chrono::duration<double, std::milli>(t3 - t2).count();
  });
  R.status = st;
  return st;
}

mpm_status mpm_get_residual(const mpm_scene* cs, double* r) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !r) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(cudaStreamSynchronize(s->st), "sync");
    std::vector<double> full(s->ndof), du(1);
    ck(cudaMemcpy(full.data(), s->d_r, s->ndof * sizeof(double), cudaMemcpyDeviceToHost), "download");
    std::vector<uint8_t> f(s->ndof);
    ck(cudaMemcpy(f.data(), s->d_fixed, s->ndof, cudaMemcpyDeviceToHost), "download");
    std::vector<int> n2r(s->nnode);
    ck(cudaMemcpy(n2r.data(), s->d_node2row, s->nnode * sizeof(int), cudaMemcpyDeviceToHost), "download");
    for (long long d = 0; d < s->ndof; ++d) {
      r[d] = (f[d] || n2r[d / s->B] < 0) ? 0.0 : full[d];
      if (s->up && d % s->B == s->D) r[d] /= s->psc;   // mass-balance rows in physical units
    }
  });
}

mpm_status mpm_get_du(const mpm_scene* cs, double* du) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !du) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(cudaStreamSynchronize(s->st), "sync");
    ck(cudaMemcpy(du, s->d_du, s->ndof * sizeof(double), cudaMemcpyDeviceToHost), "download");
    if (s->up)
      for (long long d = s->D; d < s->ndof; d += s->B) du[d] *= s->psc;
  });
}

mpm_status mpm_get_du_dev(const mpm_scene* cs, double* d_du) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !d_du) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(launch_du_out(s->d_du, d_du, s->ndof, s->B, s->D, s->psc, s->st), "du out");
    s->launches += 1;
  });
}

mpm_status mpm_get_residual_dev(const mpm_scene* cs, double* d_r) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !d_r) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(launch_residual_out(s->d_r, s->d_fixed, s->d_node2row, d_r, s->ndof, s->B, s->D, s->psc, s->st),
       "residual out");
    s->launches += 1;
  });
}

mpm_status mpm_get_positions_dev(const mpm_scene* cs, double* d_x) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !d_x) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(launch_positions_out(s->P, s->D, d_x, s->st), "positions out");
    s->launches += 1;
  });
}

mpm_status mpm_set_dirichlet_dev(mpm_scene* s, int n, const long long* d_dof, const double* d_value) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (n < 0 || (n > 0 && (!d_dof || !d_value))) fail(MPM_ERR_INVALID_ARG, "dirichlet arrays");
    ck(cudaMemsetAsync(s->d_fixed, 0, s->ndof, s->st), "memset");
    ck(cudaMemsetAsync(s->d_bcval, 0, s->ndof * sizeof(double), s->st), "memset");
    ck(cudaMemsetAsync(s->d_nplastic, 0, sizeof(int), s->st), "memset");
    ck(launch_dirichlet_in(n, d_dof, d_value, s->d_fixed, s->d_bcval, s->ndof, s->B, s->D, s->psc, s->d_nplastic,
                           s->st),
       "dirichlet in");
    s->launches += 1;
    ck(cudaMemcpyAsync(s->h_int + 3, s->d_nplastic, sizeof(int), cudaMemcpyDeviceToHost, s->st), "copy");
    ck(cudaStreamSynchronize(s->st), "sync");
    if (s->h_int[3] != 0) fail(MPM_ERR_INVALID_ARG, "dirichlet dof out of range");
  });
}

mpm_status mpm_get_mass(const mpm_scene* cs, double* mass) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !mass) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(cudaStreamSynchronize(s->st), "sync");
    ck(cudaMemcpy(mass, s->d_M, s->nnode * sizeof(double), cudaMemcpyDeviceToHost), "download");
  });
}

}  // extern "C"

namespace {
template <int D>
void pattern_mask(mpm_scene* s, std::vector<int>& mask) {
  const int S = stencil_slots(D);
  int* d_mask = s->dalloc<int>((size_t)std::max(s->nrow, 1) * S);
  ck(cudaMemsetAsync(d_mask, 0, (size_t)std::max(s->nrow, 1) * S * sizeof(int), s->st), "memset");
  ck(launch_pattern_count<D>(s->G, s->d_rows, s->nrow, s->d_node2row, s->d_count, d_mask, s->st), "pattern");
  s->launches += 1;
  mask.resize((size_t)s->nrow * S);
  ck(cudaMemcpyAsync(mask.data(), d_mask, mask.size() * sizeof(int), cudaMemcpyDeviceToHost, s->st), "download");
  ck(cudaStreamSynchronize(s->st), "sync");
  s->dfree(d_mask);
}
}  // namespace

extern "C" {

mpm_status mpm_get_counts(const mpm_scene* cs, int* n_active, long long* nnzb) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(cudaStreamSynchronize(s->st), "sync");
    if (n_active) *n_active = s->nrow;
    if (nnzb) {
      std::vector<int> mask;
      if (s->D == 2) pattern_mask<2>(s, mask);
      else pattern_mask<3>(s, mask);
      long long c = 0;
      for (int m : mask) c += m;
      *nnzb = c;
    }
  });
}

mpm_status mpm_get_jacobian_bsr(const mpm_scene* cs, long long cap, int* row_node, long long* row_ptr,
                                int* col_node, double* val) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !row_node || !row_ptr || !col_node || !val) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (!s->staged && s->nrow == 0) fail(MPM_ERR_STATE, "no Jacobian assembled");
    const int D = s->D, S = stencil_slots(D), B = s->B, DD = B * B;
    std::vector<int> mask;
    if (D == 2) pattern_mask<2>(s, mask);
    else pattern_mask<3>(s, mask);
    std::vector<int> rows(s->nrow);
    ck(cudaMemcpy(rows.data(), s->d_rows, s->nrow * sizeof(int), cudaMemcpyDeviceToHost), "download");
    std::vector<uint8_t> fx(s->ndof);
    ck(cudaMemcpy(fx.data(), s->d_fixed, s->ndof, cudaMemcpyDeviceToHost), "download");
    const size_t nval = (size_t)s->cap * S * DD;
    std::vector<double> K(nval);
    if (s->mixed) {
      std::vector<float> Kf(nval);
      ck(cudaMemcpy(Kf.data(), s->d_K, nval * sizeof(float), cudaMemcpyDeviceToHost), "download");
      for (size_t q = 0; q < nval; ++q) K[q] = Kf[q];
    } else {
      ck(cudaMemcpy(K.data(), s->d_K, nval * sizeof(double), cudaMemcpyDeviceToHost), "download");
    }
    const int nx1 = s->G.nx1, ny1 = s->G.ny1;
    long long nb = 0;
    row_ptr[0] = 0;
    for (int r = 0; r < s->nrow; ++r) {
      row_node[r] = rows[r];
      for (int sl = 0; sl < S; ++sl) {
        if (!mask[(size_t)r * S + sl]) continue;
        if (nb >= cap) fail(MPM_ERR_INVALID_ARG, "capacity too small for the Jacobian");
        int dx = sl % 5 - 2, dy = (sl / 5) % 5 - 2, dz = D == 3 ? sl / 25 - 2 : 0;
        col_node[nb] = rows[r] + dx + nx1 * (dy + ny1 * dz);
        // back to physical units: the pressure rows and columns carry psc
        // (the identity entry of a prescribed pressure stays 1)
        const bool centre = (dx == 0 && dy == 0 && dz == 0);
        for (int a = 0; a < B; ++a)
          for (int b = 0; b < B; ++b) {
            double sc = 1.0;
            const bool ident = centre && a == b && fx[(size_t)rows[r] * B + a];
            if (s->up && a == D && !ident) sc /= s->psc;
            if (s->up && b == D && !ident) sc /= s->psc;
            val[nb * DD + a * B + b] = K[((size_t)sl * s->cap + r) * DD + a * B + b] * sc;
          }
        ++nb;
      }
      row_ptr[r + 1] = nb;
    }
  });
}

mpm_status mpm_get_mg_level(const mpm_scene* cs, int level, int* levels, int dims[3], int* nrow, int cap,
                            int* nodes, double* vals, unsigned char* fixed, double* lambda_max) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !levels) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (!s->mg || s->mg_L == 0) fail(MPM_ERR_STATE, "no multigrid hierarchy (MPM_PC_MG, after an assembly)");
    *levels = s->mg_L;
    if (level == 0 && lambda_max) {
      ck(cudaStreamSynchronize(s->st), "sync");
      double n2 = 0;
      ck(cudaMemcpy(&n2, s->d_mg_nrm + MG_POWER_IT, sizeof(double), cudaMemcpyDeviceToHost), "download");
      *lambda_max = std::sqrt(n2);
    }
    if (level < 1) return;
    if (level >= s->mg_L) fail(MPM_ERR_INVALID_ARG, "level out of range");
    const auto& m = s->mgl[level];
    if (dims) {
      dims[0] = m.nx1;
      dims[1] = m.ny1;
      dims[2] = m.nz1;
    }
    if (nrow) *nrow = m.nrow;
    ck(cudaStreamSynchronize(s->st), "sync");
    if (lambda_max) {
      double n2 = 0;
      ck(cudaMemcpy(&n2, s->d_mg_nrm + (size_t)level * (MG_POWER_IT + 1) + MG_POWER_IT, sizeof(double),
                    cudaMemcpyDeviceToHost),
         "download");
      *lambda_max = std::sqrt(n2);
    }
    if (fixed) ck(cudaMemcpy(fixed, m.fixed, m.nnode * s->B, cudaMemcpyDeviceToHost), "download");
    if (!nodes) return;
    if (cap < m.nrow || !vals) fail(MPM_ERR_INVALID_ARG, "capacity too small for the level");
    ck(cudaMemcpy(nodes, m.rows, m.nrow * sizeof(int), cudaMemcpyDeviceToHost), "download");
    const int S = stencil_slots(s->D), BB = s->B * s->B;
    const size_t nval = (size_t)m.cap * S * BB;
    std::vector<double> K(nval);
    if (s->mixed) {
      std::vector<float> Kf(nval);
      ck(cudaMemcpy(Kf.data(), m.val, nval * sizeof(float), cudaMemcpyDeviceToHost), "download");
      for (size_t q = 0; q < nval; ++q) K[q] = Kf[q];
    } else {
      ck(cudaMemcpy(K.data(), m.val, nval * sizeof(double), cudaMemcpyDeviceToHost), "download");
    }
    for (int r = 0; r < m.nrow; ++r)
      for (int sl = 0; sl < S; ++sl)
        for (int k = 0; k < BB; ++k) vals[((size_t)r * S + sl) * BB + k] = K[((size_t)sl * m.cap + r) * BB + k];
  });
}

mpm_status mpm_mg_apply(mpm_scene* s, const double* b, double* z) {
  if (!s || !b || !z) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<MgApplyF>(s, b, z); });
}

mpm_status mpm_get_particles(const mpm_scene* cs, double* x, double* be, double* pc, double* F, double* tau) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    ck(cudaStreamSynchronize(s->st), "sync");
    const int np = s->np, D = s->D;
    if (np == 0) return;
    std::vector<int> orig(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    std::vector<double> h(np);
    auto down = [&](const double* d) {
      ck(cudaMemcpy(h.data(), d, np * sizeof(double), cudaMemcpyDeviceToHost), "download");
    };
    if (x) {
      for (int p = 0; p < np; ++p)
        for (int a = 0; a < 3; ++a) x[3 * p + a] = 0.0;
      for (int a = 0; a < D; ++a) {
        down(s->P.x[a]);
        for (int p = 0; p < np; ++p) x[3 * orig[p] + a] = h[p];
      }
    }
    if (be) {
      static const int map2[4] = {0, 1, 2, 3};
      for (int p = 0; p < np; ++p)
        for (int k = 0; k < 6; ++k) be[6 * p + k] = 0.0;
      for (int k = 0; k < s->nbe; ++k) {
        down(s->P.be[k]);
        int dst = D == 2 ? map2[k] : k;
        for (int p = 0; p < np; ++p) be[6 * orig[p] + dst] = h[p];
      }
    }
    if (pc) {
      down(s->P.pc);
      for (int p = 0; p < np; ++p) pc[orig[p]] = h[p];
    }
    if (F) {
      for (int p = 0; p < np; ++p)
        for (int k = 0; k < 9; ++k) F[9 * p + k] = (k % 4 == 0) ? 1.0 : 0.0;
      for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) {
          down(s->P.F[a * D + c]);
          for (int p = 0; p < np; ++p) F[9 * orig[p] + 3 * a + c] = h[p];
        }
    }
    if (tau) {
      double* d_tau = s->dalloc<double>((size_t)np * 9);
      if (D == 2) ck(launch_stress_out<2>(s->P, s->G, s->d_mats, d_tau, s->st), "stress");
      else ck(launch_stress_out<3>(s->P, s->G, s->d_mats, d_tau, s->st), "stress");
      ck(cudaStreamSynchronize(s->st), "sync");
      ck(cudaMemcpy(tau, d_tau, (size_t)np * 9 * sizeof(double), cudaMemcpyDeviceToHost), "download");
      s->dfree(d_tau);
    }
  });
}

mpm_status mpm_adjoint(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* grad_E, double* grad_phi,
                       double* grad_k) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<AdjointF>(s, dL_dU, dL_dx, grad_E, grad_phi, grad_k); });
}

mpm_status mpm_adjoint_step(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* sbar_x,
                            double* sbar_be, double* sbar_pc, double* sbar_F, double* grad_E, double* grad_phi,
                            double* grad_k) {
  if (!s || !sbar_x || !sbar_be || !sbar_pc || !sbar_F) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    const int np = s->np;
    std::vector<double> sb((size_t)std::max(np, 1) * 19, 0.0);
    for (int p = 0; p < np; ++p) {
      double* q = &sb[(size_t)p * 19];
      for (int a = 0; a < 3; ++a) q[a] = sbar_x[3 * p + a];
      for (int k = 0; k < 6; ++k) q[3 + k] = sbar_be[6 * p + k];
      q[9] = sbar_pc[p];
      for (int k = 0; k < 9; ++k) q[10 + k] = sbar_F[9 * p + k];
    }
    dispatch<AdjointStepF>(s, dL_dU, dL_dx, sb.data(), grad_E, grad_phi, grad_k);
    for (int p = 0; p < np; ++p) {
      const double* q = &sb[(size_t)p * 19];
      for (int a = 0; a < 3; ++a) sbar_x[3 * p + a] = q[a];
      for (int k = 0; k < 6; ++k) sbar_be[6 * p + k] = q[3 + k];
      sbar_pc[p] = q[9];
      for (int k = 0; k < 9; ++k) sbar_F[9 * p + k] = q[10 + k];
    }
  });
}

mpm_status mpm_set_state(mpm_scene* s, const double* x, const double* be, const double* pc, const double* F) {
  if (!s) return MPM_ERR_INVALID_ARG;
  mpm_status rc = guarded(s, [&] {
    const int np = s->np, D = s->D;
    if (!x || np == 0) return;
    for (int p = 0; p < np; ++p)
      for (int a = 0; a < D; ++a) {
        const double sg = (x[3 * p + a] - s->G.o[a]) / s->G.h;
        const double fb = std::floor(sg - 0.5);
        if (!(fb >= 0 && fb <= s->G.n[a] - 2)) fail(MPM_ERR_INVALID_ARG, "particle outside the grid interior");
      }
    ck(cudaStreamSynchronize(s->st), "sync");
    s->staged = false;
    std::vector<int> orig(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    std::vector<double> h(np);
    for (int a = 0; a < D; ++a) {
      for (int p = 0; p < np; ++p) h[p] = x[3 * orig[p] + a];
      ck(cudaMemcpy(s->P.x[a], h.data(), np * sizeof(double), cudaMemcpyHostToDevice), "upload");
    }
  });
  if (rc != MPM_OK) return rc;
  return mpm_set_particles(s, be, pc, F);
}

mpm_status mpm_get_particle_increment(const mpm_scene* cs, double* du_p) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !du_p) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] { dispatch<IncrementF>(s, du_p); });
}

mpm_status mpm_set_params(mpm_scene* s, const double* E_p, const double* phi_p, const double* k_p) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    const int np = s->np;
    for (int p = 0; p < np; ++p) {
      if (E_p && !(E_p[p] > 0)) fail(MPM_ERR_INVALID_ARG, "E_p must be positive");
      if (phi_p && !(phi_p[p] >= 0 && phi_p[p] < 90)) fail(MPM_ERR_INVALID_ARG, "phi_p must be in [0, 90)");
      if (k_p && !(k_p[p] >= 0)) fail(MPM_ERR_INVALID_ARG, "k_p must be >= 0");
    }
    if (k_p && !s->up) fail(MPM_ERR_INVALID_ARG, "k_p needs a u-p scene");
    ck(cudaStreamSynchronize(s->st), "sync");
    s->staged = false;
    if (np == 0) return;
    std::vector<int> orig(np), mat(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    ck(cudaMemcpy(mat.data(), s->P.mat, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    std::vector<double> h(np);
    auto up = [&](double* d) {
      ck(cudaMemcpy(d, h.data(), np * sizeof(double), cudaMemcpyHostToDevice), "upload");
    };
    if (E_p) {
      for (int p = 0; p < np; ++p) h[p] = E_p[orig[p]];
      up(s->P.Ep);
    }
    if (phi_p) {
      for (int p = 0; p < np; ++p) h[p] = phi_p[orig[p]];
      up(s->P.phip);
    }
    if (k_p) {
      for (int p = 0; p < np; ++p) h[p] = k_p[orig[p]] * s->hmats[mat[p]].dkdt_dk;
      up(s->P.kdt);
    }
  });
}

mpm_status mpm_get_pressure(const mpm_scene* cs, double* pp) {
  mpm_scene* s = const_cast<mpm_scene*>(cs);
  if (!s || !pp) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (!s->up) fail(MPM_ERR_INVALID_ARG, "not a u-p scene");
    ck(cudaStreamSynchronize(s->st), "sync");
    const int np = s->np;
    if (np == 0) return;
    std::vector<int> orig(np);
    std::vector<double> h(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    ck(cudaMemcpy(h.data(), s->P.pp, np * sizeof(double), cudaMemcpyDeviceToHost), "download");
    for (int p = 0; p < np; ++p) pp[orig[p]] = h[p];
  });
}

mpm_status mpm_set_traction(mpm_scene* s, int n, const int* particle, const double* f) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    if (n < 0 || (n > 0 && (!particle || !f))) fail(MPM_ERR_INVALID_ARG, "traction arrays");
    const int np = s->np, D = s->D;
    for (int k = 0; k < n; ++k) {
      if (particle[k] < 0 || particle[k] >= np) fail(MPM_ERR_INVALID_ARG, "traction particle out of range");
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(f[3 * k + a])) fail(MPM_ERR_INVALID_ARG, "non-finite traction force");
    }
    ck(cudaStreamSynchronize(s->st), "sync");
    if (!s->P.fext[0]) {
      // allocated on first use, for both the live arrays and the sort target
      for (int a = 0; a < D; ++a) {
        s->P.fext[a] = s->dalloc<double>(np);
        s->Q.fext[a] = s->dalloc<double>(np);
      }
    }
    if (np == 0) return;
    std::vector<int> orig(np), inv(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    for (int p = 0; p < np; ++p) inv[orig[p]] = p;
    std::vector<double> h((size_t)D * np, 0.0);
    for (int k = 0; k < n; ++k)
      for (int a = 0; a < D; ++a) h[(size_t)a * np + inv[particle[k]]] = f[3 * k + a];
    for (int a = 0; a < D; ++a)
      ck(cudaMemcpy(s->P.fext[a], h.data() + (size_t)a * np, np * sizeof(double), cudaMemcpyHostToDevice),
         "upload");
    s->staged = false;
  });
}

mpm_status mpm_set_particles(mpm_scene* s, const double* be, const double* pc, const double* F) {
  if (!s) return MPM_ERR_INVALID_ARG;
  return guarded(s, [&] {
    const int np = s->np, D = s->D;
    for (int p = 0; p < np; ++p) {
      if (be) {
        const double* b = be + 6 * p;
        double m2 = b[0] * b[1] - b[3] * b[3];
        double m3 = b[0] * (b[1] * b[2] - b[4] * b[4]) - b[3] * (b[3] * b[2] - b[4] * b[5]) +
                    b[5] * (b[3] * b[4] - b[1] * b[5]);
        if (!(b[0] > 0 && m2 > 0 && m3 > 0)) fail(MPM_ERR_INVALID_ARG, "be must be positive definite");
        if (D == 2 && (b[4] != 0.0 || b[5] != 0.0)) fail(MPM_ERR_INVALID_ARG, "2D be has no yz/xz parts");
      }
      if (F) {
        const double* f = F + 9 * p;
        double d = f[0] * (f[4] * f[8] - f[5] * f[7]) - f[1] * (f[3] * f[8] - f[5] * f[6]) +
                   f[2] * (f[3] * f[7] - f[4] * f[6]);
        if (!(d > 0)) fail(MPM_ERR_INVALID_ARG, "det(F) must be positive");
      }
    }
    ck(cudaStreamSynchronize(s->st), "sync");
    s->staged = false;
    if (np == 0) return;
    std::vector<int> orig(np);
    ck(cudaMemcpy(orig.data(), s->P.orig, np * sizeof(int), cudaMemcpyDeviceToHost), "download");
    std::vector<double> h(np);
    auto up = [&](double* d) {
      ck(cudaMemcpy(d, h.data(), np * sizeof(double), cudaMemcpyHostToDevice), "upload");
    };
    if (be)
      for (int k = 0; k < s->nbe; ++k) {
        for (int p = 0; p < np; ++p) h[p] = be[6 * orig[p] + k];
        up(s->P.be[k]);
      }
    if (pc) {
      for (int p = 0; p < np; ++p) h[p] = pc[orig[p]];
      up(s->P.pc);
    }
    if (F)
      for (int a = 0; a < D; ++a)
        for (int c = 0; c < D; ++c) {
          for (int p = 0; p < np; ++p) h[p] = F[9 * orig[p] + 3 * a + c];
          up(s->P.F[a * D + c]);
        }
  });
}

mpm_status mpm_footprint_bytes(const mpm_scene_desc* desc, int np, size_t* out) {
  if (!out) return MPM_ERR_INVALID_ARG;
  try {
    validate_desc(desc);
    if (np < 0) return MPM_ERR_INVALID_ARG;
    *out = footprint(desc, np);
    return MPM_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

void mpm_destroy_scene(mpm_scene* s) { destroy(s); }

const char* mpm_status_string(mpm_status st) {
  switch (st) {
    case MPM_OK: return "ok";
    case MPM_ERR_INVALID_ARG: return "invalid argument";
    case MPM_ERR_OOM: return "out of device memory";
    case MPM_ERR_CUDA: return "CUDA error";
    case MPM_ERR_NOT_CONVERGED: return "Newton did not converge";
    case MPM_ERR_KRYLOV_MAXIT: return "Krylov iteration limit";
    case MPM_ERR_KRYLOV_BREAKDOWN: return "Krylov breakdown";
    case MPM_ERR_NONFINITE: return "non-finite value";
    case MPM_ERR_TIMEOUT: return "timeout";
    case MPM_ERR_BOUNDS: return "particle support left the grid";
    case MPM_ERR_RETURN_MAP: return "return map did not converge";
    case MPM_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* mpm_last_error(const mpm_scene* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
