/*
 * mpm_serve.h -- continuous-batching serving loop over implicit-MPM scenes.
 *
 * The paper (GeoWarp, arXiv 2507.09435) runs one simulation at a time; this
 * is a convenience of this library for many independent implicit solves of
 * different sizes and materials arriving over time.  A request is a whole
 * scene plus its schedule of load steps (the paper's Sec. 2.2 load-step loop,
 * mpm_solve_step per step).  The server keeps `slots` worker threads, each
 * with its own CUDA stream; a queued request is admitted, in arrival order,
 * as soon as a slot is free and its device footprint (mpm_footprint_bytes)
 * fits in the memory budget beside the requests already running (a request
 * larger than the budget runs when nothing else does).  Admitted scenes stay
 * resident (particles, sort, Jacobian pattern and matrix) for all their load
 * steps, and the kernels of concurrent scenes overlap on the device.
 *
 * Arrays passed to mpm_server_submit are host arrays, copied at the call.
 * All functions are thread-safe.  Errors: MPM_ERR_INVALID_ARG for bad
 * arguments or an unknown ticket; a request's own failure (non-convergence,
 * a bad scene) is reported in its mpm_request_result, not by the call.
 */
#ifndef MPM_SERVE_H
#define MPM_SERVE_H

#include "mpm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_server mpm_server;

typedef struct {
  const mpm_scene_desc* desc;
  int np;
  const double* x;            /* np*3 positions                                   */
  const double* vol0;         /* np                                               */
  const double* mass;         /* np                                               */
  const int* mat_id;          /* np                                               */
  const double* E_p;          /* np or NULL                                       */
  const double* phi_p;        /* np or NULL                                       */
  const double* pc0_p;        /* np or NULL                                       */
  const double* be0;          /* np*6 initial elastic left Cauchy-Green or NULL   */
  const mpm_material* mats;
  int nmat;
  int ntraction;              /* particle-carried forces (see mpm_set_traction)   */
  const int* traction_particle;
  const double* traction_force;  /* ntraction*3                                   */
  int nsteps;                 /* load steps                                       */
  const int* step_ndof;       /* nsteps: prescribed DOFs of each step             */
  const long long* step_dof;  /* sum(step_ndof): DOF indices, step after step     */
  const double* step_value;   /* sum(step_ndof): prescribed values                */
  const double* step_gravity; /* nsteps*3                                         */
} mpm_request;

typedef struct {
  int status;                 /* mpm_status of the request                        */
  int steps_done;             /* load steps committed                             */
  int newton_iters;           /* over all steps                                   */
  int krylov_iters;
  double t_queue_ms;          /* submit -> admission                              */
  double t_service_ms;        /* admission -> done (scene creation to destruction) */
  double t_latency_ms;        /* submit -> done                                   */
  size_t footprint;           /* admitted device bytes                            */
  int slot;                   /* worker that ran it                               */
} mpm_request_result;

typedef struct {
  int slots;
  size_t budget;              /* device bytes the running requests may take       */
  size_t in_use;              /* footprint of the running requests                */
  size_t peak_in_use;
  int running;
  int peak_running;           /* most requests running at once                    */
  long long submitted, completed, failed;
} mpm_server_stats;

/* Start a server with `slots` workers on the current CUDA device and a memory
 * budget in bytes (0: 80% of the device memory free at the call). */
mpm_status mpm_server_create(int slots, size_t budget_bytes, mpm_server** out);

/* Queue a request; returns at once with its ticket. */
mpm_status mpm_server_submit(mpm_server* sv, const mpm_request* req, long long* ticket);

/* Block until the request is done and copy its result. */
mpm_status mpm_server_wait(mpm_server* sv, long long ticket, mpm_request_result* out);

/* Final particle positions (np*3) and, for MPM_UP scenes, pore pressures (np)
 * of a finished request (either pointer may be NULL). */
mpm_status mpm_server_result_particles(mpm_server* sv, long long ticket, double* x, double* pp);

/* Forget a finished request (its stored result). */
mpm_status mpm_server_release(mpm_server* sv, long long ticket);

mpm_status mpm_server_get_stats(const mpm_server* sv, mpm_server_stats* out);

/* Finish the running requests, drop the queued ones, stop the workers. */
void mpm_server_destroy(mpm_server* sv);

#ifdef __cplusplus
}
#endif

#endif /* MPM_SERVE_H */
