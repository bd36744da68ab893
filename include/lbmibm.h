/*
 * lbmibm.h -- C ABI of the GB300 (sm_103a) library for the coupled D3Q19 BGK
 * lattice Boltzmann step with the Ota-Suzuki-Inamuro multi-direct-forcing
 * immersed boundary loop (Beny & Latt, arXiv:1904.02108).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every function returning int returns LBM_OK (0) on success, a negative
 *    LBM_E* code on error, or the positive warning LBM_WNOTCONVERGED.  On an
 *    error, lbm_last_error(h) returns a static description (valid until the
 *    next call on the same handle).  A NULL handle is LBM_EINVAL.
 *  - Lattice coordinates are lattice units; cell (X, Y, Z) is centred on the
 *    integer point.  The domain is periodic in all three directions.
 *  - Eulerian fields passed in or out are component-major, x fastest:
 *    rho[nz][ny][nx], U[3][nz][ny][nx] (FP32).  Lagrangian vectors are
 *    point-major: v[n][3].
 *  - Host pointers are read (inputs) or written (outputs) during the call;
 *    the library copies inputs and keeps no reference to caller memory
 *    (except the asynchronous calls, which say how long a buffer is used,
 *    and ibm_update_points with mapped host transfers, lbm_set_host_io).
 *    Functions whose name ends in _dev take device pointers instead and are
 *    ordered on the handle's stream.
 *  - All device work is enqueued on the handle's CUDA stream (lbm_set_stream;
 *    default: the legacy default stream).  Calls that return host data
 *    synchronise that stream.
 *  - nx, ny, nz must be positive multiples of 4 (the 4x4x4 brick used to bin
 *    Lagrangian points and to store forces).
 *  - The library allocates its device memory with cudaMalloc at creation and
 *    frees it in lbm_destroy.  One handle must not be used from two host
 *    threads at once.
 */
#ifndef LBMIBM_H
#define LBMIBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)       /* bad argument (dims, tau <= 1/2, n < 0, ...)  */
#define LBM_ENOMEM (-2)       /* device or host allocation failed            */
#define LBM_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed  */
#define LBM_ENONFINITE (-4)   /* NaN/Inf found in inputs or in the FP64 sums  */
#define LBM_ESTATE (-5)       /* state buffer of the wrong size or version    */
#define LBM_WNOTCONVERGED 1   /* warning: IBM iteration cap reached; the step
                                 still completed                             */

/* Population storage: FP32, or 16-bit deviations f_i - t_i. */
#define LBM_STORE_F32 0
#define LBM_STORE_BF16 1
#define LBM_STORE_F16 2

/* Weighting function w(r) of Sec. 3, support |r| < 2. */
#define LBM_DELTA_COSINE 0    /* (1 + cos(pi r / 2)) / 4                      */
#define LBM_DELTA_PESKIN 1    /* Peskin's four-point kernel                   */

/* Initial velocity correction du of each step's fixed point (Sec. 3). */
#define LBM_WARM_ZERO 0       /* du = 0, as in the paper                      */
#define LBM_WARM_PREVIOUS 1   /* du = previous step's final du                */
#define LBM_WARM_MLP 2        /* du = previous du + V * MLP(features), the
                                 learned warm start (mlp_set_weights)        */

typedef struct lbm lbm_t;

typedef struct {
  int nx, ny, nz;      /* lattice size, multiples of 4                        */
  double tau;          /* BGK relaxation time (Eq. 2), > 1/2                  */
  int storage;         /* LBM_STORE_*                                         */
  int delta;           /* LBM_DELTA_*                                         */
  int warm_start;      /* LBM_WARM_*                                          */
  double ibm_tol;      /* residual target when lbm_step gets n_ibm_iter == 0  */
  int ibm_max_iter;    /* iteration cap in that mode                          */
  int stats;           /* 1: accumulate FP64 mass/momentum every step         */
} lbm_opts;

typedef struct {
  double mass;           /* sum over cells and i of f_i after the last step,
                            in FP64: per cell rho, from the step's moments
                            (the BGK collision conserves it exactly)        */
  double momentum[3];    /* sum of e_i f_i after the last step: per cell
                            rho U + rho G (the collision adds exactly the
                            force impulse rho G, Eqs. 2-3)                   */
  int64_t step;          /* number of completed steps                         */
  int last_ibm_iters;    /* fixed-point iterations of the last step           */
  double last_residual;  /* eps of the last iteration (tolerance mode), else
                            -1                                                */
  int64_t not_converged; /* steps that hit the iteration cap                  */
  int64_t active_bricks; /* 4x4x4 bricks in the support of the points         */
  int64_t kernel_launches; /* kernels launched by this handle so far          */
} lbm_stats;

/* ---- lifetime -------------------------------------------------------- */

/* Default options: tau 0.8, FP32 storage, cosine kernel, zero warm start,
 * ibm_tol 1e-4, ibm_max_iter 500, stats on. */
void lbm_default_opts(lbm_opts *o);

/* Lattice at rest: f_i = t_i (rho = 1, U = 0) on every cell (Sec. 2).
 * Errors: LBM_EINVAL (dims not positive multiples of 4, tau <= 1/2, out
 * NULL), LBM_ENOMEM, LBM_ECUDA.  On error *out is set to NULL. */
int lbm_create(int nx, int ny, int nz, double tau, lbm_t **out);
int lbm_create_ex(const lbm_opts *o, lbm_t **out);

/* Frees every device buffer of the handle.  NULL is a no-op. */
void lbm_destroy(lbm_t *h);

/* Description of the last error on h (h may be NULL: last creation error). */
const char *lbm_last_error(const lbm_t *h);

/* Stream for all further work of h (a cudaStream_t; NULL = legacy default). */
int lbm_set_stream(lbm_t *h, void *stream);

/* ---- the immersed object (Sec. 3, Alg. 1) ----------------------------- */

/* Lagrangian points of the immersed surface.
 *  X[n][3]        FP64 positions.  With bodies (ibm_set_bodies), the rest
 *                 pose to which the rigid transform M(t) applies; without,
 *                 fixed positions.
 *  U_target[n][3] surface velocity u_k used when no bodies are set (NULL:
 *                 zero).  Ignored when bodies are set (u_k = x(t) - x(t-1)).
 *  area[n]        s(k), the surface area a point represents (NULL: 1).
 *  body[n]        body index of each point (NULL: 0).
 * n = 0 removes all points.  Replaces any previous set and resets the warm
 * start.  Errors: LBM_EINVAL (n < 0, X NULL with n > 0, body index out of
 * range of the bodies set), LBM_ENONFINITE (NaN/Inf in any input),
 * LBM_ENOMEM, LBM_ECUDA. */
int ibm_set_points(lbm_t *h, int64_t n, const double *X, const float *U_target,
                   const float *area, const int32_t *body);

/* Moves the current points: new X[n][3] (and U_target[n][3] when not NULL)
 * for the same n points, copied from host memory on the handle's stream
 * (asynchronously for page-locked memory; the caller keeps the buffers valid
 * until the stream has passed the copy).  No reallocation, no
 * synchronisation, areas, bodies and the warm-start history are kept: the
 * per-step input of a caller that moves its own points (the paper's
 * immersedBoundary(object, U) with the object updated each step).  Positions
 * are not checked here; a non-finite one gives an unspecified point, never an
 * out-of-range access.  With mapped host transfers (lbm_set_host_io) the
 * buffers are instead read by the next step's kinematics; when the last step
 * ran as a one-step call in that mode, the next step's kinematics and pair
 * lists start at this call, on an internal stream beside that step's
 * collide (the next lbm_step takes them; a later ibm_update_points,
 * ibm_set_points, ibm_set_bodies, lbm_set_time, lbm_set_host_io,
 * lbm_load_state, lbm_save_state, lbm_read_stats, lbm_autotune, a batched or
 * replayed step discards them, the positions staying uploaded).  This entry
 * point has no counterpart in the paper.
 * Errors: LBM_EINVAL (n differs from the point count, X NULL), LBM_ECUDA. */
int ibm_update_points(lbm_t *h, int64_t n, const double *X, const float *U_target);

/* Rigid rotating bodies: M_b(t) rotates by phase[b] + omega[b] * t radians
 * about the z axis through centre[b][3] (Alg. 1 applies M(t) at the first
 * fixed-point iteration; u_k = x(t) - x(t-1)).  nb = 0 removes the bodies
 * (points become fixed).  t counts completed steps. */
int ibm_set_bodies(lbm_t *h, int nb, const double *centre, const double *omega,
                   const double *phase);

/* Uniform body force added to G on every cell (test hook for Poiseuille
 * flow; not in the paper). */
int lbm_set_body_force(lbm_t *h, double gx, double gy, double gz);

/* ---- time stepping (Sec. 2 summary, Sec. 3 fixed point) --------------- */

/* Advances n_steps coupled steps.  Each step: rho, U from the populations
 * (Eq. 1) on the bricks around the points; the multi-direct-forcing fixed
 * point (Sec. 3) for G; U^G = U + tau G; BGK collision (Eqs. 2-3) and
 * streaming (Eq. 4) on every cell.  n_ibm_iter > 0: exactly that many
 * fixed-point iterations (the paper uses 5).  n_ibm_iter == 0: iterate until
 * the residual eps = ||S[s g_n]|| / ||S[s u_k]|| <= ibm_tol or ibm_max_iter
 * iterations; returns LBM_WNOTCONVERGED if any step hit the cap.
 * Errors: LBM_EINVAL (n_steps < 0, n_ibm_iter < 0), LBM_ECUDA.  The call
 * does not wait for the GPU: a step whose FP64 mass or momentum sum is not
 * finite (stats on) is reported as LBM_ENONFINITE by the next
 * lbm_read_stats.  In a call of several eager steps (no captured graphs, no
 * stage timing, no overlapped step) the kinematics and pair lists of each
 * step after the first are built on an internal stream while the step
 * before it collides; the results are bitwise those of one-step calls, and
 * no work of a later step is left pending when the call returns. */
int lbm_step(lbm_t *h, int n_steps, int n_ibm_iter);

/* The iteration that solves the fixed point of Sec. 3 in lbm_step.
 * LBM_SOLVER_MDF (default): the multi-direct-forcing loop of the paper,
 * du += s g_n, G_{n+1} = G_n + S[s g_n].  LBM_SOLVER_CG: conjugate gradients
 * on the same fixed point written on the lattice, B G = c with
 * B = S diag(s) I and c = S[s (u_k - I[U0])] (the paper's loop is
 * Richardson's iteration with unit step on this system, and eps is the norm
 * of its residual); B is symmetric positive semi-definite and c in its range,
 * so CG converges where the point-space system is singular.  Not in the
 * paper (a Krylov replacement for the loop).  Both reach the same force; an
 * iteration of either is one gather of the brick pass and one interpolation,
 * with the same eps, warm starts and outputs (du; u_interp of the last
 * iteration's iterate).  In tolerance mode CG confirms each stop on the
 * true residual u_k - I[U0 + S[du]] (its FP32 recursion drifts from it) and
 * returns the iterate whose true residual met ibm_tol.  Not part of the
 * saved state.  Returns LBM_OK or LBM_EINVAL (NULL h, unknown solver). */
#define LBM_SOLVER_MDF 0
#define LBM_SOLVER_CG 1
int ibm_set_solver(lbm_t *h, int solver);
int ibm_get_solver(const lbm_t *h);   /* -1 for NULL h */

/* How U (Eq. 1) is pre-computed before the fixed point on the cells the
 * interpolation reads (Sec. 5: U is needed only near the surfaces).
 * LBM_U0_BRICKS (default): every cell of the 4x4x4 bricks that some point's
 * support touches, each cell once.  LBM_U0_BOX: the paper's box strategy,
 * every cell of each body's bounding box (the box of its points' rest
 * positions moved by M(t), widened by the support and rounded out to whole
 * bricks; for points without bodies, the box of their positions) into a
 * full-lattice U, as in the paper, from which the active bricks take their
 * cells; allocates 12 B per cell on first use and recomputes the boxes from
 * the host positions of ibm_set_points / ibm_update_points.  LBM_U0_KERNEL:
 * the paper's kernel strategy, the cells of every point's support (its 4 x 4
 * x 4 taps: the fifth tap of the paper's 5 x 5 x 5 block has weight 0), a
 * cell computed once per support that covers it.  All three give bitwise the
 * same steps; they differ in work and memory traffic.  Single lattices only
 * (lbm_batch_step refuses other strategies).  Not part of the saved state.
 * Returns LBM_OK, LBM_EINVAL (NULL h, unknown strategy) or LBM_ENOMEM. */
#define LBM_U0_BRICKS 0
#define LBM_U0_BOX 1
#define LBM_U0_KERNEL 2
int lbm_set_u0_strategy(lbm_t *h, int strategy);
int lbm_get_u0_strategy(const lbm_t *h);   /* -1 for NULL h */

/* Current step counter t (completed steps); lbm_set_time overrides it. */
int64_t lbm_time(const lbm_t *h);
int lbm_set_time(lbm_t *h, int64_t t);

/* ---- reading results ------------------------------------------------- */

/* rho[N], U[3][N] of the current populations (Eq. 1) and G[3][N], the
 * force field applied in the last step (zero away from the points).  Any
 * output may be NULL.  Host buffers (lbm_read_fields) or device buffers
 * (lbm_read_fields_dev). */
int lbm_read_fields(lbm_t *h, float *rho, float *U, float *G);
int lbm_read_fields_dev(lbm_t *h, float *rho, float *U, float *G);

/* Per-point results of the last step, point order of ibm_set_points:
 * x[n][3] positions x(t) (FP64), u_interp[n][3] velocity interpolated at the
 * last iteration u_n(k), du[n][3] the velocity correction du(k) (Sec. 3).
 * Any output may be NULL. */
int ibm_read_points(lbm_t *h, double *x, float *u_interp, float *du);
int ibm_read_points_dev(lbm_t *h, double *x, float *u_interp, float *du);

/* Statistics; the FP64 sums are those of the last step with stats on.
 * Returns LBM_ENONFINITE (with the statistics filled in) when one of those
 * sums is NaN or infinite. */
int lbm_read_stats(lbm_t *h, lbm_stats *s);

/* Non-blocking read-back into host memory: the same values as
 * ibm_read_points and as the sums of lbm_read_stats (sums[4] = mass,
 * momentum x, y, z; left unchanged when the lattice has no sums yet), with
 * the device-to-host copies enqueued on the handle's stream and no
 * synchronisation.  The values are in the caller's buffers once the stream
 * has passed the call (cudaStreamSynchronize, or an event recorded after it);
 * the buffers must stay valid until then, and page-locked (pinned) host
 * memory makes the copies asynchronous.  A later read-back of the same kind
 * is ordered after this one on the stream.  No counterpart in the paper
 * (pipelined host I/O).  Returns LBM_OK, LBM_EINVAL (NULL h or sums) or
 * LBM_ECUDA. */
int ibm_read_points_async(lbm_t *h, double *x, float *u_interp, float *du);
int lbm_read_sums_async(lbm_t *h, double *sums);

/* How ibm_update_points, ibm_read_points_async and lbm_read_sums_async move
 * data between host and device (no counterpart in the paper: pipelined host
 * I/O of a caller that moves its points every step).
 *  LBM_HOST_IO_COPY (default): copies enqueued on the handle's stream.
 *  LBM_HOST_IO_MAPPED: for page-locked host buffers with a device mapping
 *    (cudaHostAlloc / cudaMallocHost, or registered with
 *    cudaHostRegisterMapped), the kernels access the host memory directly
 *    (over NVLink-C2C on a Grace-Blackwell node), so that no copy operation
 *    sits between the kernels of consecutive steps: the positions / targets
 *    of ibm_update_points are read by the kinematics of the next step (which
 *    writes them through to the handle's device copy), and the read-outs are
 *    written by small kernels on the handle's stream.  The caller keeps an
 *    uploaded buffer unchanged until the next step has run (an event recorded
 *    on the stream after that lbm_step has completed), and a read-out buffer
 *    valid until the stream has passed the call, as for asynchronous copies.
 *    A one-step call in this mode records an event after its fixed point, so
 *    that the next upload can start the next step's kinematics and pair
 *    lists beside this step's collide (see ibm_update_points).
 *    A step replayed from a captured graph, a batched step and lbm_save_state
 *    copy a pending upload in stream order first.  Buffers that are not
 *    device-mapped host memory are copied as in LBM_HOST_IO_COPY.
 * Values and results are bitwise those of LBM_HOST_IO_COPY.  Switching to
 * LBM_HOST_IO_COPY copies a pending upload first.  Errors: LBM_EINVAL (NULL
 * handle or mode pointer, unknown mode), LBM_ECUDA. */
#define LBM_HOST_IO_COPY 0
#define LBM_HOST_IO_MAPPED 1
int lbm_set_host_io(lbm_t *h, int mode);
int lbm_get_host_io(lbm_t *h, int *mode);

/* Full populations f[19][N] (FP32) of the current state, in the velocity
 * order of lbm_velocity_set, and their replacement.  Host buffers.
 * lbm_write_populations returns LBM_ENONFINITE, and leaves the state as it
 * was, when a value is NaN or infinite. */
int lbm_read_populations(lbm_t *h, float *f);
int lbm_write_populations(lbm_t *h, const float *f);

/* The stored deviations d_i = f_i - t_i (FP32 values of the storage type),
 * same layout and pull offset as lbm_read_populations.  Host buffer. */
int lbm_read_deviations(lbm_t *h, float *d);

/* Residual eps_n = ||S[s g_n]|| / ||S[s u_k]|| of every fixed-point iteration
 * of the last step in tolerance mode (Sec. 3 stops when g is "negligibly
 * small"; the norm is over the lattice, in FP64; if every u_k vanishes the
 * denominator is ||S[s (u_k - I[U0])]||).  Writes min(n, cap) values and
 * returns n, the number of iterations of that step; 0 after a fixed-count
 * step. */
int lbm_read_residuals(lbm_t *h, double *eps, int cap);

/* The D3Q19 velocity set e[19][3] and weights t[19] the library uses. */
void lbm_velocity_set(int *e, double *t);

/* ---- launch shapes and the autotuner ----------------------------------- */

/* How the step kernels spread their work over the GPU.  No field depends on
 * it: every launch shape gives bitwise the same populations, forces, point
 * values and FP64 sums (the paper fixes the kernels' work, not their launch
 * geometry; this is a GB300 tuning knob with no counterpart there). */
typedef struct {
  int collide_block; /* threads per block of the collide-stream kernel:
                        128 or 256                                         */
  int brick_blocks;  /* blocks of the brick kernels (one warp each,
                        grid-stride over the active bricks), >= 1          */
  int point_block;   /* threads per block of the per-point kernels:
                        128, 256 or 512                                    */
  int moments_spb;   /* bricks per block of the moments kernel: 1, 2 or 4   */
  int sort_blocks;   /* blocks of the pair sort (a warp per brick), >= 1   */
  int collide_staged; /* 16-bit storage: 0 pulls two x-neighbouring cells
                         per thread with 4-byte loads; 1 (single lattice)
                         brings the pulled rows into shared memory with
                         bulk asynchronous copies (rows of 8k cells,
                         16-byte aligned; other sizes fall back to 0); 2
                         takes four cells per thread (8-byte loads and
                         stores, blocks of 128 whatever collide_block)     */
  int sort_blocks_ahead; /* blocks of the pair sort of a step prepared while
                            the step before it collides (lbm_step), >= 1  */
} lbm_launch_shape;

/* The handle's launch shape (defaults: 256, 9728, 256, 4, 4864, 2, 608).  Set
 * returns LBM_EINVAL for a value outside the ranges above. */
int lbm_get_launch_shape(lbm_t *h, lbm_launch_shape *out);
int lbm_set_launch_shape(lbm_t *h, const lbm_launch_shape *s);

/* Picks the launch shape by timing trial steps on this handle's own lattice
 * and points: one parameter at a time (collide block, brick grid, point
 * block, moments bricks per block, sort grid, and with 16-bit storage the
 * staged collide), each candidate timed with CUDA
 * events around steps_per_trial whole steps (>= 1; consecutive kernels
 * overlap, so the step is the objective) after one untimed step, in two
 * interleaved rounds (the faster kept), with n_ibm_iter (> 0) fixed
 * iterations; a candidate replaces the current value only when more than 1 %
 * faster.  The lattice is restored afterwards (populations, corrections,
 * step counter, sums), so the
 * call does not advance the simulation; it allocates a copy of one
 * population lattice for that.  The chosen shape is set on the handle and
 * written to *chosen (may be NULL).  Stage timing is off on return. */
int lbm_autotune(lbm_t *h, int n_ibm_iter, int steps_per_trial, lbm_launch_shape *chosen);

/* on != 0: in a step with points, the cells outside that
 * step's active bricks (those no point's support reaches, which need no IBM
 * force, Sec. 2 step 3 with G = body force) collide on the handle's stream
 * while the IBM stages (Sec. 3, Algs. 1-2) run on an internal stream of the
 * greatest priority; the cells of the active bricks collide after the IBM
 * loop on that stream, and the two meet before the step ends.  Every cell's
 * arithmetic is the same either way; only the grouping of the FP64 partial
 * sums of lbm_stats differs.  on == 0 (the default): one collide launch over
 * every cell after the IBM loop, all on the handle's stream.  On a dense
 * propeller array the overlapped step is slower (the latency-bound IBM
 * kernels get SM slots only as collide blocks retire, and the collide's
 * stream through L2 evicts their working set).  No counterpart in the paper
 * (a scheduling choice).  Returns LBM_OK or LBM_EINVAL (NULL h). */
int lbm_set_overlap(lbm_t *h, int on);

/* ---- captured steps and batches of lattices ------------------------------ */

/* on != 0: lbm_step with n_ibm_iter > 0 captures two consecutive steps into
 * a CUDA graph once the warm-start history is steady, and replays it for
 * every further pair of steps (a new capture follows any change of points,
 * bodies, options or iteration count).  Stage timing is not recorded inside
 * replayed steps.  Work is ordered on the handle's stream through events. */
int lbm_set_graph(lbm_t *h, int on);

/* A batch advances several lattices (different sizes, points and bodies)
 * together: each stage of the step is one kernel launch over all of them.
 * The handles stay owned by the caller and must not be destroyed before the
 * batch; they must share the storage format, the stats option, the warm-start
 * mode and history, the stream, and be at the same lattice parity (created
 * together or stepped together).  Results are read through the individual
 * handles.  n_ibm_iter > 0: that many fixed-point iterations in every
 * domain.  n_ibm_iter == 0 (the paper's loop only, every handle with the
 * same ibm_tol and ibm_max_iter): every domain iterates until its own
 * residual meets ibm_tol or the cap, exactly the iterations it would take
 * alone (lbm_read_residuals and lbm_read_stats per handle); returns
 * LBM_WNOTCONVERGED if a domain hit the cap.  Captured graphs are used for
 * fixed counts only. */
typedef struct lbm_batch lbm_batch_t;
int lbm_batch_create(int n, lbm_t *const *handles, lbm_batch_t **out);
int lbm_batch_step(lbm_batch_t *b, int n_steps, int n_ibm_iter);
int lbm_batch_set_graph(lbm_batch_t *b, int on);
void lbm_batch_destroy(lbm_batch_t *b);
/* A batch launches with its own shape: the first handle's at creation, or
 * the one lbm_batch_set_launch_shape / lbm_batch_autotune set (the autotuner
 * times whole batch steps, n_ibm_iter > 0, and restores every lattice). */
int lbm_batch_get_launch_shape(lbm_batch_t *b, lbm_launch_shape *out);
int lbm_batch_set_launch_shape(lbm_batch_t *b, const lbm_launch_shape *s);
int lbm_batch_autotune(lbm_batch_t *b, int n_ibm_iter, int steps_per_trial,
                       lbm_launch_shape *chosen);

/* ---- instrumentation -------------------------------------------------- */

/* Stage timing with CUDA events recorded on the handle's stream around the
 * stages of lbm_step selected by `mask` (bit i = stage i; LBM_TIME_ALL for
 * every stage; 0 disables).  Each call clears the accumulated times.  Stage
 * names: lbm_stage_name(i) for i < lbm_num_stages(); lbm_read_timing
 * synchronises the stream, then ms[i] holds the accumulated event time and
 * launches[i] the number of kernel launches timed in stage i. */
#define LBM_TIME_ALL 0x7fffffff
int lbm_enable_timing(lbm_t *h, int mask);
int lbm_num_stages(void);
const char *lbm_stage_name(int i);
int lbm_read_timing(lbm_t *h, double *ms, int64_t *launches);

/* ---- checkpoint / resume ---------------------------------------------- */

/* Serialises populations, points, bodies, warm-start state and the step
 * counter.  buf == NULL: *len receives the size.  Resume is bitwise exact. */
int lbm_save_state(lbm_t *h, void *buf, size_t *len);
int lbm_load_state(lbm_t *h, const void *buf, size_t len);

/* ---- stateless operators on caller device memory --------------------- */

/* Interpolation, fluid -> surface (Sec. 3, Alg. 1):
 *   u(k) = sum_X U(X) w(x_k - X) w(y_k - Y) w(z_k - Z)
 * U: device [3][nz][ny][nx] FP32; x: device [n][3] FP64; u: device [n][3]
 * FP32 (written).  Enqueued on `stream`.  Errors: LBM_EINVAL, LBM_ECUDA. */
int ibm_interpolate_dev(int nx, int ny, int nz, int delta, const float *U,
                        int64_t n, const double *x, float *u, void *stream);

/* Spreading, surface -> fluid (Sec. 3, Alg. 2), without atomics:
 *   F(X) = sum_k v(k) w(x_k - X) w(y_k - Y) w(z_k - Z)
 * F: device [3][nz][ny][nx] FP32, overwritten (zero away from the points).
 * scratch: device memory of ibm_spread_scratch_bytes(nx,ny,nz,n) bytes, at
 * least 256-byte aligned, owned by the caller; NULL makes the call allocate
 * and free it itself.  Enqueued on `stream`. */
size_t ibm_spread_scratch_bytes(int nx, int ny, int nz, int64_t n);
int ibm_spread_dev(int nx, int ny, int nz, int delta, int64_t n,
                   const double *x, const float *v, float *F, void *scratch,
                   void *stream);

/* ---- learned warm start (not in the paper) ------------------------------ */

/* Per-point MLP y = W3 s(W2 s(W1 x + b1) + b2) + b3, s(v) = v / (1 + e^-v),
 * x in R^16, two hidden layers of 64, y in R^3.  Parameters P: FP32 vector of
 * LBM_MLP_NPARAM values [W1 (64x16, row-major out x in), b1, W2 (64x64), b2,
 * W3 (3x64), b3].  The kernels run on BF16 tensor cores with FP32
 * accumulation from a packed BF16 copy of P (mlp_pack_dev).
 *
 * Features of point k (velocities / LBM_MLP_VSCALE, lengths /
 * LBM_MLP_LSCALE): u_i = I[U0 + S[du_prev]](k), the velocity interpolated
 * with the previous step's force applied (3), u_k (3), the previous step's
 * du (3), local point density (pairs of its bricks per brick cell) (1),
 * radius and axial offset from its body's axis and omega r (3), u_k - u_i
 * (3).  In LBM_WARM_MLP mode the fixed point starts from
 * du_prev + V * MLP(x). */
#define LBM_MLP_NPARAM 5443
#define LBM_MLP_VSCALE 0.05
#define LBM_MLP_LSCALE 16.0

size_t mlp_packed_bytes(void);
int mlp_pack_dev(const float *P, void *packed, void *stream);
/* Y[n][3] = MLP(X[n][16]); device pointers. */
int mlp_forward_dev(int64_t n, const float *X, const void *packed, float *Y, void *stream);
/* grad (device, LBM_MLP_NPARAM floats) and *loss (device float, may be
 * NULL) of the mean 0.5 |MLP(x) - t|^2 over X[n][16], T[n][3];
 * P is the FP32 parameter vector packed as `packed`; scratch: device memory
 * of mlp_grad_scratch_bytes(n) bytes. */
size_t mlp_grad_scratch_bytes(int64_t n);
int mlp_loss_grad_dev(int64_t n, const float *X, const float *T, const float *P,
                      const void *packed, float *grad, float *loss, void *scratch,
                      void *stream);
/* One Adam step (bias-corrected, step >= 1) on P with moments m, v (device,
 * LBM_MLP_NPARAM floats each); repacks into `packed` if not NULL. */
int mlp_adam_dev(float *P, float *m, float *v, const float *grad, int64_t step, double lr,
                 double beta1, double beta2, double eps, void *packed, void *stream);
/* Weights of the learned warm start of h (host or device FP32 vector). */
int mlp_set_weights(lbm_t *h, const float *P);
int mlp_set_weights_dev(lbm_t *h, const float *P);
/* Compute the features every step even without the learned start (for
 * generating training data). */
int lbm_set_features(lbm_t *h, int on);
/* Training sample of the last step: X[n][16] its features, T[n][3] =
 * (final du - previous du) / LBM_MLP_VSCALE; device buffers. */
int ibm_read_mlp_sample_dev(lbm_t *h, float *X, float *T);

/* ---- spreading without any allocation ---------------------------------- */

/* Size of the library's static scratch area on each device (16 MiB). */
#define LBM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* Same result as ibm_spread_dev, for callers that cannot allocate device
 * memory: code embedded in a host application whose memory pool owns the
 * whole device, or a time-critical loop that must not pay cudaMalloc's
 * implicit device synchronisation.  The paper has no counterpart; this is a
 * service of the library.
 *
 * Inputs and output are the caller's, exactly as for ibm_spread_dev.  The
 * scratch space is a static device array of LBM_NOALLOC_SCRATCH_BYTES that
 * every device which loads the library keeps until the process exits; the
 * call allocates and frees nothing.  Problems whose
 * ibm_spread_scratch_bytes(nx, ny, nz, n) exceeds that size are rejected with
 * LBM_EINVAL (for example 64^3 with 12,000 points needs about 4.3 MiB).
 *
 * The first call on a device (the current device when it is made) looks up
 * the array's device address and keeps it for the rest of the process; make
 * that first call before any stream capture begins.  After cudaDeviceReset
 * on a device (or any other teardown of its primary context) the kept
 * address is stale: do not call this entry point on that device again.  The
 * descriptor of the problem goes to the device as a kernel parameter, not
 * as a copy from host memory.  All calls on a device share the one array
 * and it keeps the previous call's contents (the call clears what must start
 * at zero), so
 * calls that overlap on the GPU, on different streams or from different host
 * threads, race: serialise them. */
int ibm_spread_dev_noalloc(int nx, int ny, int nz, int delta, int64_t n,
                           const double *x, const float *v, float *F, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBMIBM_H */
