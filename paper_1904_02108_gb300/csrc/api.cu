// C ABI of the library (include/lbmibm.h): handle lifetime, argument checks,
// device memory, and the host orchestration of one time step:
//
//   kinematics -> binning -> moments on active bricks -> n x (interpolation,
//   spreading) -> fused collide-stream -> FP64 sums
//
// all enqueued on the handle's stream.  No CPU fallback exists: every step of
// the method runs in the kernels of lbm.cu and ibm.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbmibm.h"
#include "kernels.h"

using namespace lbmibm;

namespace {

const char *kStageNames[] = {"kinematics",   "pairs",          "brick_init", "point_update",
                             "brick_spread", "collide_stream", "stats",      "residual",
                             "mlp",          "collide_active"};
constexpr int kNumStages = 10;
enum Stage {
  ST_KIN,
  ST_PAIRS,
  ST_INIT,
  ST_UPDATE,
  ST_SPREAD,
  ST_COLLIDE,
  ST_STATS,
  ST_RESID,
  ST_MLP,
  ST_COLLIDE_ACTIVE
};
// the fewest iterations launched between two host checks of the
// tolerance-mode stop flag
constexpr int kCheckChunk = 16;
constexpr int kCgChunk = 4;

thread_local std::string g_create_error;

size_t storage_bytes(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

}  // namespace

struct lbm {
  Geometry g{};
  double tau = 0.8;
  int storage = 0, delta = 0, warm = 0, max_iter = 500, stats_on = 1;
  double tol = 1e-4;
  cudaStream_t st = nullptr;

  void *f[2] = {nullptr, nullptr};
  int cur = 0;

  // immersed points
  int64_t np = 0, cap_np = 0;
  int nb = 0, max_body = -1;
  double *X = nullptr;
  int *body = nullptr;
  float *area = nullptr, *utarget = nullptr;
  double *centre = nullptr, *omega = nullptr, *phase = nullptr;
  PointPrep pp{};
  BrickMap m{};
  PairMap pm{};
  float *U0s = nullptr, *Gs = nullptr, *res = nullptr;
  float4 *du = nullptr, *uint = nullptr;
  float4 *cg = nullptr;       // [5][np] conjugate-gradient point vectors
  double *cg_part = nullptr;  // [ceil(np / 256)][2] block sums of delta, rho
  double *xpos = nullptr;
  bool have_du = false;
  int solver = LBM_SOLVER_MDF;  // the fixed point's iteration
  // U0 pre-computation (LBM_U0_*); the box strategy's rest-pose boxes per
  // body (host copy, uploaded to rest_box when box_dirty) and full-lattice U
  int u0_mode = LBM_U0_BRICKS;
  std::vector<double> box_host;
  std::vector<int> body_host;  // body of each point as given (empty: all 0)
  double *rest_box = nullptr;
  int nbox = 0, cap_box = 0;
  bool box_dirty = false;
  float *Ufull = nullptr;
  // the surface velocities are known not to vanish (rotating bodies, or
  // non-zero targets given to ibm_set_points): tolerance mode then needs no
  // host check of the residual denominator before iterating
  bool bodies_moving = false, targets_nonzero = false;
  double gbody[3] = {0, 0, 0};
  int64_t t = 0;

  // overlap: the collide of the cells outside the active bricks runs on st
  // while the IBM stages and the active bricks' collide run on ibm_st
  // (higher priority); off by default (slower on dense arrays, where the
  // latency-bound IBM kernels lose their SM slots and L2 to the collide)
  bool overlap = false;
  cudaStream_t ibm_st = nullptr, ibm_cap = nullptr;  // ibm_cap: inside captures
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double *slot_partial = nullptr;

  // statistics
  double *partial = nullptr, *sums = nullptr, *red_scratch = nullptr;
  unsigned *ticket = nullptr;
  int nparts = 0;
  bool sums_valid = false;
  int last_iters = 0;
  int tol_hint = 0;  // iterations of the last tolerance-mode step
  double last_eps = -1.0;
  int64_t not_converged = 0;
  IbmState *state = nullptr;       // device
  IbmState *state_host = nullptr;  // pinned mirror of the header fields

  // device descriptor of this lattice (a batch of one) and the step counter
  DomainDesc *desc = nullptr;
  DomainDesc desc_host{};
  // Steps prepared ahead: a step's kinematics and pair lists built on ahead_st
  // while the step before it collides.  The prepared step writes the other of
  // two brick maps (the colliding step still reads its own), so it runs on
  // desc_alt, the descriptor identical to desc but for the brick map; the two
  // swap when it becomes the current step.
  DomainDesc *desc_alt = nullptr;
  DomainDesc desc_host_alt{};
  int *bslot_alt = nullptr;
  cudaStream_t ahead_st = nullptr;
  cudaEvent_t ev_ahead_go = nullptr, ev_ahead_done = nullptr;
  bool pairs_ahead = false;  // the next step's pairs are built (or on their way)
  double *xpos_alt = nullptr;  // the prepared step's positions (read-outs keep xpos)
  // ev_ahead_go marks the end of the last step's fixed point, so that moved
  // points given by ibm_update_points can have the next step prepared at once
  bool loop_mark = false;
  // the end-of-step sums of a step followed by another in the same call run
  // on ahead_st after its collide (ev_collided), joined before the next
  // collide (ev_finished), which rewrites the partials they read
  cudaEvent_t ev_collided = nullptr, ev_finished = nullptr;
  bool finish_pending = false;
  int64_t *t_dev = nullptr;
  bool desc_dirty = true;
  uint64_t version = 1;  // changes whenever a pointer in the descriptor does

  // captured steps (fixed iteration count)
  bool graph_on = false;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_iters = -1, g_cur = -1;
  uint64_t g_version = 0;
  int64_t g_launches = 0;

  // learned warm start
  bool features_on = false;
  float *feat = nullptr;           // [np][16] features of the last step
  float *mlp_P = nullptr;          // [MLP_NPARAM] FP32 weights
  void *mlp_packed = nullptr;      // BF16 packed copy
  int64_t nlaunch = 0;

  // timing
  int timing = 0;  // stage mask
  struct Pending {
    int stage;
    cudaEvent_t a, b;
    int launches;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  double ms[kNumStages] = {0};
  int64_t launches[kNumStages] = {0};

  // launch shapes of the step kernels (lbm_autotune)
  LaunchShape shape;

  // read-out temporaries (allocated on first use)
  float *tmp = nullptr;
  size_t tmp_bytes = 0;

  // host transfers (lbm_set_host_io).  LBM_HOST_IO_MAPPED: uploads from and
  // read-outs into page-locked host memory are done by kernels through its
  // device mapping (no copy operations between the steps' kernels).  x_src /
  // u_src: the device addresses of the last ibm_update_points' mapped
  // buffers, read by the next step's kinematics and written through to X /
  // utarget (or copied there before a replayed or batched step).
  int host_io = LBM_HOST_IO_COPY;
  const double *x_src = nullptr;
  const float *u_src = nullptr;

  std::string err;
};

namespace {

int fail(lbm_t *h, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(lbm_t *h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return code;
}

#define CK(h, call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                        \
  } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc((void **)p, count * sizeof(T));
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

cudaEvent_t get_event(lbm_t *h) {
  if (!h->free_events.empty()) {
    cudaEvent_t e = h->free_events.back();
    h->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Times the launches of a stage on stream s with events (when the stage's
// timing is on) and counts them.
struct StageTimer {
  lbm_t *h;
  int stage;
  int n;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(lbm_t *h_, int stage_, cudaStream_t s_, int n_ = 1)
      : h(h_), stage(stage_), n(n_), s(s_) {
    if (h->timing & (1 << stage)) {
      a = get_event(h);
      if (a) cudaEventRecord(a, s);
    }
    h->nlaunch += n;
  }
  ~StageTimer() {
    if (a) {
      cudaEvent_t b = get_event(h);
      if (b) {
        cudaEventRecord(b, s);
        h->pending.push_back({stage, a, b, n});
      }
    }
  }
};

int ensure_tmp(lbm_t *h, size_t bytes) {
  if (h->tmp_bytes >= bytes) return LBM_OK;
  dfree(h->tmp);
  h->tmp_bytes = 0;
  CK(h, cudaMalloc((void **)&h->tmp, bytes));
  h->tmp_bytes = bytes;
  return LBM_OK;
}

// The device address of page-locked, device-mapped host memory p, else NULL
// (pageable memory, device memory, NULL).
const void *mapped_ptr(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}


// Moves mapped uploads still to be read into X / utarget with copies on s
// (before a step whose kinematics will not read them itself).
int flush_points(lbm_t *h, cudaStream_t s) {
  if (h->x_src)
    CK(h, cudaMemcpyAsync(h->X, h->x_src, sizeof(double) * 3 * h->np, cudaMemcpyDefault, s));
  if (h->u_src)
    CK(h, cudaMemcpyAsync(h->utarget, h->u_src, sizeof(float) * 3 * h->np, cudaMemcpyDefault,
                          s));
  h->x_src = nullptr;
  h->u_src = nullptr;
  return LBM_OK;
}

void free_points(lbm_t *h) {
  h->x_src = nullptr;
  h->u_src = nullptr;
  dfree(h->X);
  dfree(h->body);
  dfree(h->area);
  dfree(h->utarget);
  dfree(h->pp.base);
  dfree(h->pp.wts);
  dfree(h->pp.ut);
  dfree(h->du);
  dfree(h->uint);
  dfree(h->cg);
  dfree(h->cg_part);
  dfree(h->xpos);
  dfree(h->xpos_alt);
  dfree(h->m.slot_brick);
  dfree(h->m.order);
  dfree(h->pm.count);
  dfree(h->pm.start);
  dfree(h->pm.cursor);
  dfree(h->pm.k);
  dfree(h->pm.brick);
  dfree(h->pm.w);
  dfree(h->pm.part);
  dfree(h->pm.point_pairs);
  h->pm.max_pairs = 0;
  dfree(h->feat);
  dfree(h->U0s);
  dfree(h->rest_box);
  h->cap_box = 0;
  dfree(h->Gs);
  dfree(h->res);
  dfree(h->slot_partial);
  h->cap_np = 0;
  h->m.max_slots = 0;
}

bool all_finite(const double *a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!isfinite(a[i])) return false;
  return true;
}
bool all_finite(const float *a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!isfinite(a[i])) return false;
  return true;
}

// The bounding box of each body's points (their rest positions when bodies
// rotate them, else their fixed positions): [nbox][6] = min x, y, z, max x,
// y, z, for the box strategy of the U0 pre-computation.
void rest_boxes(const double *X, const int *body, int64_t n, std::vector<double> &out) {
  int nbox = 0;
  for (int64_t k = 0; k < n; k++) nbox = std::max(nbox, (body ? body[k] : 0) + 1);
  out.assign(6 * (size_t)nbox, 0.0);
  for (int b = 0; b < nbox; b++)
    for (int a = 0; a < 3; a++) {
      out[6 * b + a] = HUGE_VAL;
      out[6 * b + 3 + a] = -HUGE_VAL;
    }
  for (int64_t k = 0; k < n; k++) {
    const int b = body ? body[k] : 0;
    for (int a = 0; a < 3; a++) {
      out[6 * b + a] = std::min(out[6 * b + a], X[3 * k + a]);
      out[6 * b + 3 + a] = std::max(out[6 * b + 3 + a], X[3 * k + a]);
    }
  }
  // a body index without points: an empty box at the origin
  for (int b = 0; b < nbox; b++)
    if (out[6 * b] > out[6 * b + 3])
      for (int a = 0; a < 6; a++) out[6 * b + a] = 0.0;
}

}  // namespace

extern "C" {

// (the steps prepared ahead; defined with the step below)
static int discard_ahead(lbm_t *h);
static BatchDims dims_of(const lbm_t *h);
static int launch_ahead_chain(lbm_t *h, const BatchDims &dims, const DomainDesc *Dn,
                              const double *Xsrc, const float *Usrc, long long t_step);

void lbm_default_opts(lbm_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->tau = 0.8;
  o->storage = LBM_STORE_F32;
  o->delta = LBM_DELTA_COSINE;
  o->warm_start = LBM_WARM_ZERO;
  o->ibm_tol = 1e-4;
  o->ibm_max_iter = 500;
  o->stats = 1;
}

const char *lbm_last_error(const lbm_t *h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

void lbm_velocity_set(int *e, double *t) {
  for (int i = 0; i < Q; i++) {
    if (e) {
      e[3 * i] = ex(i);
      e[3 * i + 1] = ey(i);
      e[3 * i + 2] = ez(i);
    }
    if (t) t[i] = wtd(i);
  }
}

void lbm_destroy(lbm_t *h) {
  if (!h) return;
  discard_ahead(h);
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  dfree(h->f[0]);
  dfree(h->f[1]);
  free_points(h);
  dfree(h->centre);
  dfree(h->omega);
  dfree(h->phase);
  dfree(h->m.brick_count);
  dfree(h->m.brick_slot);
  dfree(h->bslot_alt);
  dfree(h->m.counters);
  dfree(h->m.tiles);
  dfree(h->partial);
  dfree(h->sums);
  dfree(h->red_scratch);
  dfree(h->ticket);
  dfree(h->tmp);
  dfree(h->state);
  if (h->state_host) cudaFreeHost(h->state_host);
  dfree(h->desc);
  dfree(h->desc_alt);
  dfree(h->t_dev);
  dfree(h->Ufull);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ibm_st) cudaStreamDestroy(h->ibm_st);
  if (h->ibm_cap) cudaStreamDestroy(h->ibm_cap);
  if (h->ahead_st) cudaStreamDestroy(h->ahead_st);
  if (h->ev_ahead_go) cudaEventDestroy(h->ev_ahead_go);
  if (h->ev_ahead_done) cudaEventDestroy(h->ev_ahead_done);
  if (h->ev_collided) cudaEventDestroy(h->ev_collided);
  if (h->ev_finished) cudaEventDestroy(h->ev_finished);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  dfree(h->mlp_P);
  if (h->mlp_packed) cudaFree(h->mlp_packed);
  for (auto &p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->free_events) cudaEventDestroy(e);
  delete h;
}

int lbm_create_ex(const lbm_opts *o, lbm_t **out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!o) return fail(nullptr, LBM_EINVAL, "opts is NULL");
  if (o->nx <= 0 || o->ny <= 0 || o->nz <= 0 || o->nx % 4 || o->ny % 4 || o->nz % 4)
    return fail(nullptr, LBM_EINVAL, "dims %d x %d x %d must be positive multiples of 4",
                o->nx, o->ny, o->nz);
  const int64_t ncell = (int64_t)o->nx * o->ny * o->nz;
  if (ncell >= (1LL << 31))
    return fail(nullptr, LBM_EINVAL, "lattice of %lld cells is above 2^31",
                (long long)ncell);
  if (!(o->tau > 0.5) || !isfinite(o->tau))
    return fail(nullptr, LBM_EINVAL, "tau = %g must be > 1/2", o->tau);
  if (o->storage < 0 || o->storage > 2) return fail(nullptr, LBM_EINVAL, "bad storage");
  if (o->delta < 0 || o->delta > 1) return fail(nullptr, LBM_EINVAL, "bad delta kernel");
  if (o->warm_start < 0 || o->warm_start > 2) return fail(nullptr, LBM_EINVAL, "bad warm start");
  if (o->ibm_max_iter <= 0 || !(o->ibm_tol >= 0))
    return fail(nullptr, LBM_EINVAL, "bad ibm_tol/ibm_max_iter");
  lbm_t *h = new lbm();
  h->g.nx = o->nx;
  h->g.ny = o->ny;
  h->g.nz = o->nz;
  h->g.nbx = o->nx / 4;
  h->g.nby = o->ny / 4;
  h->g.nbz = o->nz / 4;
  h->g.ncell = ncell;
  h->g.nbrick = h->g.nbx * h->g.nby * h->g.nbz;
  geometry_divisors(h->g);
  h->tau = o->tau;
  h->storage = o->storage;
  h->delta = o->delta;
  h->warm = o->warm_start;
  h->tol = o->ibm_tol;
  h->max_iter = o->ibm_max_iter;
  h->stats_on = o->stats;
  const size_t pop = (size_t)Q * ncell * storage_bytes(h->storage);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    e = cudaMalloc(&h->f[k], pop);
    if (e == cudaSuccess) e = cudaMemset(h->f[k], 0, pop);  // deviations 0: rest
  }
  if (e == cudaSuccess) e = dalloc(&h->m.brick_count, h->g.nbrick);
  if (e == cudaSuccess) e = cudaMemset(h->m.brick_count, 0, sizeof(int) * h->g.nbrick);
  if (e == cudaSuccess) e = dalloc(&h->m.brick_slot, h->g.nbrick);
  if (e == cudaSuccess) e = cudaMemset(h->m.brick_slot, 0xff, sizeof(int) * h->g.nbrick);
  if (e == cudaSuccess) e = dalloc(&h->bslot_alt, h->g.nbrick);
  if (e == cudaSuccess) e = cudaMemset(h->bslot_alt, 0xff, sizeof(int) * h->g.nbrick);
  if (e == cudaSuccess) e = dalloc(&h->m.counters, BRICK_COUNTERS);
  if (e == cudaSuccess) e = cudaMemset(h->m.counters, 0, BRICK_COUNTERS * sizeof(int));
  {
    const size_t nt = (h->g.nbrick + COMPACT_TILE - 1) / COMPACT_TILE;
    if (e == cudaSuccess) e = dalloc(&h->m.tiles, nt);
    if (e == cudaSuccess) e = cudaMemset(h->m.tiles, 0, nt * sizeof(unsigned long long));
  }
  h->nparts = collide_partials(h->g);
  if (e == cudaSuccess) e = dalloc(&h->partial, (size_t)h->nparts * 4);
  if (e == cudaSuccess) e = dalloc(&h->sums, 4);
  if (e == cudaSuccess) e = dalloc(&h->red_scratch, 128 * 4);
  if (e == cudaSuccess) e = dalloc(&h->ticket, 1);
  if (e == cudaSuccess) e = cudaMemset(h->ticket, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = dalloc(&h->desc, 1);
  if (e == cudaSuccess) e = dalloc(&h->desc_alt, 1);
  if (e == cudaSuccess) e = dalloc(&h->t_dev, 2);
  if (e == cudaSuccess) e = cudaMemset(h->t_dev, 0, 2 * sizeof(int64_t));
  if (e == cudaSuccess) e = dalloc(&h->state, 1);
  if (e == cudaSuccess) e = cudaMemset(h->state, 0, sizeof(IbmState));
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->state_host, sizeof(IbmState));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    fail(nullptr, code, "allocation of a %d x %d x %d lattice: %s", o->nx, o->ny, o->nz,
         cudaGetErrorString(e));
    lbm_destroy(h);
    return code;
  }
  *out = h;
  return LBM_OK;
}

int lbm_create(int nx, int ny, int nz, double tau, lbm_t **out) {
  lbm_opts o;
  lbm_default_opts(&o);
  o.nx = nx;
  o.ny = ny;
  o.nz = nz;
  o.tau = tau;
  return lbm_create_ex(&o, out);
}

int lbm_set_stream(lbm_t *h, void *stream) {
  if (!h) return LBM_EINVAL;
  h->st = (cudaStream_t)stream;
  return LBM_OK;
}

int ibm_set_points(lbm_t *h, int64_t n, const double *X, const float *U_target,
                   const float *area, const int32_t *body) {
  if (!h) return LBM_EINVAL;
  if (n < 0) return fail(h, LBM_EINVAL, "n = %lld < 0", (long long)n);
  if (n > 0 && !X) return fail(h, LBM_EINVAL, "X is NULL");
  if (n > (1LL << 28)) return fail(h, LBM_EINVAL, "too many points");
  if (n > 0) {
    if (!all_finite(X, 3 * n)) return fail(h, LBM_ENONFINITE, "non-finite position");
    if (U_target && !all_finite(U_target, 3 * n))
      return fail(h, LBM_ENONFINITE, "non-finite target velocity");
    if (area && !all_finite(area, n)) return fail(h, LBM_ENONFINITE, "non-finite area");
  }
  int maxb = -1;
  if (body)
    for (int64_t k = 0; k < n; k++) {
      if (body[k] < 0) return fail(h, LBM_EINVAL, "negative body index at %lld", (long long)k);
      if (body[k] > maxb) maxb = body[k];
    }
  if (n > 0 && !body) maxb = 0;
  {
    const int ra = discard_ahead(h);  // (the prepared step's points are void)
    if (ra) return ra;
  }
  h->x_src = nullptr;  // (mapped uploads of the previous points are void)
  h->u_src = nullptr;
  if (h->nb > 0 && maxb >= h->nb)
    return fail(h, LBM_EINVAL, "body index %d out of range of %d bodies", maxb, h->nb);
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  if (n > h->cap_np) {
    free_points(h);
    const int64_t ms = std::min<int64_t>(h->g.nbrick, 8 * n);
    CK(h, dalloc(&h->X, 3 * n));
    CK(h, dalloc(&h->body, n));
    CK(h, dalloc(&h->area, n));
    CK(h, dalloc(&h->utarget, 3 * n));
    CK(h, dalloc(&h->pp.base, n));
    CK(h, dalloc(&h->pp.wts, 12 * n));
    CK(h, dalloc(&h->pp.ut, n));
    CK(h, dalloc(&h->du, n));
    CK(h, dalloc(&h->uint, n));
    CK(h, dalloc(&h->cg, 5 * n));
    CK(h, dalloc(&h->cg_part, 2 * ((n + 255) / 256)));
    CK(h, dalloc(&h->xpos, 3 * n));
    CK(h, dalloc(&h->xpos_alt, 3 * n));
    CK(h, dalloc(&h->m.slot_brick, ms));
    CK(h, dalloc(&h->m.order, (size_t)ORDER_BUCKETS * ms));
    CK(h, dalloc(&h->pm.count, ms));
    CK(h, dalloc(&h->pm.start, ms + 1));
    CK(h, dalloc(&h->pm.cursor, ms));
    CK(h, dalloc(&h->feat, (size_t)MLP_IN * n));
    CK(h, dalloc(&h->pm.k, 8 * n));
    CK(h, dalloc(&h->pm.brick, 8 * n));
    CK(h, dalloc(&h->pm.w, 3 * 8 * n));
    CK(h, dalloc(&h->pm.part, 8 * n));
    CK(h, dalloc(&h->pm.point_pairs, 8 * n));
    h->pm.max_pairs = 8 * n;
    CK(h, dalloc(&h->U0s, (size_t)ms * SLOT_FLOATS));
    // finite from the start: the kernel strategy of the U0 pre-computation
    // leaves the cells of an active brick outside every support as they were
    CK(h, cudaMemset(h->U0s, 0, sizeof(float) * ms * SLOT_FLOATS));
    CK(h, dalloc(&h->Gs, (size_t)ms * SLOT_FLOATS));
    CK(h, dalloc(&h->res, ms));
    CK(h, dalloc(&h->slot_partial, (size_t)ms * 4));
    h->cap_np = n;
    h->m.max_slots = (int)ms;
  }
  h->np = n;
  h->max_body = maxb;
  h->have_du = false;
  h->desc_dirty = true;
  if (body) h->body_host.assign(body, body + n);
  else h->body_host.clear();
  rest_boxes(X, body, n, h->box_host);
  h->box_dirty = true;
  if (n > 0) {
    CK(h, cudaMemcpy(h->X, X, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    std::vector<float> a(n, 1.0f);
    if (area) memcpy(a.data(), area, sizeof(float) * n);
    CK(h, cudaMemcpy(h->area, a.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    std::vector<int> b(n, 0);
    if (body) memcpy(b.data(), body, sizeof(int) * n);
    CK(h, cudaMemcpy(h->body, b.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    std::vector<float> u(3 * n, 0.0f);
    if (U_target) memcpy(u.data(), U_target, sizeof(float) * 3 * n);
    h->targets_nonzero = std::any_of(u.begin(), u.end(), [](float v) { return v != 0.0f; });
    CK(h, cudaMemcpy(h->utarget, u.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
    CK(h, cudaMemset(h->du, 0, sizeof(float4) * n));
    CK(h, cudaMemset(h->uint, 0, sizeof(float4) * n));
  } else {
    CK(h, cudaMemset(h->m.brick_slot, 0xff, sizeof(int) * h->g.nbrick));
    CK(h, cudaMemset(h->bslot_alt, 0xff, sizeof(int) * h->g.nbrick));
    CK(h, cudaMemset(h->m.counters, 0, 2 * sizeof(int)));
  }
  return LBM_OK;
}

int ibm_update_points(lbm_t *h, int64_t n, const double *X, const float *U_target) {
  if (!h) return LBM_EINVAL;
  if (n != h->np) return fail(h, LBM_EINVAL, "%lld points, the handle has %lld", (long long)n,
                              (long long)h->np);
  if (n == 0) return LBM_OK;
  if (!X) return fail(h, LBM_EINVAL, "X is NULL");
  if (h->pairs_ahead) {
    // a step prepared from earlier positions: these supersede them
    const int ra = discard_ahead(h);
    if (ra) return ra;
  }
  const void *mx = h->host_io == LBM_HOST_IO_MAPPED ? mapped_ptr(X) : nullptr;
  const void *mu = mx && U_target ? mapped_ptr(U_target) : nullptr;
  if (mx && (!U_target || mu) && h->loop_mark && !h->pairs_ahead) {
    // the last step's fixed point is marked (ev_ahead_go): the next step's
    // kinematics (reading these buffers) and pair lists start now, beside
    // that step's collide
    h->loop_mark = false;
    const float *us = mu ? (const float *)mu : h->u_src;
    if (U_target) h->targets_nonzero = false;
    h->x_src = nullptr;
    h->u_src = nullptr;
    if (h->u0_mode == LBM_U0_BOX) {
      rest_boxes(X, h->body_host.empty() ? nullptr : h->body_host.data(), n, h->box_host);
      h->box_dirty = true;
    }
    const int rc = launch_ahead_chain(h, dims_of(h), h->desc_alt, (const double *)mx, us,
                                      (long long)h->t);
    if (rc == LBM_OK) h->pairs_ahead = true;
    return rc;
  }
  if (mx && (!U_target || mu)) {
    // read by the next step's kinematics (an earlier mapped target without
    // a new one stays to be read)
    h->x_src = (const double *)mx;
    if (mu) h->u_src = (const float *)mu;
    if (U_target) h->targets_nonzero = false;
  } else {
    int r = flush_points(h, h->st);  // (earlier mapped uploads first)
    if (r) return r;
    CK(h, cudaMemcpyAsync(h->X, X, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->st));
    if (U_target) {
      CK(h, cudaMemcpyAsync(h->utarget, U_target, sizeof(float) * 3 * n,
                            cudaMemcpyHostToDevice, h->st));
      h->targets_nonzero = false;  // (not scanned here: checked on the device again)
    }
  }
  if (h->u0_mode == LBM_U0_BOX) {
    // the boxes of the moved points (bodies keep their indices)
    rest_boxes(X, h->body_host.empty() ? nullptr : h->body_host.data(), n, h->box_host);
    h->box_dirty = true;
  }
  return LBM_OK;
}

int ibm_set_bodies(lbm_t *h, int nb, const double *centre, const double *omega,
                   const double *phase) {
  if (!h) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (nb < 0) return fail(h, LBM_EINVAL, "nb = %d < 0", nb);
  if (nb > 0 && (!centre || !omega || !phase))
    return fail(h, LBM_EINVAL, "centre/omega/phase must be given");
  if (nb > 0 && (!all_finite(centre, 3 * nb) || !all_finite(omega, nb) ||
                 !all_finite(phase, nb)))
    return fail(h, LBM_ENONFINITE, "non-finite body parameter");
  if (nb > 0 && h->max_body >= nb)
    return fail(h, LBM_EINVAL, "points refer to body %d, only %d bodies", h->max_body, nb);
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  dfree(h->centre);
  dfree(h->omega);
  dfree(h->phase);
  h->nb = nb;
  h->bodies_moving = nb > 0 && std::any_of(omega, omega + nb, [](double w) { return w != 0.0; });
  h->desc_dirty = true;
  if (nb > 0) {
    CK(h, dalloc(&h->centre, 3 * nb));
    CK(h, dalloc(&h->omega, nb));
    CK(h, dalloc(&h->phase, nb));
    CK(h, cudaMemcpy(h->centre, centre, sizeof(double) * 3 * nb, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->omega, omega, sizeof(double) * nb, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->phase, phase, sizeof(double) * nb, cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

int lbm_set_body_force(lbm_t *h, double gx, double gy, double gz) {
  if (!h) return LBM_EINVAL;
  if (!isfinite(gx) || !isfinite(gy) || !isfinite(gz))
    return fail(h, LBM_ENONFINITE, "non-finite body force");
  h->gbody[0] = gx;
  h->gbody[1] = gy;
  h->gbody[2] = gz;
  h->desc_dirty = true;
  return LBM_OK;
}

int64_t lbm_time(const lbm_t *h) { return h ? h->t : -1; }
int lbm_set_time(lbm_t *h, int64_t t) {
  if (!h) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  CK(h, cudaMemcpy(h->t_dev, &t, sizeof t, cudaMemcpyHostToDevice));
  h->t = t;
  return LBM_OK;
}

// ---- one time step --------------------------------------------------------

// The descriptor of h (pointers of its arrays and per-domain parameters).
static DomainDesc host_desc(const lbm_t *h) {
  DomainDesc d{};
  d.g = h->g;
  d.delta = h->delta;
  d.np = (int)h->np;
  d.tau = (float)h->tau;
  d.om = 1.0f / d.tau;
  for (int c = 0; c < 3; c++) d.gbody[c] = (float)h->gbody[c];
  d.f[0] = h->f[0];
  d.f[1] = h->f[1];
  d.t = h->t_dev;
  d.X = h->X;
  d.body = h->body;
  d.area = h->area;
  d.utarget = h->utarget;
  d.centre = h->centre;
  d.omega = h->omega;
  d.phase = h->phase;
  d.nb = h->nb;
  d.cblocks = h->nparts;
  d.pp = h->pp;
  d.m = h->m;
  d.pm = h->pm;
  d.U0s = h->U0s;
  d.Gs = h->Gs;
  d.res = h->res;
  d.du = h->du;
  d.uint = h->uint;
  d.cg = h->cg;
  d.cg_part = h->cg_part;
  d.xpos = h->xpos;
  d.partial = h->partial;
  d.sums = h->sums;
  d.slot_partial = h->slot_partial;
  d.red_scratch = h->red_scratch;
  d.ticket = h->ticket;
  d.state = h->state;
  d.feat = h->feat;
  d.mlp_packed = h->mlp_packed;
  d.u0_mode = h->u0_mode;
  d.nbox = h->nbox;
  d.rest_box = h->rest_box;
  d.Ufull = h->Ufull;
  return d;
}

static int sync_desc(lbm_t *h) {
  if (!h->desc_dirty) return LBM_OK;
  const DomainDesc d = host_desc(h);
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  CK(h, cudaMemcpy(h->desc, &d, sizeof d, cudaMemcpyHostToDevice));
  h->desc_host = d;
  DomainDesc da = d;
  da.m.brick_slot = h->bslot_alt;
  da.xpos = h->xpos_alt;
  CK(h, cudaMemcpy(h->desc_alt, &da, sizeof da, cudaMemcpyHostToDevice));
  h->desc_host_alt = da;
  h->desc_dirty = false;
  h->version++;
  return LBM_OK;
}

static BatchDims dims_of(const lbm_t *h) {
  BatchDims b{};
  b.nd = 1;
  b.max_cells = h->g.ncell;
  b.max_points = (int)h->np;
  b.max_bodies = h->nb;
  b.max_bricks = h->g.nbrick;
  b.max_slots = h->np > 0 ? h->m.max_slots : 0;
  b.ls = h->shape;
  return b;
}

// What one step launches, for one lattice or a batch (uniform host-side
// decisions; per-domain differences live in the descriptors).  With split,
// the cells outside the step's active bricks collide on st while the IBM
// stages and then the active bricks' collide run on sti; the two meet
// before the end of the step.  Without split, sti == st and one collide
// launch does every cell after the IBM loop.
struct StepCtx {
  lbm_t *acct;          // launch counting, timing, errors
  const DomainDesc *D;  // device descriptors
  const DomainDesc *Dhost;  // host copy for a single lattice, else NULL
  BatchDims dims;
  int storage, stats, cur;
  int warm_mode;
  int solver;  // LBM_SOLVER_*
  int u0_mode, nbox;  // U0 pre-computation (single lattice; a batch: bricks)
  bool have_du, features;
  cudaStream_t st, sti;
  bool split;
  cudaEvent_t ev_fork, ev_join;
  const double *x_src;  // mapped uploads for this step's kinematics, or NULL
  const float *u_src;
  bool pairs_done;  // kinematics and pair lists were built ahead (ahead_st)
  bool ahead;       // build the next step's after this step's fixed point
  bool mark_loop;   // else record ev_ahead_go there (see lbm_t::loop_mark)
  const DomainDesc *D_next;  // the prepared step's descriptors (NULL: desc_alt)
  bool defer_finish;         // the end-of-step sums on ahead_st (lbm_t::finish_pending)
  long long t_next; // the next step's index (its kinematics)
};

// Kinematics and slots on st; with split, the fork to sti and the collide of
// the cells outside the active bricks on st.
static int enqueue_head(StepCtx &c) {
  lbm_t *h = c.acct;
  if (c.pairs_done) return LBM_OK;  // (never split)
  {
    StageTimer T(h, ST_KIN, c.st, 1);
    CK(h, launch_prepare_points(c.D, c.dims, c.st, c.x_src, c.u_src));
  }
  {
    StageTimer T(h, ST_PAIRS, c.st, c.dims.work_off ? 2 : 1);
    CK(h, launch_compact(c.D, c.dims, c.st));
    CK(h, launch_batch_worklist(c.D, c.dims, c.st));
  }
  if (c.split) {
    CK(h, cudaEventRecord(c.ev_fork, c.st));
    CK(h, cudaStreamWaitEvent(c.sti, c.ev_fork, 0));
    StageTimer T(h, ST_COLLIDE, c.st);
    CK(h, launch_collide_stream(c.storage, c.D, c.Dhost, c.dims, c.cur, c.stats, 1, c.st));
  }
  return LBM_OK;
}

// Pairs, moments, learned start / features, and the first brick pass, on
// sti.  Returns the warm flag of the fixed point.
static int enqueue_prefix(StepCtx &c, bool *warm_out) {
  lbm_t *h = c.acct;
  const bool mlp = c.warm_mode == LBM_WARM_MLP;
  const bool feat = mlp || c.features;
  const bool warm = (c.warm_mode == LBM_WARM_PREVIOUS && c.have_du) || mlp;
  *warm_out = warm;
  const cudaStream_t s = c.sti;
  if (!c.pairs_done) {
    StageTimer T(h, ST_PAIRS, s, 2);
    CK(h, launch_pair_lists(c.D, c.dims, s));
  }
  if (c.u0_mode == LBM_U0_BOX) {
    // the paper's box strategy (Sec. 5): U on each body's moved bounding
    // box, then the active bricks' cells from it
    StageTimer T(h, ST_INIT, s, 2);
    CK(h, launch_box_moments(c.storage, c.D, c.nbox, c.cur, s));
  } else if (c.u0_mode == LBM_U0_KERNEL) {
    // the paper's kernel strategy (Sec. 5): U on every point's support
    StageTimer T(h, ST_INIT, s, 1);
    CK(h, launch_point_moments(c.storage, c.D, c.dims.max_points, c.cur, s));
  } else {
    StageTimer T(h, ST_INIT, s, 1);
    CK(h, launch_brick_moments(c.storage, c.D, c.dims, c.cur, s));
  }
  if (feat) {
    // features from the shares of I[U0 + S[du_prev]] (the previous step's
    // force applied); the learned start du = du_prev + V MLP(x)
    StageTimer T(h, ST_MLP, s, mlp ? 3 : 2);
    CK(h, launch_brick_init(c.D, c.dims, c.have_du, s));
    CK(h, launch_mlp_features(c.D, c.dims, c.have_du, s));
    if (mlp) CK(h, launch_mlp_warm(c.D, c.dims, c.have_du, s));
  }
  // G_0 = S[du_init] and the shares of I[U0 + G_0], unless the feature pass
  // above already left exactly these
  const bool init_done = feat && !mlp && (warm == c.have_du);
  if (!init_done) {
    StageTimer T(h, ST_INIT, s, 1);
    CK(h, launch_brick_init(c.D, c.dims, warm, s));
  }
  return LBM_OK;
}

// Conjugate gradients on the lattice form of the fixed point, n_iter
// iterations (or, tol_mode, until the device-side stop): r_0 from the shares
// of brick_init, then per iteration the gather of S[v] with its pair shares,
// the dot products and the updates; G = S[du] after the last.
static int enqueue_cg_start(StepCtx &c, bool warm, cudaStream_t s) {
  lbm_t *h = c.acct;
  StageTimer T(h, ST_UPDATE, s);
  CK(h, launch_cg_start(c.D, c.dims, warm, s));
  return LBM_OK;
}

// confirm: r is the true residual, and an iterate that meets tol is kept
// without this iteration's update
static int enqueue_cg_iteration(StepCtx &c, int it, int tol_mode, cudaStream_t s,
                                bool confirm = false) {
  lbm_t *h = c.acct;
  {
    StageTimer T(h, ST_SPREAD, s);
    CK(h, launch_cg_brick(c.D, c.dims, tol_mode, s));
  }
  {
    StageTimer T(h, ST_UPDATE, s, 2);
    CK(h, launch_cg_dot(c.D, c.dims, tol_mode, s));
    CK(h, launch_cg_update(c.D, c.dims, it, h->tol, h->max_iter, tol_mode, confirm, s));
  }
  return LBM_OK;
}

static int enqueue_final_spread(StepCtx &c, cudaStream_t s) {
  lbm_t *h = c.acct;
  StageTimer T(h, ST_SPREAD, s);
  CK(h, launch_brick_spread(c.D, c.dims, 0, 0, s));
  return LBM_OK;
}

static int enqueue_fixed_loop(StepCtx &c, int n_iter, bool warm) {
  lbm_t *h = c.acct;
  if (c.solver == LBM_SOLVER_CG) {
    int r = enqueue_cg_start(c, warm, c.sti);
    for (int it = 0; r == LBM_OK && it < n_iter; it++) r = enqueue_cg_iteration(c, it, 0, c.sti);
    return r ? r : enqueue_final_spread(c, c.sti);
  }
  for (int it = 0; it < n_iter; it++) {
    {
      StageTimer T(h, ST_UPDATE, c.sti);
      CK(h, launch_point_update(c.D, c.dims, it == 0, warm, 0, c.sti));
    }
    {
      StageTimer T(h, ST_SPREAD, c.sti);
      CK(h, launch_brick_spread(c.D, c.dims, it + 1 < n_iter, 0, c.sti));
    }
  }
  return LBM_OK;
}

// The next step's kinematics and pair lists on ahead_st (a stream of the
// greatest priority), once this step's fixed point is done with its own:
// they need no populations, so they run while this step collides (an
// HBM-bound pass that leaves SM slots and L2 to them).  They write the other
// brick map, through desc_alt, and finish before the next step's first
// kernel on st (ev_ahead_done).
static int ensure_ahead(lbm_t *h) {
  if (!h->ahead_st) {
    int lo = 0, hi = 0;
    CK(h, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(h, cudaStreamCreateWithPriority(&h->ahead_st, cudaStreamNonBlocking, hi));
  }
  if (!h->ev_ahead_go) CK(h, cudaEventCreateWithFlags(&h->ev_ahead_go, cudaEventDisableTiming));
  if (!h->ev_ahead_done)
    CK(h, cudaEventCreateWithFlags(&h->ev_ahead_done, cudaEventDisableTiming));
  if (!h->ev_collided) CK(h, cudaEventCreateWithFlags(&h->ev_collided, cudaEventDisableTiming));
  if (!h->ev_finished) CK(h, cudaEventCreateWithFlags(&h->ev_finished, cudaEventDisableTiming));
  return LBM_OK;
}

// The chain of step t_step on ahead_st after ev_ahead_go, into the other
// brick map (desc_alt); Xsrc / Usrc: mapped uploads it reads (else the
// device copies).
static int launch_ahead_chain(lbm_t *h, const BatchDims &dims, const DomainDesc *Dn,
                              const double *Xsrc, const float *Usrc, long long t_step) {
  CK(h, cudaStreamWaitEvent(h->ahead_st, h->ev_ahead_go, 0));
  BatchDims da = dims;
  da.ls.sort_blocks = da.ls.sort_blocks_ahead;
  {
    StageTimer T(h, ST_KIN, h->ahead_st, 1);
    CK(h, launch_prepare_points(Dn, dims, h->ahead_st, Xsrc, Usrc, t_step));
  }
  {
    StageTimer T(h, ST_PAIRS, h->ahead_st, dims.work_off ? 4 : 3);
    CK(h, launch_compact(Dn, dims, h->ahead_st));
    CK(h, launch_batch_worklist(Dn, dims, h->ahead_st));
    CK(h, launch_pair_lists(Dn, da, h->ahead_st));
  }
  CK(h, cudaEventRecord(h->ev_ahead_done, h->ahead_st));
  return LBM_OK;
}

// After this step's fixed point: the next step's chain (c.ahead), or only the
// mark of the fixed point's end for an upload to start it (c.mark_loop).
static int enqueue_ahead(StepCtx &c) {
  lbm_t *h = c.acct;
  if (!c.ahead && !c.mark_loop) return LBM_OK;
  int r = ensure_ahead(h);
  if (r) return r;
  CK(h, cudaEventRecord(h->ev_ahead_go, c.st));
  if (!c.ahead) return LBM_OK;
  r = launch_ahead_chain(h, c.dims, c.D_next ? c.D_next : h->desc_alt, nullptr, nullptr,
                         c.t_next);
  if (r) return r;
  if (!c.D_next) h->pairs_ahead = true;  // (inside a capture the graph joins it)
  return LBM_OK;
}

// The collide of the cells with the IBM force (split: the active bricks on
// sti, then the join), and the end of the step on st.
static int enqueue_suffix(StepCtx &c) {
  lbm_t *h = c.acct;
  if (c.split) {
    {
      StageTimer T(h, ST_COLLIDE_ACTIVE, c.sti);
      CK(h, launch_collide_active(c.storage, c.D, c.dims, c.cur, c.stats, c.sti));
    }
    CK(h, cudaEventRecord(c.ev_join, c.sti));
    CK(h, cudaStreamWaitEvent(c.st, c.ev_join, 0));
  } else {
    if (h->finish_pending && !c.D_next) {
      // the previous step's sums (on ahead_st) have read its partials
      CK(h, cudaStreamWaitEvent(c.st, h->ev_finished, 0));
      h->finish_pending = false;
    }
    StageTimer T(h, ST_COLLIDE, c.st);
    CK(h, launch_collide_stream(c.storage, c.D, c.Dhost, c.dims, c.cur, c.stats, 0, c.st));
  }
  if (c.defer_finish) {
    // (the next step of the call waits for these sums before its collide)
    CK(h, cudaEventRecord(h->ev_collided, c.st));
    CK(h, cudaStreamWaitEvent(h->ahead_st, h->ev_collided, 0));
    StageTimer T(h, ST_STATS, h->ahead_st);
    CK(h, launch_finish_step(c.D, c.dims, c.stats, c.split, h->ahead_st));
    CK(h, cudaEventRecord(h->ev_finished, h->ahead_st));
    h->finish_pending = true;
    return LBM_OK;
  }
  {
    StageTimer T(h, ST_STATS, c.st);
    CK(h, launch_finish_step(c.D, c.dims, c.stats, c.split, c.st));
  }
  return LBM_OK;
}

// One full step with a fixed iteration count (n_iter > 0, or no points).
static int enqueue_step(StepCtx &c, int n_iter) {
  if (c.dims.max_points > 0) {
    int r = enqueue_head(c);
    if (r) return r;
    bool warm = false;
    r = enqueue_prefix(c, &warm);
    if (r) return r;
    r = enqueue_fixed_loop(c, n_iter, warm);
    if (r) return r;
    r = enqueue_ahead(c);
    if (r) return r;
  }
  return enqueue_suffix(c);
}

// The tolerance-driven fixed point of Sec. 3 for one lattice: iterations
// until eps <= ibm_tol or ibm_max_iter, the stop decided on the device and
// read by the host after each chunk of iterations (sized from the previous
// step's count).  Returns LBM_WNOTCONVERGED when the cap was hit.
static int tolerance_loop(StepCtx &c, bool warm) {
  lbm_t *h = c.acct;
  cudaStream_t st = c.sti;
  // where the surface velocities are known not to vanish, the denominator
  // needs no check by the host (and no round trip before the iterations)
  const bool moving = h->nb > 0 ? h->bodies_moving : h->targets_nonzero;
  {
    // denominator ||S[s u_k]||^2
    StageTimer T(h, ST_RESID, st, 2);
    CK(h, launch_brick_norm(c.D, c.dims, 0, st));
    CK(h, launch_ibm_den(c.D, c.dims, moving ? 2 : 0, st));
  }
  if (!moving) {
    CK(h, cudaMemcpyAsync(h->state_host, h->state, 64, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
  }
  if (!moving && h->state_host->den2 == 0.0) {
    // all surface velocities vanish: ||S[s (u_k - I[U0])]||^2 instead
    StageTimer T(h, ST_RESID, st, warm ? 5 : 3);
    if (warm) CK(h, launch_brick_init(c.D, c.dims, 0, st));
    CK(h, launch_point_residual0(c.D, c.dims, st));
    CK(h, launch_brick_norm(c.D, c.dims, 1, st));
    CK(h, launch_ibm_den(c.D, c.dims, 1, st));
    if (warm) CK(h, launch_brick_init(c.D, c.dims, 1, st));
  }
  const bool cg = c.solver == LBM_SOLVER_CG;
  bool g_current = false;  // (CG) G = S[du] already holds for the result
  if (cg) {
    int r = enqueue_cg_start(c, warm, st);
    if (r) return r;
  }
  int it = 0;
  // chunks of half the iterations the previous step still had to go at this
  // point (at least kCheckChunk): few reads of the stop flag, and few
  // launches past convergence (their kernels return at once, but are not free)
  // (CG, which converges in a few dozen iterations: chunks of the previous
  // step's remaining count, then of kCgChunk)
  while (it < h->max_iter) {
    const int left = h->tol_hint - it;
    const int want = cg ? (left > 0 ? left : kCgChunk)
                        : (left > 0 ? std::max(kCheckChunk, left / 2) : kCheckChunk);
    const int chunk = std::min(want, h->max_iter - it);
    for (int j = 0; j < chunk; j++, it++) {
      if (cg) {
        int r = enqueue_cg_iteration(c, it, 1, st);
        if (r) return r;
        continue;
      }
      {
        StageTimer T(h, ST_UPDATE, st);
        CK(h, launch_point_update(c.D, c.dims, it == 0, warm, 1, st));
      }
      {
        StageTimer T(h, ST_SPREAD, st);
        CK(h, launch_brick_spread(c.D, c.dims, 1, 1, st));
      }
      {
        StageTimer T(h, ST_RESID, st);
        CK(h, launch_ibm_check(c.D, c.dims, it, h->tol, h->max_iter, st));
      }
    }
    CK(h, cudaMemcpyAsync(h->state_host, h->state, 64, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (!h->state_host->done) continue;
    // CG: confirm the stop on the true residual (the recursion drifts from
    // it by amplified FP32 rounding): replace r by u_k - I[U0 + S[du]] and run
    // one more iteration, whose check then decides (and, if it passes, keeps
    // the checked iterate); if it fails, iterate on
    it = h->state_host->iters;
    if (!cg || h->state_host->capped || it >= h->max_iter) break;
    {
      StageTimer T(h, ST_SPREAD, st);
      CK(h, launch_brick_spread(c.D, c.dims, 1, 0, st));
    }
    {
      StageTimer T(h, ST_UPDATE, st);
      CK(h, launch_cg_replace(c.D, c.dims, st));
    }
    int r = enqueue_cg_iteration(c, it++, 1, st, true);
    if (r) return r;
    CK(h, cudaMemcpyAsync(h->state_host, h->state, 64, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    // a confirmed stop keeps the iterate whose G = S[du] the pass above left
    g_current = h->state_host->done && !h->state_host->capped;
    if (h->state_host->done) break;
  }
  if (cg && !g_current) {
    int r = enqueue_final_spread(c, st);
    if (r) return r;
  }
  h->last_iters = h->state_host->iters;
  h->tol_hint = h->last_iters;
  h->last_eps = h->state_host->last_eps;
  if (h->state_host->capped) {
    h->not_converged++;
    return LBM_WNOTCONVERGED;
  }
  return LBM_OK;
}

static StepCtx ctx_of(lbm_t *h, cudaStream_t st) {
  StepCtx c{};
  c.acct = h;
  c.D = h->desc;
  c.Dhost = &h->desc_host;
  c.dims = dims_of(h);
  c.storage = h->storage;
  c.stats = h->stats_on;
  c.cur = h->cur;
  c.warm_mode = h->warm;
  c.solver = h->solver;
  c.u0_mode = h->u0_mode;
  c.nbox = h->nbox;
  c.have_du = h->have_du;
  c.features = h->features_on;
  c.st = st;
  c.sti = st;
  c.split = false;
  return c;
}

// The IBM stream (greatest priority) and the fork/join events of a handle;
// capture: the stream used inside graph captures.  Sets c.sti and c.split
// when the step runs split.
static int ensure_split(lbm_t *h, StepCtx &c, bool capture) {
  if (!h->overlap || c.dims.max_points <= 0) return LBM_OK;
  cudaStream_t *ps = capture ? &h->ibm_cap : &h->ibm_st;
  if (!*ps) {
    int lo = 0, hi = 0;
    CK(h, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(h, cudaStreamCreateWithPriority(ps, cudaStreamNonBlocking, hi));
  }
  if (!h->ev_fork) CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  c.sti = *ps;
  c.split = true;
  c.ev_fork = h->ev_fork;
  c.ev_join = h->ev_join;
  return LBM_OK;
}

// host-side bookkeeping after a step was enqueued
static void after_step(lbm_t *h, int n_iter) {
  if (h->np > 0) {
    h->have_du = true;
    if (n_iter > 0) {
      h->last_iters = n_iter;
      h->last_eps = -1.0;
    }
  } else {
    h->last_iters = 0;
    h->last_eps = -1.0;
  }
  if (h->stats_on) h->sums_valid = true;
  h->cur ^= 1;
  h->t++;
}

// The prepared step (kinematics and pair lists built ahead) becomes the
// current one: the handle's stream waits for its chain, and its descriptor,
// brick map and positions become the handle's.  No-op when there is none.
static int take_ahead(lbm_t *h, bool *taken) {
  *taken = h->pairs_ahead;
  if (!h->pairs_ahead) return LBM_OK;
  h->pairs_ahead = false;
  CK(h, cudaStreamWaitEvent(h->st, h->ev_ahead_done, 0));
  std::swap(h->desc, h->desc_alt);
  std::swap(h->desc_host, h->desc_host_alt);
  std::swap(h->m.brick_slot, h->bslot_alt);
  std::swap(h->xpos, h->xpos_alt);
  h->version++;  // (a captured step holds the other descriptor)
  return LBM_OK;
}

// A prepared step that will not be taken (the points, bodies, time or
// transfer mode change, or the next steps are replayed or batched): the
// handle's stream waits for its chain, whose writes stay in the other brick
// map; its write-through of mapped uploads into the device copies stands.
static int discard_ahead(lbm_t *h) {
  h->loop_mark = false;
  if (h->finish_pending) {
    h->finish_pending = false;
    CK(h, cudaStreamWaitEvent(h->st, h->ev_finished, 0));
  }
  if (!h->pairs_ahead) return LBM_OK;
  h->pairs_ahead = false;
  CK(h, cudaStreamWaitEvent(h->st, h->ev_ahead_done, 0));
  return LBM_OK;
}

// ahead: also prepare the next step (its kinematics and pair lists) while this
// one collides; the caller makes the next step the next call of step_once.
static int step_once(lbm_t *h, int n_iter, bool ahead = false) {
  bool pre = false;
  int rj = take_ahead(h, &pre);
  if (rj) return rj;
  h->loop_mark = false;
  StepCtx c = ctx_of(h, h->st);
  c.pairs_done = pre;
  const bool can = h->np > 0 && !h->overlap && !h->timing;
  c.ahead = ahead && can;
  // (the box pre-computation reads the step counter the sums advance)
  c.defer_finish = c.ahead && h->u0_mode != LBM_U0_BOX;
  // a one-step call in mapped transfer mode marks its fixed point's end, for
  // the next upload of moved points (ibm_update_points) to start the next step
  c.mark_loop = !c.ahead && can && h->host_io == LBM_HOST_IO_MAPPED && !h->graph_on;
  c.t_next = (long long)h->t + 1;
  if (h->np > 0) {
    // the kinematics read the mapped uploads themselves
    c.x_src = h->x_src;
    c.u_src = h->u_src;
    h->x_src = nullptr;
    h->u_src = nullptr;
  }
  int r0 = ensure_split(h, c, false);
  if (r0) return r0;
  int warn = LBM_OK;
  if (h->np > 0 && n_iter == 0) {
    int r = enqueue_head(c);
    if (r) return r;
    bool warm = false;
    r = enqueue_prefix(c, &warm);
    if (r) return r;
    warn = tolerance_loop(c, warm);
    if (warn < 0) return warn;
    r = enqueue_ahead(c);
    if (r) return r;
    r = enqueue_suffix(c);
    if (r) return r;
  } else {
    int r = enqueue_step(c, n_iter);
    if (r) return r;
  }
  h->loop_mark = c.mark_loop;
  after_step(h, n_iter);
  return warn;
}

// ---- captured steps ------------------------------------------------------------
//
// Two consecutive steps (the lattices swap each step, so two steps bring the
// pointers back) are captured once into a CUDA graph and replayed; the step
// counter and every other changing quantity live on the device.  Captured on a
// private stream ordered after and before the handle's stream with events.

struct GraphSlot {
  cudaStream_t *cap_stream;
  cudaEvent_t *ev_in, *ev_out;
  cudaGraphExec_t *exec;
};

static int ensure_capture_stream(lbm_t *acct, cudaStream_t *cs, cudaEvent_t *a, cudaEvent_t *b) {
  if (!*cs) CK(acct, cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking));
  if (!*a) CK(acct, cudaEventCreateWithFlags(a, cudaEventDisableTiming));
  if (!*b) CK(acct, cudaEventCreateWithFlags(b, cudaEventDisableTiming));
  return LBM_OK;
}

// Captures two steps of `c` (c.st is replaced by the capture stream) into
// *exec; *launches receives the kernels per replay.
// D_alt (Dhost_alt for a single lattice): the descriptors of the same
// lattices with their other brick maps, or NULL.  With them the first step of
// the pair runs on them and the second step's kinematics and pair lists are
// built beside the first one's collide, on the primary descriptors (which the
// second step then uses, so that after a replay the primary brick maps are
// the current ones); the prepared step's index comes from the device (the one
// the first step's kinematics used, plus one).
static int capture_two_steps(StepCtx c, int n_iter, cudaStream_t cs, cudaGraphExec_t *exec,
                             int64_t *launches, const DomainDesc *D_alt = nullptr,
                             const DomainDesc *Dhost_alt = nullptr) {
  lbm_t *h = c.acct;
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  const int saved_timing = h->timing;
  const int64_t l0 = h->nlaunch;
  h->timing = 0;
  c.st = cs;
  c.sti = cs;
  c.split = false;
  int r0 = ensure_split(h, c, true);
  if (r0) return r0;
  const bool ahead = D_alt && !c.split && c.dims.max_points > 0;
  if (ahead) {
    r0 = ensure_ahead(h);
    if (r0) return r0;
  }
  CK(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int r = LBM_OK;
  if (ahead) {
    StepCtx a = c;
    a.D = D_alt;
    a.Dhost = Dhost_alt;
    a.ahead = true;
    a.D_next = c.D;
    a.t_next = -2;
    a.defer_finish = h->u0_mode != LBM_U0_BOX;  // (joined before the second collide)
    r = enqueue_step(a, n_iter);
    if (r == LBM_OK && cudaStreamWaitEvent(cs, h->ev_ahead_done, 0) != cudaSuccess)
      r = fail(h, LBM_ECUDA, "stream capture: joining the prepared step");
    if (r == LBM_OK) {
      c.cur ^= 1;
      c.have_du = true;
      c.pairs_done = true;
      r = enqueue_step(c, n_iter);
    }
  } else {
    r = enqueue_step(c, n_iter);
    if (r == LBM_OK) {
      c.cur ^= 1;
      c.have_du = c.have_du || c.dims.max_points > 0;
      r = enqueue_step(c, n_iter);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  h->timing = saved_timing;
  *launches = h->nlaunch - l0;
  h->nlaunch = l0;
  if (r != LBM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return fail(h, LBM_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
  return LBM_OK;
}

static int replay(lbm_t *acct, cudaStream_t user, cudaStream_t cs, cudaEvent_t a, cudaEvent_t b,
                  cudaGraphExec_t exec) {
  CK(acct, cudaEventRecord(a, user));
  CK(acct, cudaStreamWaitEvent(cs, a, 0));
  CK(acct, cudaGraphLaunch(exec, cs));
  CK(acct, cudaEventRecord(b, cs));
  CK(acct, cudaStreamWaitEvent(user, b, 0));
  return LBM_OK;
}

int lbm_step(lbm_t *h, int n_steps, int n_ibm_iter) {
  if (!h) return LBM_EINVAL;
  if (n_steps < 0 || n_ibm_iter < 0)
    return fail(h, LBM_EINVAL, "n_steps = %d, n_ibm_iter = %d", n_steps, n_ibm_iter);
  if (h->nb > 0 && h->max_body >= h->nb)
    return fail(h, LBM_EINVAL, "points refer to body %d, only %d bodies", h->max_body, h->nb);
  if (h->warm == LBM_WARM_MLP && !h->mlp_packed && h->np > 0)
    return fail(h, LBM_EINVAL, "learned warm start without weights (mlp_set_weights)");
  if (h->u0_mode == LBM_U0_BOX && h->box_dirty) {
    const int nbox = (int)(h->box_host.size() / 6);
    if (nbox > h->cap_box) {
      CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
      dfree(h->rest_box);
      CK(h, dalloc(&h->rest_box, 6 * (size_t)nbox));
      h->cap_box = nbox;
      h->desc_dirty = true;
    }
    if (nbox != h->nbox) h->desc_dirty = true;
    h->nbox = nbox;
    if (nbox > 0)
      CK(h, cudaMemcpyAsync(h->rest_box, h->box_host.data(), sizeof(double) * 6 * nbox,
                            cudaMemcpyHostToDevice, h->st));
    h->box_dirty = false;
  }
  int r = sync_desc(h);
  if (r) return r;
  int warn = LBM_OK;
  int s = 0;
  const bool graphable = h->graph_on && (n_ibm_iter > 0 || h->np == 0);
  // mapped uploads are read by the next eager step's kinematics; a replayed
  // step gets them copied first
  if (graphable && (h->have_du || h->np == 0) && n_steps >= 2) {
    r = flush_points(h, h->st);
    if (r) return r;
  }
  while (s < n_steps) {
    // replay captured pairs of steps once the host-side decisions are steady
    const bool steady = h->have_du || h->np == 0;
    if (graphable && steady && n_steps - s >= 2) {
      if (!h->gexec || h->g_iters != n_ibm_iter || h->g_cur != h->cur ||
          h->g_version != h->version) {
        r = ensure_capture_stream(h, &h->cap_stream, &h->ev_in, &h->ev_out);
        if (r) return r;
        r = capture_two_steps(ctx_of(h, h->st), n_ibm_iter, h->cap_stream, &h->gexec,
                              &h->g_launches, h->timing ? nullptr : h->desc_alt,
                              &h->desc_host_alt);
        if (r) return r;
        h->g_iters = n_ibm_iter;
        h->g_cur = h->cur;
        h->g_version = h->version;
      }
      r = discard_ahead(h);
      if (r) return r;
      r = replay(h, h->st, h->cap_stream, h->ev_in, h->ev_out, h->gexec);
      if (r) return r;
      h->nlaunch += h->g_launches;
      after_step(h, n_ibm_iter);
      after_step(h, n_ibm_iter);
      s += 2;
      continue;
    }
    // the next step of this call prepared while this one collides (eager
    // steps without stage timing; never past the call, so that every read-out
    // and every other entry point sees the last step's state)
    const bool ahead = !graphable && !h->timing && s + 1 < n_steps;
    r = step_once(h, n_ibm_iter, ahead);
    if (r < 0) {
      discard_ahead(h);
      return r;
    }
    if (r == LBM_WNOTCONVERGED) warn = r;
    s++;
  }
  return warn;
}

int lbm_set_graph(lbm_t *h, int on) {
  if (!h) return LBM_EINVAL;
  h->graph_on = on != 0;
  return LBM_OK;
}

int lbm_set_overlap(lbm_t *h, int on) {
  if (!h) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (h->overlap != (on != 0)) {
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->ibm_st) cudaStreamSynchronize(h->ibm_st);
    h->overlap = on != 0;
    h->version++;  // a new capture
  }
  return LBM_OK;
}

int ibm_set_solver(lbm_t *h, int solver) {
  if (!h) return LBM_EINVAL;
  if (solver != LBM_SOLVER_MDF && solver != LBM_SOLVER_CG)
    return fail(h, LBM_EINVAL, "unknown solver %d", solver);
  if (h->solver != solver) {
    if (h->st) cudaStreamSynchronize(h->st);
    h->solver = solver;
    h->version++;  // a new capture
  }
  return LBM_OK;
}

int ibm_get_solver(const lbm_t *h) { return h ? h->solver : -1; }

int lbm_set_u0_strategy(lbm_t *h, int strategy) {
  if (!h) return LBM_EINVAL;
  if (strategy != LBM_U0_BRICKS && strategy != LBM_U0_BOX && strategy != LBM_U0_KERNEL)
    return fail(h, LBM_EINVAL, "unknown U0 strategy %d", strategy);
  if (h->u0_mode == strategy) return LBM_OK;
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  if (strategy == LBM_U0_BOX && !h->Ufull) {
    cudaError_t e = dalloc(&h->Ufull, 3 * (size_t)h->g.ncell);
    if (e != cudaSuccess) {
      h->Ufull = nullptr;
      return fail(h, LBM_ENOMEM, "full-lattice U of the box strategy: %s", cudaGetErrorString(e));
    }
    h->box_dirty = true;
  }
  h->u0_mode = strategy;
  h->desc_dirty = true;  // (a new capture)
  return LBM_OK;
}

int lbm_get_u0_strategy(const lbm_t *h) { return h ? h->u0_mode : -1; }

// ---- batches ----------------------------------------------------------------------

struct lbm_batch {
  std::vector<lbm_t *> hs;
  DomainDesc *D = nullptr;
  DomainDesc *D_alt = nullptr;  // the same with the handles' other brick maps
  uint64_t built_for = 0;  // sum of the handles' versions at the last build
  bool graph_on = false;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_iters = -1, g_cur = -1;
  uint64_t g_version = 0;
  int64_t g_launches = 0;
  LaunchShape shape;
  uint64_t shape_version = 0;  // changes with the shape (a new capture)
  int *work_off = nullptr;     // [(ORDER_BUCKETS + 1) n + 2] the step's work list
  // the collide's block tables (128, 256, 512 cells per block, one
  // allocation): (domain, block within the domain) for every block of cells
  // a domain has, so that no block of the grid falls past its domain
  int2 *cblk = nullptr;
  int cblk_off[3] = {0, 0, 0}, ncblk[3] = {0, 0, 0};
  std::string err;
};

extern "C" {

int lbm_batch_create(int n, lbm_t *const *handles, lbm_batch_t **out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !handles) return fail(nullptr, LBM_EINVAL, "empty batch");
  if (n > 65535) return fail(nullptr, LBM_EINVAL, "too many domains");
  for (int i = 0; i < n; i++) {
    if (!handles[i]) return fail(nullptr, LBM_EINVAL, "NULL handle %d", i);
    for (int j = 0; j < i; j++)
      if (handles[j] == handles[i]) return fail(nullptr, LBM_EINVAL, "handle %d twice", i);
    if (handles[i]->storage != handles[0]->storage)
      return fail(nullptr, LBM_EINVAL, "storage of handle %d differs", i);
  }
  lbm_batch_t *b = new lbm_batch();
  b->hs.assign(handles, handles + n);
  b->shape = handles[0]->shape;
  std::vector<int2> tab;
  for (int l = 0; l < 3; l++) {
    const int64_t cpb = 128 << l;
    b->cblk_off[l] = (int)tab.size();
    for (int d = 0; d < n; d++) {
      const int64_t nb = (handles[d]->g.ncell + cpb - 1) / cpb;
      for (int64_t k = 0; k < nb; k++) tab.push_back(make_int2(d, (int)k));
    }
    b->ncblk[l] = (int)tab.size() - b->cblk_off[l];
  }
  if (cudaMalloc(&b->D, sizeof(DomainDesc) * n) != cudaSuccess ||
      cudaMalloc(&b->D_alt, sizeof(DomainDesc) * n) != cudaSuccess ||
      cudaMalloc(&b->work_off, sizeof(int) * ((size_t)(ORDER_BUCKETS + 1) * n + 2)) !=
          cudaSuccess ||
      cudaMalloc(&b->cblk, sizeof(int2) * tab.size()) != cudaSuccess ||
      cudaMemcpy(b->cblk, tab.data(), sizeof(int2) * tab.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    if (b->D) cudaFree(b->D);
    if (b->D_alt) cudaFree(b->D_alt);
    if (b->work_off) cudaFree(b->work_off);
    if (b->cblk) cudaFree(b->cblk);
    delete b;
    return fail(nullptr, LBM_ENOMEM, "batch descriptors");
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_t *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->D) cudaFree(b->D);
  if (b->D_alt) cudaFree(b->D_alt);
  if (b->work_off) cudaFree(b->work_off);
  if (b->cblk) cudaFree(b->cblk);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  delete b;
}

int lbm_batch_set_graph(lbm_batch_t *b, int on) {
  if (!b) return LBM_EINVAL;
  b->graph_on = on != 0;
  return LBM_OK;
}

}  // extern "C"

// The tolerance-driven fixed point for a batch (the paper's loop): every
// domain iterates until its own eps <= ibm_tol or ibm_max_iter (the kernels
// of a converged domain return at once, so each domain's iterations are
// those it would take alone), the host reading all domains' stop flags after
// each chunk.  Returns LBM_WNOTCONVERGED when a domain hit the cap.
static int batch_tolerance_loop(lbm_batch_t *b, StepCtx &c, bool warm) {
  lbm_t *h0 = c.acct;
  cudaStream_t st = c.sti;
  bool moving = true;
  int hint = 0;
  for (lbm_t *h : b->hs) {
    if (h->np > 0 && !(h->nb > 0 ? h->bodies_moving : h->targets_nonzero)) moving = false;
    hint = std::max(hint, h->tol_hint);
  }
  auto read_states = [&]() -> int {
    for (lbm_t *h : b->hs)
      if (h->np > 0)
        CK(h0, cudaMemcpyAsync(h->state_host, h->state, 64, cudaMemcpyDeviceToHost, st));
    CK(h0, cudaStreamSynchronize(st));
    return LBM_OK;
  };
  {
    // denominators ||S[s u_k]||^2 of every domain
    StageTimer T(h0, ST_RESID, st, 2);
    CK(h0, launch_brick_norm(c.D, c.dims, 0, st));
    CK(h0, launch_ibm_den(c.D, c.dims, moving ? 2 : 0, st));
  }
  if (!moving) {
    int r = read_states();
    if (r) return r;
    bool zero = false;
    for (lbm_t *h : b->hs) zero = zero || (h->np > 0 && h->state_host->den2 == 0.0);
    if (zero) {
      // the fallback denominators ||S[s (u_k - I[U0])]||^2; domains whose
      // first denominator is non-zero keep it (ibm_den mode 1)
      StageTimer T(h0, ST_RESID, st, warm ? 5 : 3);
      if (warm) CK(h0, launch_brick_init(c.D, c.dims, 0, st));
      CK(h0, launch_point_residual0(c.D, c.dims, st));
      CK(h0, launch_brick_norm(c.D, c.dims, 1, st));
      CK(h0, launch_ibm_den(c.D, c.dims, 1, st));
      if (warm) CK(h0, launch_brick_init(c.D, c.dims, 1, st));
    }
  }
  int it = 0;
  const int max_iter = h0->max_iter;
  while (it < max_iter) {
    const int left = hint - it;
    const int chunk = std::min(left > 0 ? std::max(kCheckChunk, left / 2) : kCheckChunk,
                               max_iter - it);
    for (int j = 0; j < chunk; j++, it++) {
      {
        StageTimer T(h0, ST_UPDATE, st);
        CK(h0, launch_point_update(c.D, c.dims, it == 0, warm, 1, st));
      }
      {
        StageTimer T(h0, ST_SPREAD, st);
        CK(h0, launch_brick_spread(c.D, c.dims, 1, 1, st));
      }
      {
        StageTimer T(h0, ST_RESID, st);
        CK(h0, launch_ibm_check(c.D, c.dims, it, h0->tol, max_iter, st));
      }
    }
    int r = read_states();
    if (r) return r;
    bool all = true;
    for (lbm_t *h : b->hs) all = all && (h->np == 0 || h->state_host->done);
    if (all) break;
  }
  int warn = LBM_OK;
  for (lbm_t *h : b->hs) {
    if (h->np == 0) continue;
    h->last_iters = h->state_host->iters;
    h->tol_hint = h->last_iters;
    h->last_eps = h->state_host->last_eps;
    if (h->state_host->capped) {
      h->not_converged++;
      warn = LBM_WNOTCONVERGED;
    }
  }
  return warn;
}

extern "C" {

int lbm_batch_step(lbm_batch_t *b, int n_steps, int n_ibm_iter) {
  if (!b) return LBM_EINVAL;
  lbm_t *h0 = b->hs[0];
  if (n_steps < 0 || n_ibm_iter < 0)
    return fail(h0, LBM_EINVAL, "batch steps need n_steps >= 0 and n_ibm_iter >= 0");
  if (n_ibm_iter == 0 && h0->solver != LBM_SOLVER_MDF)
    return fail(h0, LBM_EINVAL, "a batch iterates to the residual target with the paper's loop "
                                "only (ibm_set_solver)");
  // uniform host-side decisions
  for (lbm_t *h : b->hs) {
    if (n_ibm_iter == 0 && (h->tol != h0->tol || h->max_iter != h0->max_iter))
      return fail(h0, LBM_EINVAL, "batch handles differ in ibm_tol or ibm_max_iter");
    if (h->stats_on != h0->stats_on || h->warm != h0->warm ||
        h->features_on != h0->features_on || h->cur != h0->cur || h->st != h0->st ||
        h->solver != h0->solver)
      return fail(h0, LBM_EINVAL, "batch handles differ in stats, warm start, features, stream, "
                                  "solver or lattice parity");
    if (h->u0_mode != LBM_U0_BRICKS)
      return fail(h0, LBM_EINVAL, "batches pre-compute U0 on the active bricks only "
                                  "(lbm_set_u0_strategy)");
    if ((h->np > 0 && h->have_du) != (h0->np > 0 && h0->have_du) && h->np > 0 && h0->np > 0)
      return fail(h0, LBM_EINVAL, "batch handles differ in warm-start history");
    if (h->nb > 0 && h->max_body >= h->nb)
      return fail(h0, LBM_EINVAL, "points refer to a missing body");
    if (h->warm == LBM_WARM_MLP && !h->mlp_packed && h->np > 0)
      return fail(h0, LBM_EINVAL, "learned warm start without weights");
    int r = discard_ahead(h);
    if (r) return r;
    r = sync_desc(h);
    if (r) return r;
    r = flush_points(h, h0->st);  // (batched kinematics read the device copies)
    if (r) return r;
  }
  uint64_t ver = b->shape_version;
  BatchDims dims{};
  dims.nd = (int)b->hs.size();
  dims.ls = b->shape;
  if (dims.nd > 1) dims.work_off = b->work_off;
  for (int l = 0; l < 3; l++) {
    dims.cblk[l] = b->cblk + b->cblk_off[l];
    dims.ncblk[l] = b->ncblk[l];
  }
  bool have_du = false;
  for (lbm_t *h : b->hs) {
    ver = ver * 1000003u + h->version;
    dims.max_cells = std::max<int64_t>(dims.max_cells, h->g.ncell);
    dims.max_points = std::max<int>(dims.max_points, (int)h->np);
    dims.max_bodies = std::max(dims.max_bodies, h->nb);
    dims.max_bricks = std::max(dims.max_bricks, h->g.nbrick);
    if (h->np > 0) {
      dims.max_slots = std::max(dims.max_slots, h->m.max_slots);
      have_du = h->have_du;
    }
  }
  if (ver != b->built_for) {
    std::vector<DomainDesc> hd, ha;
    for (lbm_t *h : b->hs) {
      hd.push_back(host_desc(h));
      ha.push_back(hd.back());
      ha.back().m.brick_slot = h->bslot_alt;
      ha.back().xpos = h->xpos_alt;
    }
    // (earlier steps of the batch may still read the old descriptors)
    CK(h0, h0->st ? cudaStreamSynchronize(h0->st) : cudaDeviceSynchronize());
    CK(h0, cudaMemcpy(b->D, hd.data(), sizeof(DomainDesc) * hd.size(), cudaMemcpyHostToDevice));
    CK(h0, cudaMemcpy(b->D_alt, ha.data(), sizeof(DomainDesc) * ha.size(),
                      cudaMemcpyHostToDevice));
    b->built_for = ver;
  }
  StepCtx c{};
  c.acct = h0;
  c.D = b->D;
  c.dims = dims;
  c.storage = h0->storage;
  c.stats = h0->stats_on;
  c.warm_mode = h0->warm;
  c.solver = h0->solver;
  c.have_du = have_du;
  c.features = h0->features_on;
  int s = 0;
  int warn = LBM_OK;
  while (s < n_steps) {
    c.cur = h0->cur;
    const bool steady = have_du || dims.max_points == 0;
    if (b->graph_on && steady && n_steps - s >= 2 && n_ibm_iter > 0) {
      if (!b->gexec || b->g_iters != n_ibm_iter || b->g_cur != c.cur || b->g_version != ver) {
        int r = ensure_capture_stream(h0, &b->cap_stream, &b->ev_in, &b->ev_out);
        if (r) return r;
        r = capture_two_steps(c, n_ibm_iter, b->cap_stream, &b->gexec, &b->g_launches,
                              b->D_alt);
        if (r) return r;
        b->g_iters = n_ibm_iter;
        b->g_cur = c.cur;
        b->g_version = ver;
      }
      int r = replay(h0, h0->st, b->cap_stream, b->ev_in, b->ev_out, b->gexec);
      if (r) return r;
      h0->nlaunch += b->g_launches;
      for (lbm_t *h : b->hs) {
        after_step(h, n_ibm_iter);
        after_step(h, n_ibm_iter);
      }
      s += 2;
      continue;
    }
    c.st = h0->st;
    c.sti = h0->st;
    c.split = false;
    int r = ensure_split(h0, c, false);
    if (r) return r;
    if (n_ibm_iter == 0 && dims.max_points > 0) {
      r = enqueue_head(c);
      if (r) return r;
      bool warm = false;
      r = enqueue_prefix(c, &warm);
      if (r) return r;
      const int w = batch_tolerance_loop(b, c, warm);
      if (w < 0) return w;
      if (w == LBM_WNOTCONVERGED) warn = w;
      r = enqueue_suffix(c);
    } else {
      r = enqueue_step(c, n_ibm_iter);
    }
    if (r) return r;
    for (lbm_t *h : b->hs) after_step(h, n_ibm_iter);
    have_du = have_du || dims.max_points > 0;
    c.have_du = have_du;
    s++;
  }
  return warn;
}

}  // extern "C"

}  // extern "C"

// ---- launch shapes and the autotuner ---------------------------------------

namespace {

bool shape_ok(const lbm_launch_shape &s) {
  return (s.collide_block == 128 || s.collide_block == 256) &&
         (s.point_block == 128 || s.point_block == 256 || s.point_block == 512) &&
         s.brick_blocks >= 1 && s.brick_blocks <= (1 << 20) && s.sort_blocks >= 1 &&
         s.sort_blocks <= (1 << 20) && s.sort_blocks_ahead >= 1 &&
         s.sort_blocks_ahead <= (1 << 20) &&
         (s.moments_spb == 1 || s.moments_spb == 2 || s.moments_spb == 4) &&
         (s.collide_staged >= 0 && s.collide_staged <= 2);
}

lbm_launch_shape to_c(const LaunchShape &l) {
  return {l.collide_block, l.brick_blocks, l.point_block, l.moments_spb, l.sort_blocks,
          l.collide_staged, l.sort_blocks_ahead};
}

LaunchShape from_c(const lbm_launch_shape &c) {
  LaunchShape l;
  l.collide_block = c.collide_block;
  l.brick_blocks = c.brick_blocks;
  l.point_block = c.point_block;
  l.moments_spb = c.moments_spb;
  l.sort_blocks = c.sort_blocks;
  l.collide_staged = c.collide_staged;
  l.sort_blocks_ahead = c.sort_blocks_ahead;
  return l;
}

// What a trial step changes and the autotuner puts back: the current
// population lattice, the per-point corrections, the step counter, the FP64
// sums and the host-side step bookkeeping.
struct Snapshot {
  void *f = nullptr;
  float4 *du = nullptr, *uint = nullptr;
  double sums[4] = {0, 0, 0, 0};
  int cur = 0, last_iters = 0;
  int64_t t = 0, not_converged = 0, nlaunch = 0;
  bool have_du = false, sums_valid = false;
  double last_eps = -1.0;
};

int snapshot_take(lbm_t *h, Snapshot &sn) {
  CK(h, cudaStreamSynchronize(h->st));
  const size_t pop = (size_t)Q * h->g.ncell * storage_bytes(h->storage);
  CK(h, cudaMalloc(&sn.f, pop));
  CK(h, cudaMemcpy(sn.f, h->f[h->cur], pop, cudaMemcpyDeviceToDevice));
  if (h->np > 0) {
    CK(h, dalloc(&sn.du, h->np));
    CK(h, dalloc(&sn.uint, h->np));
    CK(h, cudaMemcpy(sn.du, h->du, sizeof(float4) * h->np, cudaMemcpyDeviceToDevice));
    CK(h, cudaMemcpy(sn.uint, h->uint, sizeof(float4) * h->np, cudaMemcpyDeviceToDevice));
  }
  CK(h, cudaMemcpy(sn.sums, h->sums, sizeof sn.sums, cudaMemcpyDeviceToHost));
  sn.cur = h->cur;
  sn.t = h->t;
  sn.have_du = h->have_du;
  sn.sums_valid = h->sums_valid;
  sn.last_iters = h->last_iters;
  sn.last_eps = h->last_eps;
  sn.not_converged = h->not_converged;
  sn.nlaunch = h->nlaunch;
  return LBM_OK;
}

int snapshot_restore(lbm_t *h, Snapshot &sn) {
  CK(h, cudaStreamSynchronize(h->st));
  const size_t pop = (size_t)Q * h->g.ncell * storage_bytes(h->storage);
  CK(h, cudaMemcpy(h->f[sn.cur], sn.f, pop, cudaMemcpyDeviceToDevice));
  if (h->np > 0 && sn.du) {
    CK(h, cudaMemcpy(h->du, sn.du, sizeof(float4) * h->np, cudaMemcpyDeviceToDevice));
    CK(h, cudaMemcpy(h->uint, sn.uint, sizeof(float4) * h->np, cudaMemcpyDeviceToDevice));
  }
  CK(h, cudaMemcpy(h->sums, sn.sums, sizeof sn.sums, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(h->t_dev, &sn.t, sizeof sn.t, cudaMemcpyHostToDevice));
  h->cur = sn.cur;
  h->t = sn.t;
  h->have_du = sn.have_du;
  h->sums_valid = sn.sums_valid;
  h->last_iters = sn.last_iters;
  h->last_eps = sn.last_eps;
  h->not_converged = sn.not_converged;
  h->nlaunch = sn.nlaunch;
  return LBM_OK;
}

void snapshot_free(Snapshot &sn) {
  if (sn.f) cudaFree(sn.f);
  dfree(sn.du);
  dfree(sn.uint);
  sn.f = nullptr;
}

// The autotuner's candidates, one parameter after another, and the stages
// each one is timed on.
struct TuneParam {
  int LaunchShape::*field;
  std::vector<int> values;
  int stage_mask;
};

std::vector<TuneParam> tune_params(bool points, bool staged) {
  std::vector<TuneParam> ps;
  ps.push_back({&LaunchShape::collide_block, {128, 256}, 1 << ST_COLLIDE});
  if (staged) ps.push_back({&LaunchShape::collide_staged, {0, 1, 2}, 1 << ST_COLLIDE});
  if (points) {
    ps.push_back({&LaunchShape::brick_blocks,
                  {152 * 16, 152 * 32, 152 * 64, 152 * 128},
                  (1 << ST_SPREAD) | (1 << ST_INIT)});
    ps.push_back({&LaunchShape::point_block,
                  {128, 256, 512},
                  (1 << ST_KIN) | (1 << ST_PAIRS) | (1 << ST_UPDATE)});
    ps.push_back({&LaunchShape::moments_spb, {1, 2, 4}, 1 << ST_INIT});
    ps.push_back({&LaunchShape::sort_blocks, {152 * 8, 152 * 16, 152 * 32, 152 * 64},
                  1 << ST_PAIRS});
    ps.push_back({&LaunchShape::sort_blocks_ahead, {152 * 2, 152 * 4, 152 * 8, 152 * 32},
                  1 << ST_PAIRS});
  }
  return ps;
}

// Coordinate search over tune_params: step(k) advances the lattices k steps
// with the current shape; clear(mask) starts timing (mask != 0) or stops it,
// and stage_ms reads the device time of the steps timed since (whole steps:
// the stages of a step overlap).  Each candidate is timed in kRounds interleaved
// rounds and keeps its fastest; a candidate replaces the current value only
// when it is more than kMargin faster (timing noise does not move the shape).
constexpr int kRounds = 2;
constexpr double kMargin = 0.01;

template <typename SetShape, typename Step, typename Clear, typename StageMs>
int coordinate_search(LaunchShape &shape, bool points, bool staged, int steps_per_trial,
                      SetShape set_shape, Step step, Clear clear, StageMs stage_ms) {
  for (const TuneParam &p : tune_params(points, staged)) {
    const int incumbent = shape.*p.field;
    std::vector<double> best_ms(p.values.size(), 1e300);
    for (int round = 0; round < kRounds; round++) {
      for (size_t i = 0; i < p.values.size(); i++) {
        LaunchShape trial = shape;
        trial.*p.field = p.values[i];
        int r = set_shape(trial);
        if (r) return r;
        r = clear(0);
        if (r) return r;
        r = step(1);  // untimed
        if (r < 0) return r;
        r = clear(p.stage_mask);
        if (r) return r;
        r = step(steps_per_trial);
        if (r < 0) return r;
        double ms = 0.0;
        r = stage_ms(p.stage_mask, &ms);
        if (r) return r;
        best_ms[i] = std::min(best_ms[i], ms);
      }
    }
    double inc_ms = 1e300;
    size_t arg = 0;
    for (size_t i = 0; i < p.values.size(); i++) {
      if (p.values[i] == incumbent) inc_ms = best_ms[i];
      if (best_ms[i] < best_ms[arg]) arg = i;
    }
    shape.*p.field = best_ms[arg] < inc_ms * (1.0 - kMargin) ? p.values[arg] : incumbent;
    int r = set_shape(shape);
    if (r) return r;
  }
  return clear(0);
}


}  // namespace

extern "C" {

int lbm_get_launch_shape(lbm_t *h, lbm_launch_shape *out) {
  if (!h || !out) return LBM_EINVAL;
  *out = to_c(h->shape);
  return LBM_OK;
}

int lbm_set_launch_shape(lbm_t *h, const lbm_launch_shape *s) {
  if (!h || !s) return LBM_EINVAL;
  if (!shape_ok(*s)) return fail(h, LBM_EINVAL, "launch shape out of range");
  h->shape = from_c(*s);
  h->version++;  // a captured step holds the old shape
  return LBM_OK;
}

int lbm_autotune(lbm_t *h, int n_ibm_iter, int steps_per_trial, lbm_launch_shape *chosen) {
  if (!h) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (n_ibm_iter <= 0 || steps_per_trial < 1)
    return fail(h, LBM_EINVAL, "autotune needs n_ibm_iter > 0 and steps_per_trial >= 1");
  Snapshot sn;
  int r = snapshot_take(h, sn);
  if (r) {
    snapshot_free(sn);
    return r;
  }
  const bool graph = h->graph_on;
  h->graph_on = false;
  LaunchShape shape = h->shape;
  // whole steps, timed with events on the handle's stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float last_ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    r = fail(h, LBM_ECUDA, "event creation");
  bool timing = false;
  if (r == LBM_OK)
    r = coordinate_search(
        shape, h->np > 0, h->storage != LBM_STORE_F32, steps_per_trial,
        [&](const LaunchShape &l) {
          lbm_launch_shape c = to_c(l);
          return lbm_set_launch_shape(h, &c);
        },
        [&](int k) {
          if (timing) cudaEventRecord(e0, h->st);
          const int rr = lbm_step(h, k, n_ibm_iter);
          if (timing) cudaEventRecord(e1, h->st);
          return rr;
        },
        [&](int mask) {
          timing = mask != 0;
          return LBM_OK;
        },
        [&](int, double *ms) {
          CK(h, cudaEventSynchronize(e1));
          CK(h, cudaEventElapsedTime(&last_ms, e0, e1));
          *ms = last_ms;
          return LBM_OK;
        });
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->graph_on = graph;
  const int r2 = snapshot_restore(h, sn);
  snapshot_free(sn);
  if (r) return r;
  if (r2) return r2;
  if (chosen) *chosen = to_c(h->shape);
  return LBM_OK;
}

int lbm_batch_get_launch_shape(lbm_batch_t *b, lbm_launch_shape *out) {
  if (!b || !out) return LBM_EINVAL;
  *out = to_c(b->shape);
  return LBM_OK;
}

int lbm_batch_set_launch_shape(lbm_batch_t *b, const lbm_launch_shape *s) {
  if (!b || !s) return LBM_EINVAL;
  if (!shape_ok(*s)) return fail(b->hs[0], LBM_EINVAL, "launch shape out of range");
  b->shape = from_c(*s);
  b->shape_version++;
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_t *b, int n_ibm_iter, int steps_per_trial,
                       lbm_launch_shape *chosen) {
  if (!b) return LBM_EINVAL;
  lbm_t *h0 = b->hs[0];
  if (n_ibm_iter <= 0 || steps_per_trial < 1)
    return fail(h0, LBM_EINVAL, "autotune needs n_ibm_iter > 0 and steps_per_trial >= 1");
  std::vector<Snapshot> sn(b->hs.size());
  int r = LBM_OK;
  for (lbm_t *h : b->hs)
    if (r == LBM_OK) r = discard_ahead(h);
  for (size_t i = 0; i < b->hs.size() && r == LBM_OK; i++) r = snapshot_take(b->hs[i], sn[i]);
  bool points = false;
  for (lbm_t *h : b->hs) points = points || h->np > 0;
  const bool graph = b->graph_on;
  b->graph_on = false;
  LaunchShape shape = b->shape;
  // whole batch steps, timed with events on the first handle's stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float last_ms = 0.f;
  if (r == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    r = fail(h0, LBM_ECUDA, "event creation");
  bool timing = false;
  if (r == LBM_OK)
    r = coordinate_search(
        shape, points, h0->storage != LBM_STORE_F32, steps_per_trial,
        [&](const LaunchShape &l) {
          lbm_launch_shape c = to_c(l);
          return lbm_batch_set_launch_shape(b, &c);
        },
        [&](int k) {
          if (timing) cudaEventRecord(e0, h0->st);
          const int rr = lbm_batch_step(b, k, n_ibm_iter);
          if (timing) cudaEventRecord(e1, h0->st);
          return rr;
        },
        [&](int mask) {
          timing = mask != 0;
          return LBM_OK;
        },
        [&](int, double *ms) {
          CK(h0, cudaEventSynchronize(e1));
          CK(h0, cudaEventElapsedTime(&last_ms, e0, e1));
          *ms = last_ms;
          return LBM_OK;
        });
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->graph_on = graph;
  int r2 = LBM_OK;
  for (size_t i = 0; i < b->hs.size(); i++) {
    if (sn[i].f) {
      const int ri = snapshot_restore(b->hs[i], sn[i]);
      if (ri && !r2) r2 = ri;
    }
    snapshot_free(sn[i]);
  }
  if (r) return r;
  if (r2) return r2;
  if (chosen) *chosen = to_c(b->shape);
  return LBM_OK;
}

}  // extern "C"

extern "C" {

int lbm_read_fields_dev(lbm_t *h, float *rho, float *U, float *G) {
  if (!h) return LBM_EINVAL;
  if (rho || U) CK(h, launch_moments_dense(h->storage, h->g, h->f[h->cur], rho, U, h->st));
  if (G) {
    const float gb[3] = {(float)h->gbody[0], (float)h->gbody[1], (float)h->gbody[2]};
    CK(h, launch_force_dense(h->g, h->np > 0 ? h->m.brick_slot : nullptr, h->Gs, gb, G,
                             h->st));
  }
  return LBM_OK;
}

int lbm_read_fields(lbm_t *h, float *rho, float *U, float *G) {
  if (!h) return LBM_EINVAL;
  const size_t N = (size_t)h->g.ncell;
  int r = ensure_tmp(h, sizeof(float) * 7 * N);
  if (r) return r;
  float *drho = h->tmp, *dU = h->tmp + N, *dG = h->tmp + 4 * N;
  r = lbm_read_fields_dev(h, rho ? drho : nullptr, U ? dU : nullptr, G ? dG : nullptr);
  if (r) return r;
  if (rho) CK(h, cudaMemcpyAsync(rho, drho, sizeof(float) * N, cudaMemcpyDeviceToHost, h->st));
  if (U) CK(h, cudaMemcpyAsync(U, dU, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->st));
  if (G) CK(h, cudaMemcpyAsync(G, dG, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

int ibm_read_points_dev(lbm_t *h, double *x, float *u_interp, float *du) {
  if (!h) return LBM_EINVAL;
  if (h->np == 0) return LBM_OK;
  if (x) CK(h, launch_copy_f64(3 * h->np, h->xpos, x, h->st));
  if (u_interp) CK(h, launch_pack_points(h->np, h->uint, u_interp, h->st));
  if (du) CK(h, launch_pack_points(h->np, h->du, du, h->st));
  return LBM_OK;
}

int ibm_read_points_async(lbm_t *h, double *x, float *u_interp, float *du) {
  if (!h) return LBM_EINVAL;
  const int64_t n = h->np;
  if (n == 0) return LBM_OK;
  if (h->host_io == LBM_HOST_IO_MAPPED) {
    // kernels write straight into device-mapped host buffers
    void *mx = x ? (void *)mapped_ptr(x) : nullptr, *mu = u_interp ? (void *)mapped_ptr(u_interp)
                                                                   : nullptr;
    void *md = du ? (void *)mapped_ptr(du) : nullptr;
    if ((!x || mx) && (!u_interp || mu) && (!du || md))
      return ibm_read_points_dev(h, (double *)mx, (float *)mu, (float *)md);
  }
  int r = ensure_tmp(h, sizeof(double) * 3 * n + sizeof(float) * 6 * n);
  if (r) return r;
  double *dx = (double *)h->tmp;
  float *du_ = (float *)(dx + 3 * n), *dd = du_ + 3 * n;
  r = ibm_read_points_dev(h, x ? dx : nullptr, u_interp ? du_ : nullptr, du ? dd : nullptr);
  if (r) return r;
  if (x) CK(h, cudaMemcpyAsync(x, dx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->st));
  if (u_interp)
    CK(h, cudaMemcpyAsync(u_interp, du_, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->st));
  if (du) CK(h, cudaMemcpyAsync(du, dd, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->st));
  return LBM_OK;
}

int ibm_read_points(lbm_t *h, double *x, float *u_interp, float *du) {
  const int r = ibm_read_points_async(h, x, u_interp, du);
  if (r || h->np == 0) return r;
  CK(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

int lbm_read_sums_async(lbm_t *h, double *sums) {
  if (!h || !sums) return LBM_EINVAL;
  if (!h->sums_valid) return LBM_OK;
  void *ms = h->host_io == LBM_HOST_IO_MAPPED ? (void *)mapped_ptr(sums) : nullptr;
  if (ms)
    CK(h, launch_copy_f64(4, h->sums, (double *)ms, h->st));
  else
    CK(h, cudaMemcpyAsync(sums, h->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return LBM_OK;
}

int lbm_set_host_io(lbm_t *h, int mode) {
  if (!h) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (mode != LBM_HOST_IO_COPY && mode != LBM_HOST_IO_MAPPED)
    return fail(h, LBM_EINVAL, "unknown host transfer mode %d", mode);
  if (mode == LBM_HOST_IO_COPY) {
    const int r = flush_points(h, h->st);
    if (r) return r;
  }
  h->host_io = mode;
  return LBM_OK;
}

int lbm_get_host_io(lbm_t *h, int *mode) {
  if (!h || !mode) return LBM_EINVAL;
  *mode = h->host_io;
  return LBM_OK;
}

int lbm_read_stats(lbm_t *h, lbm_stats *s) {
  if (!h || !s) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  memset(s, 0, sizeof *s);
  double sums[4] = {0, 0, 0, 0};
  if (h->sums_valid) {
    CK(h, cudaMemcpyAsync(sums, h->sums, sizeof sums, cudaMemcpyDeviceToHost, h->st));
  }
  CK(h, cudaStreamSynchronize(h->st));
  s->mass = sums[0];
  s->momentum[0] = sums[1];
  s->momentum[1] = sums[2];
  s->momentum[2] = sums[3];
  s->step = h->t;
  s->last_ibm_iters = h->last_iters;
  s->last_residual = h->last_eps;
  s->not_converged = h->not_converged;
  s->kernel_launches = h->nlaunch;
  if (h->np > 0) {
    int c[8] = {0};
    CK(h, cudaMemcpy(c, h->m.counters, sizeof c, cudaMemcpyDeviceToHost));
    s->active_bricks = c[0];
    if (c[5] & 4) {
      CK(h, cudaMemset(h->m.counters + 5, 0, sizeof(int)));
      return fail(h, LBM_ECUDA, "brick compaction scan timed out");
    }
  }
  if (h->sums_valid && !(isfinite(sums[0]) && isfinite(sums[1]) && isfinite(sums[2]) &&
                         isfinite(sums[3])))
    return fail(h, LBM_ENONFINITE, "non-finite mass or momentum sum");
  return LBM_OK;
}

static int read_pops(lbm_t *h, float *f, int deviations) {
  if (!h || !f) return LBM_EINVAL;
  const size_t n = (size_t)Q * h->g.ncell;
  int r = ensure_tmp(h, sizeof(float) * n);
  if (r) return r;
  CK(h, launch_read_populations(h->storage, h->g, h->f[h->cur], h->tmp, deviations, h->st));
  CK(h, cudaMemcpyAsync(f, h->tmp, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return LBM_OK;
}

int lbm_read_populations(lbm_t *h, float *f) { return read_pops(h, f, 0); }

int lbm_read_residuals(lbm_t *h, double *eps, int cap) {
  if (!h || cap < 0 || (cap > 0 && !eps)) return LBM_EINVAL;
  if (h->last_eps < 0.0) return 0;
  const int n = std::min(h->last_iters, (int)IbmState::HIST);
  const int m = std::min(n, cap);
  if (m > 0)
    CK(h, cudaMemcpyAsync(eps, h->state->eps, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return n;
}
int lbm_read_deviations(lbm_t *h, float *d) { return read_pops(h, d, 1); }

int lbm_write_populations(lbm_t *h, const float *f) {
  if (!h || !f) return LBM_EINVAL;
  const size_t n = (size_t)Q * h->g.ncell;
  if (!all_finite(f, n)) return fail(h, LBM_ENONFINITE, "non-finite population");
  int r = ensure_tmp(h, sizeof(float) * n);
  if (r) return r;
  CK(h, cudaMemcpyAsync(h->tmp, f, sizeof(float) * n, cudaMemcpyHostToDevice, h->st));
  CK(h, launch_write_populations(h->storage, h->g, h->tmp, h->f[h->cur], h->st));
  CK(h, cudaStreamSynchronize(h->st));
  h->have_du = false;
  return LBM_OK;
}

int lbm_enable_timing(lbm_t *h, int mask) {
  if (!h) return LBM_EINVAL;
  CK(h, h->st ? cudaStreamSynchronize(h->st) : cudaDeviceSynchronize());
  for (auto &p : h->pending) {
    h->free_events.push_back(p.a);
    h->free_events.push_back(p.b);
  }
  h->pending.clear();
  memset(h->ms, 0, sizeof h->ms);
  memset(h->launches, 0, sizeof h->launches);
  h->timing = mask;
  return LBM_OK;
}

int lbm_num_stages(void) { return kNumStages; }
const char *lbm_stage_name(int i) { return i >= 0 && i < kNumStages ? kStageNames[i] : ""; }

int lbm_read_timing(lbm_t *h, double *ms, int64_t *launches) {
  if (!h) return LBM_EINVAL;
  CK(h, cudaStreamSynchronize(h->st));
  for (auto &p : h->pending) {
    float e = 0.f;
    CK(h, cudaEventElapsedTime(&e, p.a, p.b));
    h->ms[p.stage] += e;
    h->launches[p.stage] += p.launches;
    h->free_events.push_back(p.a);
    h->free_events.push_back(p.b);
  }
  h->pending.clear();
  for (int i = 0; i < kNumStages; i++) {
    if (ms) ms[i] = h->ms[i];
    if (launches) launches[i] = h->launches[i];
  }
  return LBM_OK;
}

// ---- checkpoint ------------------------------------------------------------

namespace {
struct StateHeader {
  char magic[8];
  int32_t version, nx, ny, nz, storage, delta, warm, have_du, nb, pad;
  int64_t np, t;
  double tau, gbody[3];
};
const char kMagic[8] = {'L', 'B', 'M', 'I', 'B', 'M', '0', '1'};
}  // namespace

int lbm_save_state(lbm_t *h, void *buf, size_t *len) {
  if (!h || !len) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (buf) {
    const int rf = flush_points(h, h->st);  // (the last mapped upload belongs to the state)
    if (rf) return rf;
  }
  const size_t pop = (size_t)Q * h->g.ncell * storage_bytes(h->storage);
  const size_t np = (size_t)h->np, nb = (size_t)h->nb;
  const size_t need = sizeof(StateHeader) + pop + np * (3 * 8 + 4 + 4 + 12 + 16) +
                      nb * (3 * 8 + 8 + 8);
  if (!buf) {
    *len = need;
    return LBM_OK;
  }
  if (*len < need) return fail(h, LBM_ESTATE, "buffer of %zu bytes, need %zu", *len, need);
  StateHeader hd{};
  memcpy(hd.magic, kMagic, 8);
  hd.version = 1;
  hd.nx = h->g.nx;
  hd.ny = h->g.ny;
  hd.nz = h->g.nz;
  hd.storage = h->storage;
  hd.delta = h->delta;
  hd.warm = h->warm;
  hd.have_du = h->have_du;
  hd.nb = h->nb;
  hd.np = h->np;
  hd.t = h->t;
  hd.tau = h->tau;
  memcpy(hd.gbody, h->gbody, sizeof hd.gbody);
  char *p = (char *)buf;
  memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  CK(h, cudaStreamSynchronize(h->st));
  CK(h, cudaMemcpy(p, h->f[h->cur], pop, cudaMemcpyDeviceToHost));
  p += pop;
  if (np) {
    CK(h, cudaMemcpy(p, h->X, 24 * np, cudaMemcpyDeviceToHost));
    p += 24 * np;
    CK(h, cudaMemcpy(p, h->body, 4 * np, cudaMemcpyDeviceToHost));
    p += 4 * np;
    CK(h, cudaMemcpy(p, h->area, 4 * np, cudaMemcpyDeviceToHost));
    p += 4 * np;
    CK(h, cudaMemcpy(p, h->utarget, 12 * np, cudaMemcpyDeviceToHost));
    p += 12 * np;
    CK(h, cudaMemcpy(p, h->du, 16 * np, cudaMemcpyDeviceToHost));
    p += 16 * np;
  }
  if (nb) {
    CK(h, cudaMemcpy(p, h->centre, 24 * nb, cudaMemcpyDeviceToHost));
    p += 24 * nb;
    CK(h, cudaMemcpy(p, h->omega, 8 * nb, cudaMemcpyDeviceToHost));
    p += 8 * nb;
    CK(h, cudaMemcpy(p, h->phase, 8 * nb, cudaMemcpyDeviceToHost));
    p += 8 * nb;
  }
  *len = need;
  return LBM_OK;
}

int lbm_load_state(lbm_t *h, const void *buf, size_t len) {
  if (!h || !buf) return LBM_EINVAL;
  {
    const int ra = discard_ahead(h);  // (a prepared step would not be taken)
    if (ra) return ra;
  }
  if (len < sizeof(StateHeader)) return fail(h, LBM_ESTATE, "state buffer too short");
  StateHeader hd;
  memcpy(&hd, buf, sizeof hd);
  if (memcmp(hd.magic, kMagic, 8) || hd.version != 1)
    return fail(h, LBM_ESTATE, "not a state buffer of this library");
  if (hd.nx != h->g.nx || hd.ny != h->g.ny || hd.nz != h->g.nz || hd.storage != h->storage)
    return fail(h, LBM_ESTATE, "state of a %d x %d x %d lattice (storage %d)", hd.nx, hd.ny,
                hd.nz, hd.storage);
  const size_t pop = (size_t)Q * h->g.ncell * storage_bytes(h->storage);
  const size_t np = (size_t)hd.np, nb = (size_t)hd.nb;
  const size_t need = sizeof(StateHeader) + pop + np * (3 * 8 + 4 + 4 + 12 + 16) +
                      nb * (3 * 8 + 8 + 8);
  if (len < need) return fail(h, LBM_ESTATE, "state buffer of %zu bytes, need %zu", len, need);
  const char *p = (const char *)buf + sizeof hd;
  const char *pp = p + pop;
  const double *X = (const double *)pp;
  const int32_t *body = (const int32_t *)(pp + 24 * np);
  const float *area = (const float *)(pp + 28 * np);
  const float *ut = (const float *)(pp + 32 * np);
  const float *du = (const float *)(pp + 44 * np);
  const char *pb = pp + 60 * np;
  // bodies first (points are validated against them)
  int r = ibm_set_bodies(h, 0, nullptr, nullptr, nullptr);
  if (r) return r;
  r = ibm_set_points(h, (int64_t)np, np ? X : nullptr, np ? ut : nullptr, np ? area : nullptr,
                     np ? body : nullptr);
  if (r) return r;
  if (nb) {
    r = ibm_set_bodies(h, (int)nb, (const double *)pb, (const double *)(pb + 24 * nb),
                       (const double *)(pb + 32 * nb));
    if (r) return r;
  }
  CK(h, cudaMemcpy(h->f[h->cur], p, pop, cudaMemcpyHostToDevice));
  if (np) CK(h, cudaMemcpy(h->du, du, 16 * np, cudaMemcpyHostToDevice));
  h->have_du = hd.have_du != 0;
  CK(h, cudaMemcpy(h->t_dev, &hd.t, sizeof hd.t, cudaMemcpyHostToDevice));
  h->t = hd.t;
  h->delta = hd.delta;
  h->warm = hd.warm;
  h->tau = hd.tau;
  h->desc_dirty = true;
  memcpy(h->gbody, hd.gbody, sizeof hd.gbody);
  return LBM_OK;
}

// ---- stateless operators ----------------------------------------------------

int ibm_interpolate_dev(int nx, int ny, int nz, int delta, const float *U, int64_t n,
                        const double *x, float *u, void *stream) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || n < 0 || (delta != 0 && delta != 1))
    return fail(nullptr, LBM_EINVAL, "bad arguments to ibm_interpolate_dev");
  if (n > 0 && (!U || !x || !u)) return fail(nullptr, LBM_EINVAL, "NULL pointer");
  Geometry g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.ncell = (int64_t)nx * ny * nz;
  cudaError_t e = launch_interp_dense(g, delta, U, n, x, u, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "%s", cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"

namespace {

struct SpreadLayout {
  size_t desc, brick_count, brick_slot, slot_brick, order, counters, tiles, count, start, cursor, pk,
      pbrick, pw,
      ppart,
      point_pairs, base, wts, ut, vals, Gs, total;
  int max_slots;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

SpreadLayout spread_layout(const Geometry &g, int64_t n) {
  SpreadLayout L{};
  const int64_t ms = std::max<int64_t>(1, std::min<int64_t>(g.nbrick, 8 * n));
  const int64_t n1 = std::max<int64_t>(n, 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align256(o + bytes);
    return r;
  };
  L.desc = take(sizeof(DomainDesc));
  L.brick_count = take(sizeof(int) * g.nbrick);
  L.brick_slot = take(sizeof(int) * g.nbrick);
  L.slot_brick = take(sizeof(int) * ms);
  L.order = take(sizeof(int) * ORDER_BUCKETS * ms);
  L.counters = take(sizeof(int) * BRICK_COUNTERS);
  L.tiles = take(sizeof(unsigned long long) * ((g.nbrick + COMPACT_TILE - 1) / COMPACT_TILE));
  L.count = take(sizeof(int) * ms);
  L.start = take(sizeof(int) * (ms + 1));
  L.cursor = take(sizeof(int) * ms);
  L.pk = take(sizeof(int) * 8 * n1);
  L.pbrick = take(sizeof(int) * 8 * n1);
  L.pw = take(sizeof(float4) * 3 * 8 * n1);
  L.ppart = take(sizeof(float4) * 8 * n1);
  L.point_pairs = take(sizeof(int) * 8 * n1);
  L.base = take(sizeof(int4) * n1);
  L.wts = take(sizeof(float) * 12 * n1);
  L.ut = take(sizeof(float4) * n1);
  L.vals = take(sizeof(float4) * n1);
  L.Gs = take(sizeof(float) * SLOT_FLOATS * ms);
  L.total = o;
  L.max_slots = (int)ms;
  return L;
}

bool spread_geometry(int nx, int ny, int nz, Geometry &g) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || nx % 4 || ny % 4 || nz % 4) return false;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nbx = nx / 4;
  g.nby = ny / 4;
  g.nbz = nz / 4;
  g.ncell = (int64_t)nx * ny * nz;
  g.nbrick = g.nbx * g.nby * g.nbz;
  geometry_divisors(g);
  return g.ncell < (1LL << 31);
}

}  // namespace

extern "C" {

size_t ibm_spread_scratch_bytes(int nx, int ny, int nz, int64_t n) {
  Geometry g{};
  if (!spread_geometry(nx, ny, nz, g) || n < 0) return 0;
  return spread_layout(g, n).total;
}

int ibm_spread_dev(int nx, int ny, int nz, int delta, int64_t n, const double *x,
                   const float *v, float *F, void *scratch, void *stream) {
  Geometry g{};
  if (!spread_geometry(nx, ny, nz, g) || n < 0 || (delta != 0 && delta != 1))
    return fail(nullptr, LBM_EINVAL, "bad arguments to ibm_spread_dev");
  if (!F || (n > 0 && (!x || !v))) return fail(nullptr, LBM_EINVAL, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const SpreadLayout L = spread_layout(g, n);
  char *base = (char *)scratch;
  bool own = false;
  cudaError_t e = cudaSuccess;
  if (!base) {
    e = cudaMallocAsync((void **)&base, L.total, st);
    if (e != cudaSuccess) return fail(nullptr, LBM_ENOMEM, "%s", cudaGetErrorString(e));
    own = true;
  } else if (((uintptr_t)base) & 255) {
    return fail(nullptr, LBM_EINVAL, "scratch must be 256-byte aligned");
  }
  BrickMap m{};
  m.brick_count = (int *)(base + L.brick_count);
  m.brick_slot = (int *)(base + L.brick_slot);
  m.slot_brick = (int *)(base + L.slot_brick);
  m.order = (int *)(base + L.order);
  m.counters = (int *)(base + L.counters);
  m.tiles = (unsigned long long *)(base + L.tiles);
  m.max_slots = L.max_slots;
  PairMap pm{};
  pm.count = (int *)(base + L.count);
  pm.start = (int *)(base + L.start);
  pm.cursor = (int *)(base + L.cursor);
  pm.k = (int *)(base + L.pk);
  pm.brick = (int *)(base + L.pbrick);
  pm.w = (float4 *)(base + L.pw);
  pm.part = (float4 *)(base + L.ppart);
  pm.point_pairs = (int *)(base + L.point_pairs);
  pm.max_pairs = 8 * n;
  PointPrep pp{};
  pp.base = (int4 *)(base + L.base);
  pp.wts = (float *)(base + L.wts);
  pp.ut = (float4 *)(base + L.ut);
  float4 *vals = (float4 *)(base + L.vals);
  float *Gs = (float *)(base + L.Gs);
  if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, sizeof(float) * 3 * g.ncell, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m.brick_count, 0, sizeof(int) * g.nbrick, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m.counters, 0, sizeof(int) * BRICK_COUNTERS, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(m.tiles, 0,
                        sizeof(unsigned long long) *
                            ((g.nbrick + COMPACT_TILE - 1) / COMPACT_TILE),
                        st);
  if (n > 0) {
    // a batch of one domain whose descriptor lives in the scratch
    DomainDesc dd{};
    dd.g = g;
    dd.delta = delta;
    dd.np = (int)n;
    dd.X = x;
    dd.pp = pp;
    dd.m = m;
    dd.pm = pm;
    dd.du = vals;
    dd.Gs = Gs;
    DomainDesc *D = (DomainDesc *)(base + L.desc);
    BatchDims dims{};
    dims.nd = 1;
    dims.max_cells = g.ncell;
    dims.max_points = (int)n;
    dims.max_bricks = g.nbrick;
    dims.max_slots = m.max_slots;
    if (e == cudaSuccess) e = launch_store_desc(dd, D, st);
    if (e == cudaSuccess) e = launch_prepare_points(D, dims, st);
    if (e == cudaSuccess) e = launch_compact(D, dims, st);
    if (e == cudaSuccess) e = launch_pair_lists(D, dims, st);
    if (e == cudaSuccess) e = launch_pack_vals(n, v, vals, st);
    if (e == cudaSuccess) e = launch_brick_spread(D, dims, 0, 0, st);
    if (e == cudaSuccess) e = launch_slots_to_dense(g, m, Gs, F, st);
  }
  if (own) {
    cudaError_t e2 = cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess)
    return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s",
                cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"

// ---- spreading without any allocation ---------------------------------------
//
// Scratch for ibm_spread_dev_noalloc: a static device array, so the call never
// allocates.  Host code only knows the symbol; its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current
// and kept for the life of the process (a device reset would invalidate it;
// the header states that limit).

static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int ibm_spread_dev_noalloc(int nx, int ny, int nz, int delta, int64_t n,
                                      const double *x, const float *v, float *F,
                                      void *stream) {
  const size_t need = ibm_spread_scratch_bytes(nx, ny, nz, n);
  if (need == 0)
    return fail(nullptr, LBM_EINVAL, "bad arguments to ibm_spread_dev_noalloc");
  if (need > LBM_NOALLOC_SCRATCH_BYTES)
    return fail(nullptr, LBM_EINVAL,
                "ibm_spread_dev_noalloc: %d x %d x %d with %lld points needs %zu bytes of "
                "scratch, the static area holds %zu",
                nx, ny, nz, (long long)n, need, (size_t)LBM_NOALLOC_SCRATCH_BYTES);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(nullptr, LBM_EINVAL, "device ordinal %d out of range", dev);
  void *ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        return fail(nullptr, LBM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
    }
    ptr = g_noalloc_addr[dev];
  }
  // the allocating entry point with caller scratch: it allocates nothing and
  // clears the output and the binning state it needs at zero
  return ibm_spread_dev(nx, ny, nz, delta, n, x, v, F, ptr, stream);
}

// ---- learned warm start -------------------------------------------------------

extern "C" {

size_t mlp_packed_bytes(void) { return lbmibm::mlp_packed_bytes(); }

int mlp_pack_dev(const float *P, void *packed, void *stream) {
  if (!P || !packed) return fail(nullptr, LBM_EINVAL, "NULL pointer");
  cudaError_t e = launch_mlp_pack(P, packed, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "%s", cudaGetErrorString(e));
  return LBM_OK;
}

int mlp_forward_dev(int64_t n, const float *X, const void *packed, float *Y, void *stream) {
  if (n < 0 || (n > 0 && (!X || !packed || !Y))) return fail(nullptr, LBM_EINVAL, "bad arguments");
  cudaError_t e = launch_mlp_forward(n, X, packed, Y, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "%s", cudaGetErrorString(e));
  return LBM_OK;
}

size_t mlp_grad_scratch_bytes(int64_t n) {
  return n > 0 ? sizeof(float) * mlp_grad_scratch_floats(n) : 0;
}

int mlp_loss_grad_dev(int64_t n, const float *X, const float *T, const float *P,
                      const void *packed, float *grad, float *loss, void *scratch, void *stream) {
  if (n <= 0 || !X || !T || !P || !packed || !grad || !scratch)
    return fail(nullptr, LBM_EINVAL, "bad arguments to mlp_loss_grad_dev");
  cudaError_t e = launch_mlp_loss_grad(n, X, T, packed, P, grad, loss, (float *)scratch,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "%s", cudaGetErrorString(e));
  return LBM_OK;
}

int mlp_adam_dev(float *P, float *m, float *v, const float *grad, int64_t step, double lr,
                 double beta1, double beta2, double eps, void *packed, void *stream) {
  if (!P || !m || !v || !grad || step < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(nullptr, LBM_EINVAL, "bad arguments to mlp_adam_dev");
  cudaError_t e = launch_mlp_adam(P, m, v, grad, step, (float)lr, (float)beta1, (float)beta2,
                                  (float)eps, packed, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "%s", cudaGetErrorString(e));
  return LBM_OK;
}

static int set_weights(lbm_t *h, const float *P, cudaMemcpyKind kind) {
  if (!h || !P) return LBM_EINVAL;
  if (kind == cudaMemcpyHostToDevice && !all_finite(P, MLP_NPARAM))
    return fail(h, LBM_ENONFINITE, "non-finite MLP weight");
  if (!h->mlp_P) CK(h, dalloc(&h->mlp_P, MLP_NPARAM));
  if (!h->mlp_packed) CK(h, cudaMalloc(&h->mlp_packed, lbmibm::mlp_packed_bytes()));
  CK(h, cudaMemcpyAsync(h->mlp_P, P, sizeof(float) * MLP_NPARAM, kind, h->st));
  CK(h, launch_mlp_pack(h->mlp_P, h->mlp_packed, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  h->desc_dirty = true;
  return LBM_OK;
}

int mlp_set_weights(lbm_t *h, const float *P) { return set_weights(h, P, cudaMemcpyHostToDevice); }
int mlp_set_weights_dev(lbm_t *h, const float *P) {
  return set_weights(h, P, cudaMemcpyDeviceToDevice);
}

int lbm_set_features(lbm_t *h, int on) {
  if (!h) return LBM_EINVAL;
  h->features_on = on != 0;
  return LBM_OK;
}

int ibm_read_mlp_sample_dev(lbm_t *h, float *X, float *T) {
  if (!h) return LBM_EINVAL;
  if (h->np == 0) return LBM_OK;
  if (!(h->features_on || h->warm == LBM_WARM_MLP))
    return fail(h, LBM_EINVAL, "features are not computed (lbm_set_features)");
  if (X)
    CK(h, cudaMemcpyAsync(X, h->feat, sizeof(float) * MLP_IN * h->np, cudaMemcpyDeviceToDevice,
                          h->st));
  if (T) CK(h, launch_mlp_targets(h->np, h->feat, h->du, T, h->st));
  return LBM_OK;
}

}  // extern "C"
