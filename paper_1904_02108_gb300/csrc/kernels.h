// Host-side launchers of the device kernels (internal C++ interface between
// the C ABI in api.cu and the kernels in lbm.cu / ibm.cu).  Every launcher
// enqueues on `st` and returns the launch status; none synchronises.
#pragma once

#include "common.cuh"

namespace lbmibm {

// ----------------------------------------------------------------- lbm.cu
// Fused pull-stream + collision f[cur] -> f[1 - cur] of every domain, with
// the IBM force of its active bricks and its body force; FP64 partial sums
// per PARTIAL_CELLS cells when stats.  skip_active: the cells of the step's
// active bricks are left out (launch_collide_active does them).
// Dhost: host copy of D when dims.nd == 1 (passed as a kernel parameter), or
// NULL.
cudaError_t launch_collide_stream(int storage, const DomainDesc *D, const DomainDesc *Dhost,
                                  const BatchDims &dims, int cur, int stats, int skip_active,
                                  cudaStream_t st);
// The same collision on the cells of the active bricks only (after the IBM
// loop); FP64 partial sums per slot when stats.
cudaError_t launch_collide_active(int storage, const DomainDesc *D, const BatchDims &dims,
                                  int cur, int stats, cudaStream_t st);
// End of a step: FP64 reduction of the collide partials into sums (if
// stats; split: with the active bricks' slot partials) and t += 1 of every
// domain.
cudaError_t launch_finish_step(const DomainDesc *D, const BatchDims &dims, int stats, int split,
                               cudaStream_t st);
// FP64 partial sums per step of a lattice (one per PARTIAL_CELLS cells)
int collide_partials(const Geometry &g);
// rho[N], U[3][N] on every cell (either may be NULL).
cudaError_t launch_moments_dense(int storage, const Geometry &g, const void *f, float *rho,
                                 float *U, cudaStream_t st);
// full populations f[19][N] <-> stored deviations, with the pull offset.
cudaError_t launch_read_populations(int storage, const Geometry &g, const void *f,
                                    float *out, int deviations, cudaStream_t st);
cudaError_t launch_write_populations(int storage, const Geometry &g, const float *in,
                                     void *f, cudaStream_t st);
// dense G[3][N] from the slot storage (+ body force)
cudaError_t launch_force_dense(const Geometry &g, const int *brick_slot, const float *Gs,
                               const float gbody[3], float *G, cudaStream_t st);

// ----------------------------------------------------------------- ibm.cu
struct Bodies {
  const double *centre;  // [nb][3]
  const double *omega;   // [nb]
  const double *phase;   // [nb]
  int nb;
};
struct PointsIn {
  int64_t np;
  const double *X;        // [np][3]
  const int *body;        // [np] or NULL
  const float *area;      // [np] or NULL (1)
  const float *utarget;   // [np][3] or NULL (0)
};
// ---- step kernels over a batch of domains (D: device array of dims.nd) ----
// Kinematics (Alg. 1, first iteration; each block computes the rotation of
// its points' bodies once) + per-point weights + brick counts.  t_step >= 0:
// the kinematics of that step (a step prepared ahead, while the step before
// it still runs); else of the device's step counter.
cudaError_t launch_prepare_points(const DomainDesc *D, const BatchDims &dims, cudaStream_t st,
                                  const double *Xsrc = nullptr, const float *Usrc = nullptr,
                                  long long t_step = -1);
// counted bricks -> slots (1 launch)
cudaError_t launch_compact(const DomainDesc *D, const BatchDims &dims, cudaStream_t st);
// a batch's work list from the domains' slot counts (1 launch when
// dims.work_off, else none)
cudaError_t launch_batch_worklist(const DomainDesc *D, const BatchDims &dims, cudaStream_t st);
// (brick, point) pairs grouped by slot in a fixed order, with brick-local
// weights (2 launches when points exist, else none)
cudaError_t launch_pair_lists(const DomainDesc *D, const BatchDims &dims, cudaStream_t st);
// U0 on the active bricks (pull + Eq. 1) from lattice f[cur]
cudaError_t launch_brick_moments(int storage, const DomainDesc *D, const BatchDims &dims, int cur,
                                 cudaStream_t st);
// The paper's two other U0 pre-computations (Sec. 5), single lattice:
// box strategy (every cell of each body's moved bounding box into the
// full-lattice D->Ufull, then the active bricks' cells from it; 2 launches)
// and kernel strategy (the support of every point, 1 launch).
cudaError_t launch_box_moments(int storage, const DomainDesc *D, int nbox, int cur,
                               cudaStream_t st);
cudaError_t launch_point_moments(int storage, const DomainDesc *D, int64_t np, int cur,
                                 cudaStream_t st);
// G_0 = 0 or S[du] (use_du), pair shares of I[U0 + G_0]
cudaError_t launch_brick_init(const DomainDesc *D, const BatchDims &dims, int use_du,
                              cudaStream_t st);
// G = S[du] on the active bricks (Alg. 2 as a gather); in tolerance mode the
// squared change of G per brick into res and an early exit once converged;
// pair shares of I[U0 + G] if do_interp
cudaError_t launch_brick_spread(const DomainDesc *D, const BatchDims &dims, int do_interp,
                                int tol_mode, cudaStream_t st);
// u_n(k) from the pair shares; g = u_k - u_n; du += s g (Alg. 1 loop body)
cudaError_t launch_point_update(const DomainDesc *D, const BatchDims &dims, int first, int warm,
                                int tol_mode, cudaStream_t st);
// ||S[v]||^2 per brick into res; which 0: v = s u_k, 1: v = uint
cudaError_t launch_brick_norm(const DomainDesc *D, const BatchDims &dims, int which,
                              cudaStream_t st);
// residual denominators (mode 0: ||S[s u_k]||^2, mode 1: fallback) and the
// per-iteration convergence check of the tolerance mode
cudaError_t launch_ibm_den(const DomainDesc *D, const BatchDims &dims, int mode, cudaStream_t st);
cudaError_t launch_ibm_check(const DomainDesc *D, const BatchDims &dims, int it, double tol,
                             int max_iter, cudaStream_t st);
// conjugate gradients on the lattice form of the fixed point (ibm.cu)
cudaError_t launch_cg_start(const DomainDesc *D, const BatchDims &dims, int warm,
                            cudaStream_t st);
cudaError_t launch_cg_brick(const DomainDesc *D, const BatchDims &dims, int tol_mode,
                            cudaStream_t st);
cudaError_t launch_cg_replace(const DomainDesc *D, const BatchDims &dims, cudaStream_t st);
cudaError_t launch_cg_dot(const DomainDesc *D, const BatchDims &dims, int tol_mode,
                          cudaStream_t st);
cudaError_t launch_cg_update(const DomainDesc *D, const BatchDims &dims, int it, double tol,
                             int max_iter, int tol_mode, int confirm, cudaStream_t st);
// uint = s (u_k - u) from the pair shares (fallback denominator)
cudaError_t launch_point_residual0(const DomainDesc *D, const BatchDims &dims, cudaStream_t st);
// features of the learned warm start from the pair shares (see ibm.cu)
cudaError_t launch_mlp_features(const DomainDesc *D, const BatchDims &dims, int use_prev,
                                cudaStream_t st);
// training sample target T = (du - du_prev) / MLP_VSCALE, du_prev from X
cudaError_t launch_mlp_targets(int64_t np, const float *X, const float4 *du, float *T,
                               cudaStream_t st);

// ----------------------------------------------------------------- mlp.cu
size_t mlp_packed_bytes();
size_t mlp_train_smem_bytes();
size_t mlp_grad_scratch_floats(int64_t n);
cudaError_t launch_mlp_pack(const float *P, void *packed, cudaStream_t st);
// Y[n][3] = MLP(X)
cudaError_t launch_mlp_forward(int64_t n, const float *X, const void *packed, float *Y,
                               cudaStream_t st);
// learned start of every domain: du = (use_prev ? du : 0) + MLP_VSCALE MLP(feat)
cudaError_t launch_mlp_warm(const DomainDesc *D, const BatchDims &dims, int use_prev,
                            cudaStream_t st);
cudaError_t launch_mlp_loss_grad(int64_t n, const float *X, const float *T, const void *packed,
                                 const float *P, float *grad, float *loss, float *part,
                                 cudaStream_t st);
cudaError_t launch_mlp_adam(float *P, float *m, float *v, const float *grad, int64_t step,
                            float lr, float b1, float b2, float eps, void *packed,
                            cudaStream_t st);

// stateless operators (caller memory)
cudaError_t launch_interp_dense(const Geometry &g, int delta, const float *U, int64_t n,
                                const double *x, float *u, cudaStream_t st);
cudaError_t launch_pack_vals(int64_t n, const float *v, float4 *vals, cudaStream_t st);
// *D = dd, with dd passed as a kernel parameter
cudaError_t launch_store_desc(const DomainDesc &dd, DomainDesc *D, cudaStream_t st);
cudaError_t launch_slots_to_dense(const Geometry &g, const BrickMap &m, const float *Gs,
                                  float *F, cudaStream_t st);
cudaError_t launch_pack_points(int64_t n, const float4 *a, float *out, cudaStream_t st);
cudaError_t launch_copy_f64(int64_t n, const double *a, double *out, cudaStream_t st);

}  // namespace lbmibm
