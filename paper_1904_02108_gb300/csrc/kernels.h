// Host-side launchers of the device kernels (internal C++ interface between
// the C ABI in api.cu and the kernels in lbm.cu / ibm.cu).  Every launcher
// enqueues on `st` and returns the launch status; none synchronises.
#pragma once

#include "common.cuh"

namespace lbmibm {

// ----------------------------------------------------------------- lbm.cu
struct CollideArgs {
  const void *src;      // populations (storage type), [19][ncell]
  void *dst;
  const int *brick_slot;  // NULL: no IBM force
  const float *Gs;        // slot force storage
  float gbody[3];
  float tau;
  double *partial;        // per-block FP64 sums (4 per block) or NULL
};
int collide_blocks(const Geometry &g);
cudaError_t launch_collide_stream(int storage, const Geometry &g, const CollideArgs &a,
                                  cudaStream_t st);
// FP64 reduction of the collide partials into out[4] (mass dev, momentum);
// `scratch` holds nblocks_reduce*4 doubles, `ticket` one zeroed uint.
cudaError_t launch_stats_reduce(const double *partial, int nparts, double *scratch,
                                unsigned *ticket, double *out, double ncell,
                                cudaStream_t st);
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
  double *trig;          // [nb][4] scratch: cos phi, sin phi, and the
                         // differences to phi - omega (set per step)
};
struct PointsIn {
  int64_t np;
  const double *X;        // [np][3]
  const int *body;        // [np] or NULL
  const float *area;      // [np] or NULL (1)
  const float *utarget;   // [np][3] or NULL (0)
};
// Kinematics (Alg. 1, first iteration) + per-point weights + brick flags.
cudaError_t launch_prepare_points(const Geometry &g, int delta, const PointsIn &p,
                                  const Bodies &b, int64_t t, PointPrep &pp,
                                  const BrickMap &m, const PairMap &pm, double *xpos,
                                  cudaStream_t st);
// counted bricks -> slots; (brick, point) pairs grouped by brick in a fixed
// order, with brick-local weights (5 launches when np > 0, else 1)
cudaError_t launch_build_pairs(const Geometry &g, int64_t np, const PointPrep &pp,
                               const BrickMap &m, const PairMap &pm, cudaStream_t st);
// U0 on the active bricks (pull + Eq. 1)
cudaError_t launch_brick_moments(int storage, const Geometry &g, const void *f,
                                 const BrickMap &m, float *U0s, cudaStream_t st);
// G_0 = 0 or S[du_init], pair shares of I[U0 + G_0]
cudaError_t launch_brick_init(const BrickMap &m, const PairMap &pm, const float4 *du_init,
                              const float *U0s, float *Gs, cudaStream_t st);
// G = S[vals] on the active bricks (Alg. 2 as a gather); res[slot] = squared
// change of G (NULL: skip); pair shares of I[U0 + G] if do_interp
cudaError_t launch_brick_spread(const BrickMap &m, const PairMap &pm, const float4 *vals,
                                const float *U0s, float *Gs, float *res, int do_interp,
                                const IbmLoop &loop, cudaStream_t st);
// u_n(k) from the pair shares; g = u_k - u_n; du += s g (Alg. 1 loop body)
cudaError_t launch_point_update(int64_t np, const PointPrep &pp, const PairMap &pm,
                                float4 *du, float4 *uint, int first, int warm,
                                const IbmLoop &loop, cudaStream_t st);
// ||S[v]||^2 per brick into res (v scaled by .w if scale_by_w)
cudaError_t launch_brick_norm(const BrickMap &m, const PairMap &pm, const float4 *vals,
                              int scale_by_w, float *res, cudaStream_t st);
// residual denominators (mode 0: ||S[s u_k]||^2, mode 1: fallback) and the
// per-iteration convergence check of the tolerance mode
cudaError_t launch_ibm_den(const BrickMap &m, const float *res, IbmState *state, int mode,
                           cudaStream_t st);
cudaError_t launch_point_residual0(int64_t np, const PointPrep &pp, const PairMap &pm,
                                   float4 *out, cudaStream_t st);
cudaError_t launch_ibm_check(const BrickMap &m, const float *res, IbmState *state, int it,
                             double tol, int max_iter, cudaStream_t st);
// Per-point MLP features (16) of the learned warm start from the pair shares
// of I[U0] (brick_init without du_init), u_k, du_prev and the body-relative
// rest position; see api.cu for the list.
cudaError_t launch_mlp_features(const Geometry &g, int64_t np, const PointPrep &pp,
                                const PairMap &pm, const BrickMap &m, const float4 *du_prev,
                                const PointsIn &p, const Bodies &b, float *X, cudaStream_t st);
// training sample target T = (du - du_prev) / MLP_VSCALE, du_prev from X
cudaError_t launch_mlp_targets(int64_t np, const float *X, const float4 *du, float *T,
                               cudaStream_t st);

// ----------------------------------------------------------------- mlp.cu
size_t mlp_packed_bytes();
size_t mlp_train_smem_bytes();
size_t mlp_grad_scratch_floats(int64_t n);
cudaError_t launch_mlp_pack(const float *P, void *packed, cudaStream_t st);
// mode 0: Y[n][3] = MLP(X); mode 1: du[k] += scale * MLP(X)[k]
cudaError_t launch_mlp_forward(int64_t n, const float *X, const void *packed, float *Y,
                               float4 *du, float scale, int mode, cudaStream_t st);
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
cudaError_t launch_slots_to_dense(const Geometry &g, const BrickMap &m, const float *Gs,
                                  float *F, cudaStream_t st);
cudaError_t launch_pack_points(int64_t n, const float4 *a, float *out, cudaStream_t st);

}  // namespace lbmibm
