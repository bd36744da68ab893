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
// rho, U0 on the cells of every active brick (pull of Eq. 4 + Eq. 1); G = 0.
cudaError_t launch_moments_slots(int storage, const Geometry &g, const void *f,
                                 const BrickMap &m, float *U0s, float *Gs, cudaStream_t st);
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
                                  const BrickMap &m, double *xpos, cudaStream_t st);
// flags -> slots, bins of points by brick (deterministic order in each bin)
cudaError_t launch_build_bins(const Geometry &g, int64_t np, const PointPrep &pp,
                              const BrickMap &m, cudaStream_t st, int *nlaunch);
// One fixed-point interpolation (Alg. 1): u = I[U0 + G]; g = u_k - u;
// du += s g (du starts at 0 when first && !warm).
cudaError_t launch_interp(const Geometry &g, int64_t np, const PointPrep &pp,
                          const BrickMap &m, const float *U0s, const float *Gs, float4 *du,
                          float4 *uint, int first, int warm, cudaStream_t st);
// G = S[du] over every active brick, gathered from neighbouring bins
// (Alg. 2 without atomics); res[slot] = sum (G_new - G_old)^2 (NULL: skip).
cudaError_t launch_spread(const Geometry &g, const PointPrep &pp, const BrickMap &m,
                          const float4 *vals, float *Gs, float *res, cudaStream_t st);
// stateless operators (caller memory)
cudaError_t launch_interp_dense(const Geometry &g, int delta, const float *U, int64_t n,
                                const double *x, float *u, cudaStream_t st);
cudaError_t launch_pack_vals(int64_t n, const float *v, float4 *vals, cudaStream_t st);
cudaError_t launch_slots_to_dense(const Geometry &g, const BrickMap &m, const float *Gs,
                                  float *F, cudaStream_t st);
cudaError_t launch_pack_points(int64_t n, const float4 *a, float *out, cudaStream_t st);

}  // namespace lbmibm
