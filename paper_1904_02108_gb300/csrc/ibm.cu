// Immersed boundary kernels (Sec. 3, Alg. 1-2): rigid-body kinematics, the
// (brick, point) pair lists, and the fixed-point loop.
//
// Once per step (points do not move inside the fixed point):
//   prepare_points  x(t) = M(t)[x_rest, 1], u_k, tap weights, brick flags
//   compact         flagged bricks -> slots of the sparse force storage
//   pair_count/scan/fill/sort
//                   one pair per (brick, point) with the point's support
//                   overlapping the brick, grouped by brick, ascending point
//                   index, with the brick-local weights of the point
//   brick_init      rho, U0 on the brick's cells (Eq. 1), G = 0 (or S[du_init])
//                   and each pair's share of I[U0 + G]
// Each iteration:
//   point_update    u_n(k) = sum of the point's pair shares; g = u_k - u_n;
//                   du += s g                                   (Alg. 1)
//   brick_spread    G = S[du] over the brick, gathered from its pairs (Alg. 2
//                   without atomics), then each pair's share of I[U0 + G]
//
// Every sum runs in a fixed order (pairs ascending inside a brick, four
// partial sums combined in a fixed order, a point's shares in brick order), so
// results are bitwise reproducible, unlike the atomicAdd scatter of Alg. 2.
#include "kernels.h"
#include "lattice.cuh"

namespace lbmibm {

namespace {

// Tap weights for taps floor(x)-1 .. floor(x)+2 of a point with fractional
// offset f in [0, 1]: distances 1+f, f, 1-f, 2-f.
//  cosine: w(r) = (1 + cos(pi r / 2)) / 4  ->  ((1-s), (1+c), (1+s), (1-c)) / 4
//          with s = sin(pi f / 2), c = cos(pi f / 2);
//  Peskin: with q = sqrt(1 + 4 f (1 - f)) the four distances give
//          ((3-2f-q), (3-2f+q), (1+2f+q), (1+2f-q)) / 8.
__device__ __forceinline__ void tap_weights(int delta, float f, float w[4]) {
  if (delta == 0) {
    float s, c;
    sincospif(0.5f * f, &s, &c);
    w[0] = 0.25f * (1.f - s);
    w[1] = 0.25f * (1.f + c);
    w[2] = 0.25f * (1.f + s);
    w[3] = 0.25f * (1.f - c);
  } else {
    const float q = sqrtf(1.f + 4.f * f * (1.f - f));
    w[0] = 0.125f * (3.f - 2.f * f - q);
    w[1] = 0.125f * (3.f - 2.f * f + q);
    w[2] = 0.125f * (1.f + 2.f * f + q);
    w[3] = 0.125f * (1.f + 2.f * f - q);
  }
}

__device__ __forceinline__ int base_and_frac(double x, int n, float &f) {
  const double fl = floor(x);
  f = (float)(x - fl);
  int b = (int)(fl - n * floor(fl / n));  // wrap into [0, n)
  if (b >= n) b -= n;
  if (b < 0) b += n;
  return b;
}

// Bricks holding the support floor(x)-1 .. floor(x)+2 along one axis: the
// brick of the lowest and of the highest tap (equal when the support lies in
// one brick).
struct SupportBricks {
  int lo, hi;
};
__device__ __forceinline__ SupportBricks support_bricks(int b, int n) {
  return {wrapi(b - 1, n) >> 2, wrapi(b + 2, n) >> 2};
}

// Per body, once per step: cos/sin of phi(t) = phase + omega t and the
// differences cos phi(t) - cos phi(t-1), sin phi(t) - sin phi(t-1), the latter
// without cancellation as -2 sin(phi - omega/2) sin(omega/2) and
// 2 cos(phi - omega/2) sin(omega/2).
__global__ void body_trig_kernel(Bodies bd, int64_t t) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bd.nb) return;
  const double om = bd.omega[b];
  const double phi = bd.phase[b] + om * (double)t;
  double sn, cs, sh, ch;
  sincos(phi, &sn, &cs);
  sincos(0.5 * om, &sh, &ch);
  // phi - omega/2 by the angle-difference formulas
  const double sm = sn * ch - cs * sh, cm = cs * ch + sn * sh;
  double *o = bd.trig + 4 * b;
  o[0] = cs;
  o[1] = sn;
  o[2] = -2.0 * sm * sh;
  o[3] = 2.0 * cm * sh;
}

__global__ void __launch_bounds__(256)
    prepare_points_kernel(Geometry g, int delta, PointsIn p, Bodies bd, int64_t t,
                          PointPrep pp, BrickMap m, PairMap pm, double *__restrict__ xpos) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    m.counters[0] = 0;
    m.counters[1] = 0;
  }
  if (k >= p.np) return;
  double x[3];
  float u[3];
  const double *X = p.X + 3 * k;
  if (bd.nb > 0) {
    // Alg. 1, first iteration: x(t) = M(t) [x_rest, 1], u_k = x(t) - x(t-1)
    const int b = p.body ? p.body[k] : 0;
    const double *c = bd.centre + 3 * b;
    const double2 t0 = *(const double2 *)(bd.trig + 4 * b);
    const double2 t1 = *(const double2 *)(bd.trig + 4 * b + 2);
    const double cs = t0.x, sn = t0.y, dc = t1.x, ds = t1.y;
    const double rx = X[0] - c[0], ry = X[1] - c[1], rz = X[2] - c[2];
    x[0] = c[0] + (cs * rx - sn * ry);
    x[1] = c[1] + (sn * rx + cs * ry);
    x[2] = c[2] + rz;
    // u_k = (R(phi) - R(phi - omega)) r
    u[0] = (float)(dc * rx - ds * ry);
    u[1] = (float)(ds * rx + dc * ry);
    u[2] = 0.f;
  } else {
    x[0] = X[0];
    x[1] = X[1];
    x[2] = X[2];
    u[0] = p.utarget ? p.utarget[3 * k] : 0.f;
    u[1] = p.utarget ? p.utarget[3 * k + 1] : 0.f;
    u[2] = p.utarget ? p.utarget[3 * k + 2] : 0.f;
  }
  if (xpos) {
    xpos[3 * k] = x[0];
    xpos[3 * k + 1] = x[1];
    xpos[3 * k + 2] = x[2];
  }
  float fx, fy, fz;
  const int bx = base_and_frac(x[0], g.nx, fx);
  const int by = base_and_frac(x[1], g.ny, fy);
  const int bz = base_and_frac(x[2], g.nz, fz);
  float w[12];
  tap_weights(delta, fx, w);
  tap_weights(delta, fy, w + 4);
  tap_weights(delta, fz, w + 8);
  float4 *wo = (float4 *)(pp.wts + 12 * k);
  wo[0] = make_float4(w[0], w[1], w[2], w[3]);
  wo[1] = make_float4(w[4], w[5], w[6], w[7]);
  wo[2] = make_float4(w[8], w[9], w[10], w[11]);
  pp.base[k] = make_int4(bx, by, bz, 0);
  pp.ut[k] = make_float4(u[0], u[1], u[2], p.area ? p.area[k] : 1.f);
  int4 *pk = (int4 *)(pm.point_pairs + 8 * k);
  pk[0] = make_int4(-1, -1, -1, -1);
  pk[1] = make_int4(-1, -1, -1, -1);
  // bricks covered by the support (at most two per axis)
  const SupportBricks sx = support_bricks(bx, g.nx), sy = support_bricks(by, g.ny),
                      sz = support_bricks(bz, g.nz);
  const int zz[2] = {sz.lo, sz.hi}, yy[2] = {sy.lo, sy.hi}, xx[2] = {sx.lo, sx.hi};
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int c = 0; c < 2; c++) m.brick_flag[(zz[a] * g.nby + yy[b]) * g.nbx + xx[c]] = 1;
}

__global__ void compact_kernel(Geometry g, BrickMap m, PairMap pm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbrick) return;
  if (m.brick_flag[b]) {
    m.brick_flag[b] = 0;
    const int s = atomicAdd(m.counters, 1);
    if (s < m.max_slots) {
      m.brick_slot[b] = s;
      m.slot_brick[s] = b;
      pm.count[s] = 0;
      pm.cursor[s] = 0;
    } else {
      m.brick_slot[b] = -1;
      atomicOr(m.counters + 1, 1);
    }
  } else {
    m.brick_slot[b] = -1;
  }
}

__device__ __forceinline__ int active_slots(const BrickMap &m) {
  const int n = m.counters[0];
  return n < m.max_slots ? n : m.max_slots;
}

// Calls fn(brick) for each distinct brick of a point's support.
template <typename Fn>
__device__ __forceinline__ void for_support_bricks(const Geometry &g, int4 b, Fn fn) {
  const SupportBricks sx = support_bricks(b.x, g.nx), sy = support_bricks(b.y, g.ny),
                      sz = support_bricks(b.z, g.nz);
  const int nzb = sz.hi != sz.lo ? 2 : 1, nyb = sy.hi != sy.lo ? 2 : 1,
            nxb = sx.hi != sx.lo ? 2 : 1;
  for (int c = 0; c < nzb; c++)
    for (int a = 0; a < nyb; a++)
      for (int e = 0; e < nxb; e++)
        fn(((c ? sz.hi : sz.lo) * g.nby + (a ? sy.hi : sy.lo)) * g.nbx + (e ? sx.hi : sx.lo));
}

__global__ void pair_count_kernel(Geometry g, int64_t np, PointPrep pp, BrickMap m,
                                  PairMap pm) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  for_support_bricks(g, pp.base[k], [&](int brick) {
    const int s = m.brick_slot[brick];
    if (s >= 0) atomicAdd(pm.count + s, 1);
  });
}

// Exclusive scan of pm.count[0 .. nslots) into pm.start, one block.
__global__ void __launch_bounds__(1024) pair_scan_kernel(BrickMap m, PairMap pm) {
  __shared__ int wsum[32];
  const int n = active_slots(m);
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(lo + per, n);
  int local = 0;
  for (int i = lo; i < hi; i++) local += pm.count[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int v = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  int run = v - local + (w > 0 ? wsum[w - 1] : 0);
  for (int i = lo; i < hi; i++) {
    pm.start[i] = run;
    run += pm.count[i];
  }
  if (threadIdx.x == 1023) pm.start[n] = run;
}

__global__ void pair_fill_kernel(Geometry g, int64_t np, PointPrep pp, BrickMap m, PairMap pm) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  for_support_bricks(g, pp.base[k], [&](int brick) {
    const int s = m.brick_slot[brick];
    if (s >= 0) pm.k[pm.start[s] + atomicAdd(pm.cursor + s, 1)] = (int)k;
  });
}

// One warp per slot: sort the slot's points ascending (rank sort; the points
// of a slot are distinct), then write each pair's brick-local weights and
// register the pair with its point.
constexpr int SORT_CAP = 1024;

__global__ void __launch_bounds__(128)
    pair_sort_kernel(Geometry g, PointPrep pp, BrickMap m, PairMap pm) {
  __shared__ int buf[4][SORT_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nslots = active_slots(m);
  for (int s = blockIdx.x * 4 + w; s < nslots; s += gridDim.x * 4) {
    const int cnt = pm.count[s], st = pm.start[s];
    int *a = pm.k + st;
    // scratch copy: shared memory, or this slot's (not yet written) weights
    int *tmp = cnt <= SORT_CAP ? buf[w] : (int *)(pm.w + 3 * (size_t)st);
    for (int i = lane; i < cnt; i += 32) tmp[i] = a[i];
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const int v = tmp[i];
      int r = 0;
      for (int j = 0; j < cnt; j++) r += tmp[j] < v;
      a[r] = v;
    }
    __syncwarp();
    const int B = m.slot_brick[s];
    const int bxb = B % g.nbx, rr = B / g.nbx;
    const int byb = rr % g.nby, bzb = rr / g.nby;
    const int X0 = bxb * 4, Y0 = byb * 4, Z0 = bzb * 4;
    for (int i = lane; i < cnt; i += 32) {
      const int k = a[i];
      const int4 b = pp.base[k];
      const float4 *wp = (const float4 *)(pp.wts + 12 * (int64_t)k);
      const float4 w0 = wp[0], w1 = wp[1], w2 = wp[2];
      const float wx[4] = {w0.x, w0.y, w0.z, w0.w};
      const float wy[4] = {w1.x, w1.y, w1.z, w1.w};
      const float wz[4] = {w2.x, w2.y, w2.z, w2.w};
      float lx[4], ly[4], lz[4];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        // tap index of the brick's cell c along each axis (periodic), or none
        int dx = X0 + c - b.x + 1;
        dx = dx < 0 ? dx + g.nx : (dx >= g.nx ? dx - g.nx : dx);
        int dy = Y0 + c - b.y + 1;
        dy = dy < 0 ? dy + g.ny : (dy >= g.ny ? dy - g.ny : dy);
        int dz = Z0 + c - b.z + 1;
        dz = dz < 0 ? dz + g.nz : (dz >= g.nz ? dz - g.nz : dz);
        float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
        for (int e = 0; e < 4; e++) {
          vx = dx == e ? wx[e] : vx;
          vy = dy == e ? wy[e] : vy;
          vz = dz == e ? wz[e] : vz;
        }
        lx[c] = vx;
        ly[c] = vy;
        lz[c] = vz;
      }
      const size_t p = (size_t)st + i;
      pm.w[3 * p] = make_float4(lx[0], lx[1], lx[2], lx[3]);
      pm.w[3 * p + 1] = make_float4(ly[0], ly[1], ly[2], ly[3]);
      pm.w[3 * p + 2] = make_float4(lz[0], lz[1], lz[2], lz[3]);
      const SupportBricks sx = support_bricks(b.x, g.nx), sy = support_bricks(b.y, g.ny),
                          sz = support_bricks(b.z, g.nz);
      const int j = (sx.hi != sx.lo && bxb == sx.hi ? 1 : 0) |
                    (sy.hi != sy.lo && byb == sy.hi ? 2 : 0) |
                    (sz.hi != sz.lo && bzb == sz.hi ? 4 : 0);
      pm.point_pairs[8 * (size_t)k + j] = (int)p;
    }
    __syncwarp();
  }
}

// ---- the brick kernels: one 64-thread block per active brick ----------------

constexpr int SP_CHUNK = 128;

struct BrickSmem {
  float4 swx[SP_CHUNK];
  float swy[SP_CHUNK][4], swz[SP_CHUNK][4];
  float4 sv[SP_CHUNK];
  float sacc[4][3][64];
  float4 sF[3][16];  // U0 + G of the brick, rows of four x cells
  float sred[2];
};

// G(X) = sum over the brick's pairs of v(k) wx wy wz, for the 64 cells of the
// brick.  The block splits into four groups of 16 threads; a thread owns one
// x-row of four cells, its group takes every fourth pair, and the four partial
// sums are added in a fixed order.  Thread t returns the sum of cell t.
__device__ __forceinline__ float3 brick_gather(BrickSmem &sm, const PairMap &pm, int p0, int cnt,
                                               const float4 *__restrict__ vals) {
  const int t = threadIdx.x;
  const int grp = t >> 4, tg = t & 15, yl = tg & 3, zl = tg >> 2;
  float acc[4][3];
#pragma unroll
  for (int a = 0; a < 4; a++) acc[a][0] = acc[a][1] = acc[a][2] = 0.f;
  for (int c0 = 0; c0 < cnt; c0 += SP_CHUNK) {
    for (int q = t; q < SP_CHUNK; q += 64) {
      if (c0 + q < cnt) {
        const size_t p = (size_t)p0 + c0 + q;
        const float4 wy = pm.w[3 * p + 1], wz = pm.w[3 * p + 2];
        sm.swx[q] = pm.w[3 * p];
        sm.swy[q][0] = wy.x;
        sm.swy[q][1] = wy.y;
        sm.swy[q][2] = wy.z;
        sm.swy[q][3] = wy.w;
        sm.swz[q][0] = wz.x;
        sm.swz[q][1] = wz.y;
        sm.swz[q][2] = wz.z;
        sm.swz[q][3] = wz.w;
        sm.sv[q] = vals[pm.k[p]];
      }
    }
    __syncthreads();
    const int mm = min(SP_CHUNK, cnt - c0);
    for (int j = grp; j < mm; j += 4) {
      const float wyz = sm.swy[j][yl] * sm.swz[j][zl];
      const float4 wx = sm.swx[j];
      const float4 v = sm.sv[j];
      const float w0 = wx.x * wyz, w1 = wx.y * wyz, w2 = wx.z * wyz, w3 = wx.w * wyz;
      acc[0][0] += w0 * v.x; acc[0][1] += w0 * v.y; acc[0][2] += w0 * v.z;
      acc[1][0] += w1 * v.x; acc[1][1] += w1 * v.y; acc[1][2] += w1 * v.z;
      acc[2][0] += w2 * v.x; acc[2][1] += w2 * v.y; acc[2][2] += w2 * v.z;
      acc[3][0] += w3 * v.x; acc[3][1] += w3 * v.y; acc[3][2] += w3 * v.z;
    }
    __syncthreads();
  }
  const int row = (zl * 4 + yl) * 4;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) sm.sacc[grp][c][row + a] = acc[a][c];
  __syncthreads();
  float3 r;
  r.x = ((sm.sacc[0][0][t] + sm.sacc[1][0][t]) + sm.sacc[2][0][t]) + sm.sacc[3][0][t];
  r.y = ((sm.sacc[0][1][t] + sm.sacc[1][1][t]) + sm.sacc[2][1][t]) + sm.sacc[3][1][t];
  r.z = ((sm.sacc[0][2][t] + sm.sacc[1][2][t]) + sm.sacc[2][2][t]) + sm.sacc[3][2][t];
  return r;
}

// Each pair's share of I[F] for F = sm.sF: sum over the brick's cells of
// F(X) wx wy wz (one thread per pair; every thread reads the same F row at the
// same time, a shared-memory broadcast).
__device__ __forceinline__ void brick_interp(BrickSmem &sm, const PairMap &pm, int p0,
                                             int cnt) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    // re-read F for every pair instead of holding all 192 values in registers
    asm volatile("" ::: "memory");
    const size_t p = (size_t)p0 + i;
    const float4 wx = pm.w[3 * p], wy4 = pm.w[3 * p + 1], wz4 = pm.w[3 * p + 2];
    const float wy[4] = {wy4.x, wy4.y, wy4.z, wy4.w};
    const float wz[4] = {wz4.x, wz4.y, wz4.z, wz4.w};
    float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
    for (int z = 0; z < 4; z++) {
#pragma unroll
      for (int y = 0; y < 4; y++) {
        const float wyz = wy[y] * wz[z];
        const float4 fx = sm.sF[0][z * 4 + y], fy = sm.sF[1][z * 4 + y],
                     fz = sm.sF[2][z * 4 + y];
        ax += wyz * (((wx.x * fx.x + wx.y * fx.y) + wx.z * fx.z) + wx.w * fx.w);
        ay += wyz * (((wx.x * fy.x + wx.y * fy.y) + wx.z * fy.z) + wx.w * fy.w);
        az += wyz * (((wx.x * fz.x + wx.y * fz.y) + wx.z * fz.z) + wx.w * fz.w);
      }
    }
    pm.part[p] = make_float4(ax, ay, az, 0.f);
  }
}

__device__ __forceinline__ void store_F(BrickSmem &sm, float fx, float fy, float fz) {
  const int t = threadIdx.x;
  ((float *)sm.sF[0])[t] = fx;
  ((float *)sm.sF[1])[t] = fy;
  ((float *)sm.sF[2])[t] = fz;
}

// First pass of a step over each active brick: U0 from the populations
// (pull + Eq. 1), G_0 = 0 or S[du_init] (warm start), and the pairs' shares of
// I[U0 + G_0] for the first iteration.
template <typename S>
__global__ void __launch_bounds__(64, 16)
    brick_init_kernel(const S *__restrict__ f, Geometry g, BrickMap m, PairMap pm,
                      const float4 *__restrict__ du_init, float *__restrict__ U0s,
                      float *__restrict__ Gs) {
  __shared__ BrickSmem sm;
  const int nslots = active_slots(m);
  const int t = threadIdx.x;
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int B = m.slot_brick[s];
    const int bx = B % g.nbx, rr = B / g.nbx;
    const int by = rr % g.nby, bz = rr / g.nby;
    const int x = bx * 4 + (t & 3), y = by * 4 + ((t >> 2) & 3), z = bz * 4 + (t >> 4);
    float d[Q];
    pull<S>(f, g, x, y, z, d);
    float drho, jx, jy, jz;
    moments(d, drho, jx, jy, jz);
    const float inv = 1.f / (1.f + drho);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    float *u = U0s + (size_t)s * SLOT_FLOATS + t;
    u[0] = ux;
    u[BRICK_CELLS] = uy;
    u[2 * BRICK_CELLS] = uz;
    const int p0 = pm.start[s], cnt = pm.count[s];
    float3 G = make_float3(0.f, 0.f, 0.f);
    if (du_init) G = brick_gather(sm, pm, p0, cnt, du_init);
    float *Gp = Gs + (size_t)s * SLOT_FLOATS + t;
    Gp[0] = G.x;
    Gp[BRICK_CELLS] = G.y;
    Gp[2 * BRICK_CELLS] = G.z;
    store_F(sm, ux + G.x, uy + G.y, uz + G.z);
    __syncthreads();
    brick_interp(sm, pm, p0, cnt);
    __syncthreads();
  }
}

// One iteration's spreading over each active brick: G = S[du] (Alg. 2 as a
// gather), the squared change of G into res[slot] (if res), and, unless this
// is the last iteration, the pairs' shares of I[U0 + G] for the next one.
__global__ void __launch_bounds__(64, 16)
    brick_spread_kernel(BrickMap m, PairMap pm, const float4 *__restrict__ vals,
                        const float *__restrict__ U0s, float *__restrict__ Gs,
                        float *__restrict__ res, int do_interp) {
  __shared__ BrickSmem sm;
  const int nslots = active_slots(m);
  const int t = threadIdx.x;
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int p0 = pm.start[s], cnt = pm.count[s];
    const float3 G = brick_gather(sm, pm, p0, cnt, vals);
    float *Gp = Gs + (size_t)s * SLOT_FLOATS + t;
    if (res) {
      const float dx = G.x - Gp[0], dy = G.y - Gp[BRICK_CELLS], dz = G.z - Gp[2 * BRICK_CELLS];
      float r = dx * dx + dy * dy + dz * dz;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      if ((t & 31) == 0) sm.sred[t >> 5] = r;
    }
    Gp[0] = G.x;
    Gp[BRICK_CELLS] = G.y;
    Gp[2 * BRICK_CELLS] = G.z;
    if (do_interp) {
      const float *u = U0s + (size_t)s * SLOT_FLOATS + t;
      store_F(sm, u[0] + G.x, u[BRICK_CELLS] + G.y, u[2 * BRICK_CELLS] + G.z);
    }
    __syncthreads();
    if (res && t == 0) res[s] = sm.sred[0] + sm.sred[1];
    if (do_interp) brick_interp(sm, pm, p0, cnt);
    __syncthreads();
  }
}

// Alg. 1 loop body per point: u_n(k) = sum of its bricks' shares (brick order),
// g = u_k - u_n, du += s g (du starts at 0 when first && !warm).
__global__ void __launch_bounds__(256)
    point_update_kernel(int64_t np, PointPrep pp, PairMap pm, float4 *__restrict__ du,
                        float4 *__restrict__ uint, int first, int warm) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int4 *pk = (const int4 *)(pm.point_pairs + 8 * k);
  const int4 a = pk[0], b = pk[1];
  const int idx[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    if (idx[j] >= 0) {
      const float4 v = pm.part[idx[j]];
      ux += v.x;
      uy += v.y;
      uz += v.z;
    }
  }
  const float4 ut = pp.ut[k];
  float4 d = (first && !warm) ? make_float4(0.f, 0.f, 0.f, 0.f) : du[k];
  d.x += ut.w * (ut.x - ux);
  d.y += ut.w * (ut.y - uy);
  d.z += ut.w * (ut.z - uz);
  du[k] = d;
  uint[k] = make_float4(ux, uy, uz, 0.f);
}

__global__ void interp_dense_kernel(Geometry g, int delta, const float *__restrict__ U,
                                    int64_t n, const double *__restrict__ x,
                                    float *__restrict__ u) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float f[3], w[3][4];
  int b[3];
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; a++) {
    b[a] = base_and_frac(x[3 * k + a], dims[a], f[a]);
    tap_weights(delta, f[a], w[a]);
  }
  const size_t N = (size_t)g.ncell;
  float acc[3] = {0.f, 0.f, 0.f};
  for (int c = 0; c < 4; c++) {
    const int Z = wrapi(b[2] - 1 + c, g.nz);
    for (int bb = 0; bb < 4; bb++) {
      const int Y = wrapi(b[1] - 1 + bb, g.ny);
      const float wyz = w[1][bb] * w[2][c];
      for (int a = 0; a < 4; a++) {
        const int X = wrapi(b[0] - 1 + a, g.nx);
        const size_t o = ((size_t)Z * g.ny + Y) * g.nx + X;
        const float ww = w[0][a] * wyz;
        acc[0] += ww * U[o];
        acc[1] += ww * U[N + o];
        acc[2] += ww * U[2 * N + o];
      }
    }
  }
  u[3 * k] = acc[0];
  u[3 * k + 1] = acc[1];
  u[3 * k + 2] = acc[2];
}

__global__ void pack_vals_kernel(int64_t n, const float *__restrict__ v, float4 *__restrict__ o) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  o[k] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], 1.f);
}

__global__ void pack_points_kernel(int64_t n, const float4 *__restrict__ a, float *__restrict__ o) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float4 v = a[k];
  o[3 * k] = v.x;
  o[3 * k + 1] = v.y;
  o[3 * k + 2] = v.z;
}

__global__ void slots_to_dense_kernel(Geometry g, BrickMap m, const float *__restrict__ Gs,
                                      float *__restrict__ F) {
  const int nslots = active_slots(m);
  const int t = threadIdx.x;
  const size_t N = (size_t)g.ncell;
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int B = m.slot_brick[s];
    const int bxb = B % g.nbx, rr = B / g.nbx;
    const int byb = rr % g.nby, bzb = rr / g.nby;
    const int x = bxb * 4 + (t & 3), y = byb * 4 + ((t >> 2) & 3), z = bzb * 4 + (t >> 4);
    const size_t o = ((size_t)z * g.ny + y) * g.nx + x;
    const float *p = Gs + (size_t)s * SLOT_FLOATS + t;
    F[o] = p[0];
    F[N + o] = p[BRICK_CELLS];
    F[2 * N + o] = p[2 * BRICK_CELLS];
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename S>
cudaError_t brick_init_typed(const Geometry &g, const void *f, const BrickMap &m,
                             const PairMap &pm, const float4 *du_init, float *U0s, float *Gs,
                             cudaStream_t st) {
  brick_init_kernel<S><<<PERSISTENT_BLOCKS, 64, 0, st>>>((const S *)f, g, m, pm, du_init, U0s,
                                                         Gs);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prepare_points(const Geometry &g, int delta, const PointsIn &p,
                                  const Bodies &b, int64_t t, PointPrep &pp,
                                  const BrickMap &m, const PairMap &pm, double *xpos,
                                  cudaStream_t st) {
  if (p.np <= 0) return cudaSuccess;
  if (b.nb > 0) body_trig_kernel<<<nblk(b.nb, 128), 128, 0, st>>>(b, t);
  prepare_points_kernel<<<nblk(p.np, 256), 256, 0, st>>>(g, delta, p, b, t, pp, m, pm, xpos);
  return cudaGetLastError();
}

cudaError_t launch_build_pairs(const Geometry &g, int64_t np, const PointPrep &pp,
                               const BrickMap &m, const PairMap &pm, cudaStream_t st) {
  compact_kernel<<<nblk(g.nbrick, 256), 256, 0, st>>>(g, m, pm);
  if (np > 0) {
    pair_count_kernel<<<nblk(np, 256), 256, 0, st>>>(g, np, pp, m, pm);
    pair_scan_kernel<<<1, 1024, 0, st>>>(m, pm);
    pair_fill_kernel<<<nblk(np, 256), 256, 0, st>>>(g, np, pp, m, pm);
    pair_sort_kernel<<<PERSISTENT_BLOCKS / 8, 128, 0, st>>>(g, pp, m, pm);
  }
  return cudaGetLastError();
}

#define DISPATCH_STORAGE(storage, FN, ...)   \
  switch (storage) {                         \
    case 0:                                  \
      return FN<float>(__VA_ARGS__);         \
    case 1:                                  \
      return FN<__nv_bfloat16>(__VA_ARGS__); \
    case 2:                                  \
      return FN<__half>(__VA_ARGS__);        \
    default:                                 \
      return cudaErrorInvalidValue;          \
  }

cudaError_t launch_brick_init(int storage, const Geometry &g, const void *f, const BrickMap &m,
                              const PairMap &pm, const float4 *du_init, float *U0s, float *Gs,
                              cudaStream_t st) {
  DISPATCH_STORAGE(storage, brick_init_typed, g, f, m, pm, du_init, U0s, Gs, st);
}

cudaError_t launch_brick_spread(const BrickMap &m, const PairMap &pm, const float4 *vals,
                                const float *U0s, float *Gs, float *res, int do_interp,
                                cudaStream_t st) {
  brick_spread_kernel<<<PERSISTENT_BLOCKS, 64, 0, st>>>(m, pm, vals, U0s, Gs, res, do_interp);
  return cudaGetLastError();
}

cudaError_t launch_point_update(int64_t np, const PointPrep &pp, const PairMap &pm,
                                float4 *du, float4 *uint, int first, int warm,
                                cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  point_update_kernel<<<nblk(np, 256), 256, 0, st>>>(np, pp, pm, du, uint, first, warm);
  return cudaGetLastError();
}

cudaError_t launch_interp_dense(const Geometry &g, int delta, const float *U, int64_t n,
                                const double *x, float *u, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  interp_dense_kernel<<<nblk(n, 128), 128, 0, st>>>(g, delta, U, n, x, u);
  return cudaGetLastError();
}

cudaError_t launch_pack_vals(int64_t n, const float *v, float4 *vals, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pack_vals_kernel<<<nblk(n, 256), 256, 0, st>>>(n, v, vals);
  return cudaGetLastError();
}

cudaError_t launch_slots_to_dense(const Geometry &g, const BrickMap &m, const float *Gs,
                                  float *F, cudaStream_t st) {
  slots_to_dense_kernel<<<PERSISTENT_BLOCKS, 64, 0, st>>>(g, m, Gs, F);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(int64_t n, const float4 *a, float *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pack_points_kernel<<<nblk(n, 256), 256, 0, st>>>(n, a, out);
  return cudaGetLastError();
}

}  // namespace lbmibm
