// Immersed boundary kernels (Sec. 3, Alg. 1-2): rigid-body kinematics, point
// binning by 4x4x4 brick, interpolation of the fluid velocity onto the points
// and atomic-free spreading of the velocity correction back to the lattice.
//
// Spreading is a gather: each active brick collects the contributions of the
// points binned in its 27 neighbouring bricks in a fixed order (bins in
// z,y,x order, points in ascending index inside a bin), so the force field is
// bitwise reproducible run to run, unlike the atomicAdd scatter of Alg. 2.
#include "kernels.h"

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

// Per body, once per step: cos/sin of phi(t) = phase + omega t and the
// differences cos phi(t) - cos phi(t-1), sin phi(t) - sin phi(t-1), the latter
// without cancellation as -2 sin(phi - omega/2) sin(omega/2) and
// 2 cos(phi - omega/2) sin(omega/2).
__global__ void body_trig_kernel(Bodies bd, int64_t t) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bd.nb) return;
  const double om = bd.omega[b];
  const double phi = bd.phase[b] + om * (double)t;
  double sn, cs, sm, cm;
  sincos(phi, &sn, &cs);
  sincos(phi - 0.5 * om, &sm, &cm);
  const double sh = sin(0.5 * om);
  double *o = bd.trig + 4 * b;
  o[0] = cs;
  o[1] = sn;
  o[2] = -2.0 * sm * sh;
  o[3] = 2.0 * cm * sh;
}

__global__ void __launch_bounds__(256)
    prepare_points_kernel(Geometry g, int delta, PointsIn p, Bodies bd, int64_t t,
                          PointPrep pp, BrickMap m, double *__restrict__ xpos) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) m.counters[0] = 0;
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
  const int bin = ((bz >> 2) * g.nby + (by >> 2)) * g.nbx + (bx >> 2);
  pp.base[k] = make_int4(bx, by, bz, bin);
  pp.ut[k] = make_float4(u[0], u[1], u[2], p.area ? p.area[k] : 1.f);
  // bricks covered by the support floor(x)-1 .. floor(x)+2 (two per axis at most)
  const int xl = wrapi(bx - 1, g.nx) >> 2, xh = wrapi(bx + 2, g.nx) >> 2;
  const int yl = wrapi(by - 1, g.ny) >> 2, yh = wrapi(by + 2, g.ny) >> 2;
  const int zl = wrapi(bz - 1, g.nz) >> 2, zh = wrapi(bz + 2, g.nz) >> 2;
  const int zz[2] = {zl, zh}, yy[2] = {yl, yh}, xx[2] = {xl, xh};
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int c = 0; c < 2; c++) m.brick_flag[(zz[a] * g.nby + yy[b]) * g.nbx + xx[c]] = 1;
}

__global__ void compact_kernel(Geometry g, BrickMap m) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nbrick) return;
  if (m.brick_flag[b]) {
    m.brick_flag[b] = 0;
    const int s = atomicAdd(m.counters, 1);
    if (s < m.max_slots) {
      m.brick_slot[b] = s;
      m.slot_brick[s] = b;
      m.slot_count[s] = 0;
      m.slot_cursor[s] = 0;
    } else {
      m.brick_slot[b] = -1;
      atomicOr(m.counters + 1, 1);
    }
  } else {
    m.brick_slot[b] = -1;
  }
}

__global__ void bin_count_kernel(int64_t np, PointPrep pp, BrickMap m) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  atomicAdd(m.slot_count + m.brick_slot[pp.base[k].w], 1);
}

// Exclusive scan of slot_count[0 .. nslots) into slot_start, one block.
__global__ void __launch_bounds__(1024) bin_scan_kernel(BrickMap m) {
  __shared__ int wsum[32];
  const int n = m.counters[0] < m.max_slots ? m.counters[0] : m.max_slots;
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(lo + per, n);
  int local = 0;
  for (int i = lo; i < hi; i++) local += m.slot_count[i];
  // block exclusive scan of `local`
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
    m.slot_start[i] = run;
    run += m.slot_count[i];
  }
  if (threadIdx.x == 1023) m.slot_start[n] = run;
}

__global__ void bin_fill_kernel(int64_t np, PointPrep pp, BrickMap m) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int s = m.brick_slot[pp.base[k].w];
  const int pos = m.slot_start[s] + atomicAdd(m.slot_cursor + s, 1);
  pp.sorted[pos] = (int)k;
}

// ascending point index inside every bin (fixed summation order)
__global__ void bin_sort_kernel(PointPrep pp, BrickMap m) {
  const int n = m.counters[0] < m.max_slots ? m.counters[0] : m.max_slots;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int *a = pp.sorted + m.slot_start[s];
    const int c = m.slot_count[s];
    for (int i = 1; i < c; i++) {
      const int v = a[i];
      int j = i - 1;
      while (j >= 0 && a[j] > v) {
        a[j + 1] = a[j];
        j--;
      }
      a[j + 1] = v;
    }
  }
}

// Alg. 1 loop body: u(k) = sum over the 4x4x4 taps of (U0 + G)(X) w w w;
// g = u_k - u; du += s g.
__global__ void __launch_bounds__(128)
    interp_kernel(Geometry g, int64_t np, PointPrep pp, BrickMap m,
                  const float *__restrict__ U0s, const float *__restrict__ Gs,
                  float4 *__restrict__ du, float4 *__restrict__ uint, int first, int warm) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int k = pp.sorted[j];
  const int4 b = pp.base[k];
  const float4 *wp = (const float4 *)(pp.wts + 12 * (int64_t)k);
  const float4 w0 = wp[0], w1 = wp[1], w2 = wp[2];
  const float wx[4] = {w0.x, w0.y, w0.z, w0.w};
  const float wy[4] = {w1.x, w1.y, w1.z, w1.w};
  const float wz[4] = {w2.x, w2.y, w2.z, w2.w};
  int X[4], Y[4], Z[4];
#pragma unroll
  for (int a = 0; a < 4; a++) {
    X[a] = wrapi(b.x - 1 + a, g.nx);
    Y[a] = wrapi(b.y - 1 + a, g.ny);
    Z[a] = wrapi(b.z - 1 + a, g.nz);
  }
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int c = 0; c < 4; c++) {
#pragma unroll
    for (int bb = 0; bb < 4; bb++) {
      const int row = ((Z[c] >> 2) * g.nby + (Y[bb] >> 2)) * g.nbx;
      const int lrow = ((Z[c] & 3) * 4 + (Y[bb] & 3)) * 4;
      const float wyz = wy[bb] * wz[c];
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const int s = __ldg(m.brick_slot + row + (X[a] >> 2));
        const size_t o = (size_t)s * SLOT_FLOATS + lrow + (X[a] & 3);
        const float w = wx[a] * wyz;
        ax += w * (__ldg(U0s + o) + __ldg(Gs + o));
        ay += w * (__ldg(U0s + o + BRICK_CELLS) + __ldg(Gs + o + BRICK_CELLS));
        az += w * (__ldg(U0s + o + 2 * BRICK_CELLS) + __ldg(Gs + o + 2 * BRICK_CELLS));
      }
    }
  }
  const float4 ut = pp.ut[k];
  float4 d = (first && !warm) ? make_float4(0.f, 0.f, 0.f, 0.f) : du[k];
  d.x += ut.w * (ut.x - ax);
  d.y += ut.w * (ut.y - ay);
  d.z += ut.w * (ut.z - az);
  du[k] = d;
  uint[k] = make_float4(ax, ay, az, 0.f);
}

// G(X) = sum_k v(k) w w w over the points of the 27 neighbouring bins, for
// every cell of every active brick (one 64-thread block per brick, grid-stride
// over the active bricks).
//
// The candidates of the 27 bins are concatenated (exclusive scan of the bin
// counts) and staged in shared memory in chunks of SP_CHUNK, each with its
// brick-local weight vectors (zero where the cell is outside the point's
// support, periodic offsets resolved once per candidate).  The block splits
// into four groups of 16 threads; a thread owns one x-row of four cells and
// its group accumulates every fourth candidate.  The four partial sums are
// added in a fixed order, so the result does not depend on scheduling.
constexpr int SP_CHUNK = 128;

__global__ void __launch_bounds__(64)
    spread_kernel(Geometry g, PointPrep pp, BrickMap m, const float4 *__restrict__ vals,
                  float *__restrict__ Gs, float *__restrict__ res) {
  __shared__ float4 swx[SP_CHUNK];
  __shared__ float swy[SP_CHUNK][4], swz[SP_CHUNK][4];
  __shared__ float4 sv[SP_CHUNK];
  __shared__ int bstart[27], boff[28];
  __shared__ float sacc[4][3][64];
  __shared__ float sred[2];
  const int nslots = m.counters[0] < m.max_slots ? m.counters[0] : m.max_slots;
  const int t = threadIdx.x;
  const int grp = t >> 4, tg = t & 15, yl = tg & 3, zl = tg >> 2;
  for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
    const int B = m.slot_brick[s];
    const int bxb = B % g.nbx, rr = B / g.nbx;
    const int byb = rr % g.nby, bzb = rr / g.nby;
    const int X0 = bxb * 4, Y0 = byb * 4, Z0 = bzb * 4;
    if (t < 32) {
      int cnt = 0, st = 0;
      if (t < 27) {
        const int ix = t % 3, iy = (t / 3) % 3, iz = t / 9;
        // distinct neighbour bricks per axis: 3, or 2 / 1 when the axis has
        // only 2 / 1 bricks (periodic images coincide)
        const int cx = g.nbx >= 3 ? 3 : g.nbx, cy = g.nby >= 3 ? 3 : g.nby,
                  cz = g.nbz >= 3 ? 3 : g.nbz;
        if (ix < cx && iy < cy && iz < cz) {
          const int nbx_ = cx == 3 ? wrapi(bxb - 1 + ix, g.nbx) : (bxb ^ ix);
          const int nby_ = cy == 3 ? wrapi(byb - 1 + iy, g.nby) : (byb ^ iy);
          const int nbz_ = cz == 3 ? wrapi(bzb - 1 + iz, g.nbz) : (bzb ^ iz);
          const int ns = m.brick_slot[(nbz_ * g.nby + nby_) * g.nbx + nbx_];
          if (ns >= 0) {
            cnt = m.slot_count[ns];
            st = m.slot_start[ns];
          }
        }
      }
      int inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (t >= o) inc += v;
      }
      if (t < 27) {
        bstart[t] = st;
        boff[t] = inc - cnt;
      }
      if (t == 26) boff[27] = inc;
    }
    __syncthreads();
    const int C = boff[27];
    float acc[4][3];
#pragma unroll
    for (int a = 0; a < 4; a++) acc[a][0] = acc[a][1] = acc[a][2] = 0.f;
    for (int c0 = 0; c0 < C; c0 += SP_CHUNK) {
      for (int q = t; q < SP_CHUNK; q += 64) {
        const int cand = c0 + q;
        if (cand < C) {
          int j = 0;
          while (boff[j + 1] <= cand) j++;
          const int k = pp.sorted[bstart[j] + cand - boff[j]];
          const int4 b = pp.base[k];
          const float4 *wp = (const float4 *)(pp.wts + 12 * (int64_t)k);
          const float4 w0 = wp[0], w1 = wp[1], w2 = wp[2];
          const float wx[4] = {w0.x, w0.y, w0.z, w0.w};
          const float wy[4] = {w1.x, w1.y, w1.z, w1.w};
          const float wz[4] = {w2.x, w2.y, w2.z, w2.w};
          float lx[4], ly[4], lz[4];
#pragma unroll
          for (int c = 0; c < 4; c++) {
            // tap index of brick cell c along each axis (periodic), or outside
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
          swx[q] = make_float4(lx[0], lx[1], lx[2], lx[3]);
#pragma unroll
          for (int c = 0; c < 4; c++) {
            swy[q][c] = ly[c];
            swz[q][c] = lz[c];
          }
          sv[q] = vals[k];
        }
      }
      __syncthreads();
      const int mm = min(SP_CHUNK, C - c0);
      for (int j = grp; j < mm; j += 4) {
        const float wyz = swy[j][yl] * swz[j][zl];
        const float4 wx = swx[j];
        const float4 v = sv[j];
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
      for (int c = 0; c < 3; c++) sacc[grp][c][row + a] = acc[a][c];
    __syncthreads();
    // cell t: the four group sums in a fixed order
    const float ax = ((sacc[0][0][t] + sacc[1][0][t]) + sacc[2][0][t]) + sacc[3][0][t];
    const float ay = ((sacc[0][1][t] + sacc[1][1][t]) + sacc[2][1][t]) + sacc[3][1][t];
    const float az = ((sacc[0][2][t] + sacc[1][2][t]) + sacc[2][2][t]) + sacc[3][2][t];
    float *G = Gs + (size_t)s * SLOT_FLOATS + t;
    if (res) {
      const float dx = ax - G[0], dy = ay - G[BRICK_CELLS], dz = az - G[2 * BRICK_CELLS];
      float r = dx * dx + dy * dy + dz * dz;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      if ((t & 31) == 0) sred[t >> 5] = r;
    }
    G[0] = ax;
    G[BRICK_CELLS] = ay;
    G[2 * BRICK_CELLS] = az;
    __syncthreads();
    if (res && t == 0) res[s] = sred[0] + sred[1];
  }
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
  const int nslots = m.counters[0] < m.max_slots ? m.counters[0] : m.max_slots;
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

}  // namespace

constexpr int PERSISTENT_BLOCKS = 152 * 16;

cudaError_t launch_prepare_points(const Geometry &g, int delta, const PointsIn &p,
                                  const Bodies &b, int64_t t, PointPrep &pp,
                                  const BrickMap &m, double *xpos, cudaStream_t st) {
  if (p.np <= 0) return cudaSuccess;
  if (b.nb > 0) body_trig_kernel<<<nblk(b.nb, 128), 128, 0, st>>>(b, t);
  prepare_points_kernel<<<nblk(p.np, 256), 256, 0, st>>>(g, delta, p, b, t, pp, m, xpos);
  return cudaGetLastError();
}

cudaError_t launch_build_bins(const Geometry &g, int64_t np, const PointPrep &pp,
                              const BrickMap &m, cudaStream_t st, int *nlaunch) {
  compact_kernel<<<nblk(g.nbrick, 256), 256, 0, st>>>(g, m);
  if (np > 0) {
    bin_count_kernel<<<nblk(np, 256), 256, 0, st>>>(np, pp, m);
    bin_scan_kernel<<<1, 1024, 0, st>>>(m);
    bin_fill_kernel<<<nblk(np, 256), 256, 0, st>>>(np, pp, m);
    bin_sort_kernel<<<152 * 2, 128, 0, st>>>(pp, m);
    if (nlaunch) *nlaunch += 5;
  } else if (nlaunch) {
    *nlaunch += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_interp(const Geometry &g, int64_t np, const PointPrep &pp,
                          const BrickMap &m, const float *U0s, const float *Gs, float4 *du,
                          float4 *uint, int first, int warm, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  interp_kernel<<<nblk(np, 128), 128, 0, st>>>(g, np, pp, m, U0s, Gs, du, uint, first, warm);
  return cudaGetLastError();
}

cudaError_t launch_spread(const Geometry &g, const PointPrep &pp, const BrickMap &m,
                          const float4 *vals, float *Gs, float *res, cudaStream_t st) {
  spread_kernel<<<PERSISTENT_BLOCKS, 64, 0, st>>>(g, pp, m, vals, Gs, res);
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
