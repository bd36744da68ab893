// Immersed boundary kernels (Sec. 3, Alg. 1-2): rigid-body kinematics, the
// (brick, point) pair lists, and the fixed-point loop.
//
// Once per step (points do not move inside the fixed point):
//   prepare_points  x(t) = M(t)[x_rest, 1], u_k, tap weights, and for each
//                   brick its number of overlapping supports
//   compact         bricks with a count -> slots of the sparse force storage,
//                   in brick order, and each slot's first pair (one scan)
//   pair_fill/sort
//                   one pair per (brick, point) with the point's support
//                   overlapping the brick, grouped by brick, ascending point
//                   index, with the brick-local weights of the point
//   brick_moments   rho, U0 on the brick's cells (Eq. 1)
//   brick_init      G = 0 (or S[du_init]) and each pair's share of I[U0 + G]
// Each iteration:
//   point_update    u_n(k) = sum of the point's pair shares; g = u_k - u_n;
//                   du += s g                                   (Alg. 1)
//   brick_spread    G = S[du] over the brick, gathered from its pairs (Alg. 2
//                   without atomics), then each pair's share of I[U0 + G]
//
// Every sum runs in a fixed order (pairs ascending inside a brick, four
// partial sums combined in a fixed order, a point's shares in brick order), so
// results are bitwise reproducible, unlike the atomicAdd scatter of Alg. 2.
#include <algorithm>
#include <climits>

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
  int b = (int)fl % n;  // wrap into [0, n)
  return b < 0 ? b + n : b;
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

// Adds 1 to ctr[key] for every calling lane with `valid`; lanes of a warp with
// equal keys share one atomicAdd.  Returns the lane's slot among the
// increments of its key (the value its own atomicAdd would have returned,
// lanes taken in order).  Every active lane of the warp must call it.
__device__ __forceinline__ int aggregated_inc(int *ctr, int key, bool valid) {
  const unsigned grp = __match_any_sync(__activemask(), valid ? key : -1);
  int pos = 0;
  if (valid) {
    const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
    int old = 0;
    if (lane == leader) old = atomicAdd(ctr + key, __popc(grp));
    pos = __shfl_sync(grp, old, leader) + __popc(grp & ((1u << lane) - 1u));
  }
  return pos;
}

// Calls fn(brick, valid) eight times, once per (z, y, x) choice of low/high
// support brick; valid is false for repeats when the support lies in one
// brick along an axis.  The trip count is uniform, so warps stay converged.
template <typename Fn>
__device__ __forceinline__ void for_support_bricks8(const Geometry &g, int4 b, Fn fn) {
  const SupportBricks sx = support_bricks(b.x, g.nx), sy = support_bricks(b.y, g.ny),
                      sz = support_bricks(b.z, g.nz);
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int e = j & 1, a = (j >> 1) & 1, c = j >> 2;
    const bool valid = (!e || sx.hi != sx.lo) && (!a || sy.hi != sy.lo) && (!c || sz.hi != sz.lo);
    fn(((c ? sz.hi : sz.lo) * g.nby + (a ? sy.hi : sy.lo)) * g.nbx + (e ? sx.hi : sx.lo), valid);
  }
}

// cos phi, sin phi and the differences cos phi - cos(phi - omega),
// sin phi - sin(phi - omega) of a body with phi = phase + omega t, in FP64;
// the differences as -2 sin(phi - omega/2) sin(omega/2) and
// 2 cos(phi - omega/2) sin(omega/2), without cancellation.
struct Trig {
  double cs, sn, dc, ds;
};
__device__ __forceinline__ Trig body_trig(const Bodies &bd, int b, int64_t t) {
  const double om = bd.omega[b];
  const double phi = bd.phase[b] + om * (double)t;
  double sn, cs, sh, ch;
  sincos(phi, &sn, &cs);
  sincos(0.5 * om, &sh, &ch);
  // phi - omega/2 by the angle-difference formulas
  const double sm = sn * ch - cs * sh, cm = cs * ch + sn * sh;
  return {cs, sn, -2.0 * sm * sh, 2.0 * cm * sh};
}

// Bodies whose rotation a block of prepare_points computes once in shared
// memory (the points of a block are consecutive and belong to few bodies);
// a block whose points span more takes them per point.
constexpr int TRIG_CACHE = 16;

// Xsrc / Usrc (single lattice, else NULL): new positions / targets read
// from device-mapped host memory by this step and written through to the
// domain's X / utarget (an upload that needs no copy of its own).  The step
// whose kinematics to compute: t_step >= 0 (given when the step is prepared
// while the one before it, which advances the device's counter at its end,
// still runs), -1 the device's counter t[0], -2 one after the step the last
// prepare_points computed (t[1]: a step prepared inside a captured graph,
// whose index is not known on the host).  A launch in the first two forms
// records its step in t[1] (a domain with a counter).
__global__ void __launch_bounds__(512, 2)
    prepare_points_kernel(const DomainDesc *__restrict__ D, const double *__restrict__ Xsrc,
                          const float *__restrict__ Usrc, long long t_step) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const Geometry g = d.g;
  const int delta = d.delta;
  const PointsIn p{d.np, d.X, d.body, d.area, d.utarget};
  const Bodies bd{d.centre, d.omega, d.phase, d.nb};
  const PointPrep pp = d.pp;
  const BrickMap m = d.m;
  const PairMap pm = d.pm;
  double *__restrict__ xpos = d.xpos;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && d.t && t_step != -2) d.t[1] = t_step >= 0 ? (int64_t)t_step : d.t[0];
  if (k == 0) {
    m.counters[0] = 0;
    m.counters[1] = 0;
#pragma unroll
    for (int q = 0; q < ORDER_BUCKETS; q++) m.counters[8 + q] = 0;
  }
  const bool in = k < p.np;
  const int body = (bd.nb > 0 && in) ? (p.body ? p.body[k] : 0) : -1;
  // the point's position first: its latency (host memory for a mapped
  // upload) overlaps the block's rotation set-up below
  double X[3] = {0.0, 0.0, 0.0};
  if (in) {
    const double *Xk = (Xsrc ? Xsrc : p.X) + 3 * k;
    X[0] = Xk[0];
    X[1] = Xk[1];
    X[2] = Xk[2];
  }
  __shared__ Trig strig[TRIG_CACHE];
  __shared__ int sb_lo, sb_hi;
  int b0 = 0, nbk = 0;
  int64_t tstep = 0;
  if (bd.nb > 0) {
    // the block's range of bodies, and their rotation once per block
    const int lo = __reduce_min_sync(0xffffffffu, in ? body : INT_MAX);
    const int hi = __reduce_max_sync(0xffffffffu, in ? body : -1);
    if (threadIdx.x == 0) {
      sb_lo = INT_MAX;
      sb_hi = -1;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&sb_lo, lo);
      atomicMax(&sb_hi, hi);
    }
    __syncthreads();
    b0 = sb_lo;
    nbk = sb_hi >= 0 ? sb_hi - sb_lo + 1 : 0;
    tstep = t_step >= 0 ? (int64_t)t_step : (t_step == -2 ? d.t[1] + 1 : d.t[0]);
    if (nbk <= TRIG_CACHE && (int)threadIdx.x < nbk)
      strig[threadIdx.x] = body_trig(bd, b0 + threadIdx.x, tstep);
    __syncthreads();
  }
  if (!in) return;
  double x[3];
  float u[3];
  // (write-through into the handle's own buffers, which a single lattice's
  // descriptor lists as read-only inputs of the step)
  if (Xsrc) {
    double *Xd = const_cast<double *>(d.X) + 3 * k;
    Xd[0] = X[0];
    Xd[1] = X[1];
    Xd[2] = X[2];
  }
  const float *ut = Usrc ? Usrc : p.utarget;
  if (Usrc) {
    float *Ud = const_cast<float *>(d.utarget) + 3 * k;
    Ud[0] = Usrc[3 * k];
    Ud[1] = Usrc[3 * k + 1];
    Ud[2] = Usrc[3 * k + 2];
  }
  if (bd.nb > 0) {
    // Alg. 1, first iteration: x(t) = M(t) [x_rest, 1], u_k = x(t) - x(t-1)
    const int b = body;
    const double *c = bd.centre + 3 * b;
    const Trig tr = nbk <= TRIG_CACHE ? strig[b - b0] : body_trig(bd, b, tstep);
    const double cs = tr.cs, sn = tr.sn, dc = tr.dc, ds = tr.ds;
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
    u[0] = ut ? ut[3 * k] : 0.f;
    u[1] = ut ? ut[3 * k + 1] : 0.f;
    u[2] = ut ? ut[3 * k + 2] : 0.f;
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
  // count this point in every distinct brick of its support
  for_support_bricks8(g, make_int4(bx, by, bz, 0), [&](int brick, bool valid) {
    aggregated_inc(m.brick_count, brick, valid);
  });
}

// Look-back word of a compaction tile: epoch (6 bits, never 0), status (2
// bits: 1 = the tile's own totals, 2 = inclusive prefix), active bricks (25
// bits), pairs (31 bits).
__device__ __forceinline__ unsigned long long tile_word(unsigned epoch, unsigned status,
                                                       unsigned long long a,
                                                       unsigned long long c) {
  return ((unsigned long long)epoch << 58) | ((unsigned long long)status << 56) | (a << 31) | c;
}

constexpr unsigned SCAN_SPIN_LIMIT = 1u << 22;

// The brick kernels take the active bricks by pair count, the longest first:
// bucket q of a brick with c pairs is 0 above 96, 1 above 64, 2 above 32, 3
// otherwise.
__device__ __forceinline__ int order_bucket(int c) {
  return c > 96 ? 0 : (c > 64 ? 1 : (c > 32 ? 2 : 3));
}

// Bricks with a count -> slots in brick order, and each slot's first pair:
// one pass over the bricks in tiles of COMPACT_TILE with a single-pass scan.
// A tile takes its index from a ticket, so it only waits on tiles already
// running; it publishes its totals, then its first warp adds up its
// predecessors' words 32 at a time (stopping at the nearest inclusive prefix)
// and publishes its own prefix.
// Every wait is bounded: past SCAN_SPIN_LIMIT polls the tile sets error flag 4
// and the step's slots are left empty.
__global__ void __launch_bounds__(256) compact_kernel(const DomainDesc *__restrict__ D) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const Geometry g = d.g;
  const BrickMap m = d.m;
  const PairMap pm = d.pm;
  const int ntiles = (g.nbrick + COMPACT_TILE - 1) / COMPACT_TILE;
  if ((int)blockIdx.x >= ntiles) return;
  __shared__ int tile_s, wa[8], wc[8];
  __shared__ unsigned long long wq[8];
  __shared__ unsigned epoch_s;
  __shared__ long long pre_a, pre_c;
  __shared__ int pre_q[ORDER_BUCKETS];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) {
    tile_s = atomicAdd(m.counters + 3, 1);
    epoch_s = (unsigned)(*(volatile int *)(m.counters + 4)) % 63u + 1u;
  }
  __syncthreads();
  const int tile = tile_s;
  const unsigned epoch = epoch_s;
  const int b0 = tile * COMPACT_TILE + 4 * t;
  // nq: active bricks per order bucket, 16 bits each (at most 1024 a tile)
  int c[4], na = 0, nc = 0;
  unsigned long long nq = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    c[i] = b0 + i < g.nbrick ? m.brick_count[b0 + i] : 0;
    na += c[i] > 0;
    nc += c[i];
    if (c[i] > 0) nq += 1ull << (16 * order_bucket(c[i]));
  }
  // block-exclusive scan of (na, nc, nq)
  int ia = na, ic = nc;
  unsigned long long iq = nq;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ta = __shfl_up_sync(0xffffffffu, ia, o), tc = __shfl_up_sync(0xffffffffu, ic, o);
    const unsigned long long tq = __shfl_up_sync(0xffffffffu, iq, o);
    if (lane >= o) {
      ia += ta;
      ic += tc;
      iq += tq;
    }
  }
  if (lane == 31) {
    wa[w] = ia;
    wc[w] = ic;
    wq[w] = iq;
  }
  __syncthreads();
  int ba = 0, bc = 0, ta = 0, tc = 0;
  unsigned long long bq = 0, tq = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    if (k < w) {
      ba += wa[k];
      bc += wc[k];
      bq += wq[k];
    }
    ta += wa[k];
    tc += wc[k];
    tq += wq[k];
  }
  ia += ba - na;  // exclusive within the tile
  ic += bc - nc;
  iq += bq - nq;
  if (w == 0) {
    unsigned long long *tw = m.tiles;
    long long pa = 0, pc = 0;
    if (tile == 0) {
      if (lane == 0) atomicExch(tw + 0, tile_word(epoch, 2, (unsigned)ta, (unsigned)tc));
    } else {
      if (lane == 0) atomicExch(tw + tile, tile_word(epoch, 1, (unsigned)ta, (unsigned)tc));
      // look back 32 tiles at a time: lane l reads tile top - l (tiles before
      // 0 read as an empty inclusive prefix), waits until all 32 are
      // published, and the warp adds the words up to the nearest inclusive one
      bool ok = true;
      for (int top = tile - 1; top >= 0; top -= 32) {
        const int j = top - lane;
        unsigned long long v = 0;
        unsigned stt = 2;
        unsigned spins = 0;
        for (;;) {
          if (j >= 0) {
            v = *(volatile unsigned long long *)(tw + j);
            stt = (unsigned)(v >> 58) == epoch ? (unsigned)((v >> 56) & 3u) : 0u;
          }
          if (__all_sync(0xffffffffu, stt != 0)) break;
          if (++spins >= SCAN_SPIN_LIMIT) {
            ok = false;
            break;
          }
          __nanosleep(64);
        }
        if (!ok) break;
        const unsigned incl = __ballot_sync(0xffffffffu, stt == 2);
        const int stop = incl ? __ffs(incl) - 1 : 31;
        long long sa = 0, sc = 0;
        if (lane <= stop && j >= 0) {
          sa = (long long)((v >> 31) & 0x1ffffffull);
          sc = (long long)(v & 0x7fffffffull);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sa += __shfl_xor_sync(0xffffffffu, sa, o);
          sc += __shfl_xor_sync(0xffffffffu, sc, o);
        }
        pa += sa;
        pc += sc;
        if (incl) break;
      }
      if (!ok) {
        if (lane == 0) {
          atomicOr(m.counters + 1, 4);
          atomicOr(m.counters + 5, 4);  // kept until the host reads it
        }
        pa = 0;
        pc = 0;
      }
      if (lane == 0)
        atomicExch(tw + tile, tile_word(epoch, 2, (unsigned)(pa + ta), (unsigned)(pc + tc)));
    }
    if (lane == 0) {
      pre_a = pa;
      pre_c = pc;
    }
  } else if (w == 1 && lane < ORDER_BUCKETS) {
    // the tile's places in each bucket of order (beside warp 0's look-back)
    const int n = (int)((tq >> (16 * lane)) & 0xffffu);
    pre_q[lane] = n > 0 ? atomicAdd(m.counters + 8 + lane, n) : 0;
  }
  __syncthreads();
  int slot = (int)pre_a + ia, first = (int)pre_c + ic;
  int oq[ORDER_BUCKETS];
#pragma unroll
  for (int q = 0; q < ORDER_BUCKETS; q++) oq[q] = pre_q[q] + (int)((iq >> (16 * q)) & 0xffffu);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int b = b0 + i;
    if (b >= g.nbrick) break;
    if (c[i] > 0) {
      m.brick_count[b] = 0;
      if (slot < m.max_slots) {
        m.brick_slot[b] = slot;
        m.slot_brick[slot] = b;
        pm.count[slot] = c[i];
        pm.start[slot] = first;
        pm.cursor[slot] = 0;
        const int q = order_bucket(c[i]);
        int o = 0;
#pragma unroll
        for (int k = 0; k < ORDER_BUCKETS; k++) o = k == q ? oq[k] : o;
        m.order[(size_t)q * m.max_slots + o] = slot;
      } else {
        m.brick_slot[b] = -1;
        atomicOr(m.counters + 1, 1);
      }
      slot++;
      first += c[i];
#pragma unroll
      for (int q = 0; q < ORDER_BUCKETS; q++) oq[q] += q == order_bucket(c[i]);
    } else {
      m.brick_slot[b] = -1;
    }
  }
  if (tile == ntiles - 1 && t == 0) {
    const int total = (int)(pre_a + ta);
    m.counters[0] = total;
    // (a domain without points has no pair storage)
    if (d.np > 0 && total <= m.max_slots) pm.start[total] = (int)(pre_c + tc);
    m.counters[3] = 0;
    m.counters[4] = (int)(epoch % 63u);  // the next launch's epoch is this + 1
  }
}


__global__ void __launch_bounds__(512) pair_fill_kernel(const DomainDesc *__restrict__ D) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const Geometry g = d.g;
  const int64_t np = d.np;
  const PointPrep pp = d.pp;
  const BrickMap m = d.m;
  const PairMap pm = d.pm;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np || (m.counters[1] & 4)) return;
  // the point's (up to) eight slots and their first pairs, then every slot's
  // warp-aggregated increment issued before any result is used (one round
  // trip for the eight, not eight)
  int sl[8], first[8];
  int j = 0;
  for_support_bricks8(g, pp.base[k], [&](int brick, bool valid) {
    sl[j] = valid ? m.brick_slot[brick] : -1;
    j++;
  });
#pragma unroll
  for (int i = 0; i < 8; i++) first[i] = sl[i] >= 0 ? pm.start[sl[i]] : 0;
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  unsigned grp[8];
  int old[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    grp[i] = __match_any_sync(act, sl[i] >= 0 ? sl[i] : -1);
    old[i] = 0;
    if (sl[i] >= 0 && lane == __ffs(grp[i]) - 1)
      old[i] = atomicAdd(pm.cursor + sl[i], __popc(grp[i]));
  }
#pragma unroll
  for (int i = 0; i < 8; i++) {
    if (sl[i] >= 0) {
      const int pos = __shfl_sync(grp[i], old[i], __ffs(grp[i]) - 1) +
                      __popc(grp[i] & ((1u << lane) - 1u));
      pm.k[first[i] + pos] = (int)k;
    }
  }
}

// A point's base cell and tap weights, as prepare_points wrote them.
struct PointTaps {
  int4 base;
  float4 w0, w1, w2;  // tap weights along x, y, z
};
__device__ __forceinline__ PointTaps load_taps(const PointPrep &pp, int k) {
  const float4 *wp = (const float4 *)(pp.wts + 12 * (int64_t)k);
  return {pp.base[k], wp[0], wp[1], wp[2]};
}

// Pair p (point k with taps pt, brick B, after the sort): the brick-local
// weights of its point (the point's tap weights at the brick's cells 0..3
// along each axis, 0 outside the support, periodic offsets resolved) and the
// pair's entry in the point's list of bricks.
__device__ __forceinline__ void pair_weights(const Geometry &g, const PairMap &pm, int64_t p,
                                             int k, int B, const PointTaps &pt) {
  const int bxb = B % g.nbx, rr = B / g.nbx;
  const int byb = rr % g.nby, bzb = rr / g.nby;
  const int X0 = bxb * 4, Y0 = byb * 4, Z0 = bzb * 4;
  const int4 b = pt.base;
  const float wx[4] = {pt.w0.x, pt.w0.y, pt.w0.z, pt.w0.w};
  const float wy[4] = {pt.w1.x, pt.w1.y, pt.w1.z, pt.w1.w};
  const float wz[4] = {pt.w2.x, pt.w2.y, pt.w2.z, pt.w2.w};
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

// The b-th active slot in the order the brick kernels take them: bucket by
// bucket (m.counters[8 + q] slots in bucket q, at m.order[q * max_slots]);
// index order after a slot overflow (an error step).
__device__ __forceinline__ int slot_in_order(const BrickMap &m, int b) {
  if (m.counters[1] & 1) return b;
#pragma unroll
  for (int q = 0; q < ORDER_BUCKETS - 1; q++) {
    const int n = m.counters[8 + q];
    if (b < n) return m.order[(size_t)q * m.max_slots + b];
    b -= n;
  }
  return m.order[(size_t)(ORDER_BUCKETS - 1) * m.max_slots + b];
}

// The items of a per-brick kernel, item b from first by stride.  A batch with
// a work list (WL) takes the active slots of all its domains as one list, so
// an uneven batch keeps every block busy; otherwise the block's domain
// D[blockIdx.y].  ORDERED: in the order of pair counts, longest first (in a
// batch bucket-major: bucket q of domain d starts at off[q nd + d]); else in
// slot order, domain by domain (domain d starts at off[ORDER_BUCKETS nd + 1 +
// d]), which keeps neighbouring bricks together.  fn(domain, slot) for each
// item.
template <bool WL, bool ORDERED, typename Fn>
__device__ __forceinline__ void for_each_slot(const DomainDesc *__restrict__ D,
                                              const int *__restrict__ off, int nd, int first,
                                              int stride, Fn fn) {
  if constexpr (WL) {
    const int nb = ORDERED ? ORDER_BUCKETS * nd : nd;
    const int *o = ORDERED ? off : off + ORDER_BUCKETS * nd + 1;
    const int total = o[nb];
    for (int b = first; b < total; b += stride) {
      int lo = 0, hi = nb;  // o[lo] <= b < o[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (o[mid] <= b) lo = mid;
        else hi = mid;
      }
      const int q = ORDERED ? lo / nd : 0;
      const DomainDesc &d = D[lo - q * nd];
      const int local = b - o[lo];
      if (ORDERED && !(d.m.counters[1] & 1))
        fn(d, d.m.order[(size_t)q * d.m.max_slots + local]);
      else
        fn(d, local);
    }
  } else {
    const DomainDesc &d = D[blockIdx.y];
    const int n = active_slots(d.m);
    for (int b = first; b < n; b += stride) fn(d, ORDERED ? slot_in_order(d.m, b) : b);
  }
}

// The work list of a batch: off[q nd + d] = the items before bucket q of
// domain d (bucket-major), off[ORDER_BUCKETS nd] = all active slots; then, at
// off + ORDER_BUCKETS nd + 1, the same domain-major (nd + 1 entries).  A
// domain without points or whose compaction failed contributes none; one
// whose slots overflowed, all of them in the last bucket (index order).  One
// block.
__global__ void __launch_bounds__(1024)
    batch_worklist_kernel(const DomainDesc *__restrict__ D, int nd, int *__restrict__ off) {
  pdl_wait();
  __shared__ int wsum[32];
  __shared__ int carry;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) carry = 0;
  const int nb = ORDER_BUCKETS * nd;
  for (int i0 = 0; i0 < nb; i0 += 1024) {
    const int i = i0 + t;
    int c = 0;
    if (i < nb) {
      const int q = i / nd;
      const DomainDesc &d = D[i - q * nd];
      const int flags = d.np > 0 ? d.m.counters[1] : 4;
      if (!(flags & 4))
        c = (flags & 1) ? (q == ORDER_BUCKETS - 1 ? active_slots(d.m) : 0) : d.m.counters[8 + q];
    }
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int before = carry;
    for (int k = 0; k < w; k++) before += wsum[k];
    if (i < nb) off[i] = before + x - c;
    __syncthreads();
    if (t == 1023) carry = before + x;
    __syncthreads();
  }
  if (t == 0) off[nb] = carry;
  // domain-major: the domains' active slots in order
  int *od = off + nb + 1;
  __syncthreads();
  if (t == 0) carry = 0;
  for (int i0 = 0; i0 < nd; i0 += 1024) {
    const int i = i0 + t;
    int c = 0;
    if (i < nd) {
      const DomainDesc &d = D[i];
      c = (d.np > 0 && !(d.m.counters[1] & 4)) ? active_slots(d.m) : 0;
    }
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int before = carry;
    for (int k = 0; k < w; k++) before += wsum[k];
    if (i < nd) od[i] = before + x - c;
    __syncthreads();
    if (t == 1023) carry = before + x;
    __syncthreads();
  }
  if (t == 0) od[nd] = carry;
}

// One warp per slot: sort the slot's points ascending (a bitonic network in
// registers up to 128 pairs, in shared memory up to SORT_CAP, else a rank sort through
// this slot's not yet written weight storage; the points of a slot are
// distinct), then record with each pair its brick and brick-local weights.
constexpr int SORT_CAP = 512;

// Sort of a[0..cnt) ascending (cnt <= 32 NR, NR a power of two) in
// registers: lane holds entries lane + 32 i, i < NR, padded with INT_MAX, and
// a bitonic network runs over the 32 NR entries: exchanges between lanes by
// shuffles (distance j < 32), between a lane's registers otherwise.  Entry e
// keeps the smaller of itself and its partner e ^ j when it is the lower of
// the two in an ascending block (e & k == 0) or the upper one in a descending
// block.
template <int NR>
__device__ __forceinline__ void warp_bitonic_sort(int *a, int cnt, int lane) {
  int v[NR];
#pragma unroll
  for (int i = 0; i < NR; i++) v[i] = lane + 32 * i < cnt ? a[lane + 32 * i] : 0x7fffffff;
#pragma unroll
  for (int k = 2; k <= 32 * NR; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        // k >= 64: the direction depends on the register only
        const int jj = j >> 5;
#pragma unroll
        for (int i = 0; i < NR; i++) {
          if ((i & jj) == 0) {
            const bool up = ((32 * i) & k) == 0;
            const int x = v[i], y = v[i | jj];
            v[i] = up ? min(x, y) : max(x, y);
            v[i | jj] = up ? max(x, y) : min(x, y);
          }
        }
      } else {
        const bool lo = (lane & j) == 0;
#pragma unroll
        for (int i = 0; i < NR; i++) {
          const bool up = ((lane + 32 * i) & k) == 0;
          const int y = __shfl_xor_sync(0xffffffffu, v[i], j);
          v[i] = up == lo ? min(v[i], y) : max(v[i], y);
        }
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < NR; i++)
    if (lane + 32 * i < cnt) a[lane + 32 * i] = v[i];
}

template <bool WL>
__global__ void __launch_bounds__(128)
    pair_sort_kernel(const DomainDesc *__restrict__ D, const int *__restrict__ off, int nd) {
  pdl_wait();
  __shared__ int buf[4][SORT_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the longest lists first
  for_each_slot<WL, true>(D, off, nd, blockIdx.x * 4 + w, gridDim.x * 4, [&](const DomainDesc &d, int s) {
    const BrickMap &m = d.m;
    const PairMap &pm = d.pm;
    const PointPrep &pp = d.pp;
    const Geometry &g = d.g;
    const int cnt = pm.count[s], st = pm.start[s], B = m.slot_brick[s];
    int *a = pm.k + st;
    if (cnt <= 32) {
      warp_bitonic_sort<1>(a, cnt, lane);
    } else if (cnt <= 64) {
      warp_bitonic_sort<2>(a, cnt, lane);
    } else if (cnt <= 128) {
      warp_bitonic_sort<4>(a, cnt, lane);
    } else if (cnt <= SORT_CAP) {
      int n2 = 2;
      while (n2 < cnt) n2 <<= 1;
      int *b = buf[w];
      for (int i = lane; i < n2; i += 32) b[i] = i < cnt ? a[i] : 0x7fffffff;
      __syncwarp();
      for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < n2; i += 32) {
            const int l = i ^ j;
            if (l > i) {
              const int x = b[i], y = b[l];
              if ((x > y) == ((i & k) == 0)) {
                b[i] = y;
                b[l] = x;
              }
            }
          }
          __syncwarp();
        }
      }
      for (int i = lane; i < cnt; i += 32) a[i] = b[i];
    } else {
      int *tmp = (int *)(pm.w + 3 * (size_t)st);
      for (int i = lane; i < cnt; i += 32) tmp[i] = a[i];
      __syncwarp();
      for (int i = lane; i < cnt; i += 32) {
        const int v = tmp[i];
        int r = 0;
        for (int j = 0; j < cnt; j++) r += tmp[j] < v;
        a[r] = v;
      }
    }
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const int k = a[i];
      pm.brick[st + i] = B;
      pair_weights(g, pm, (int64_t)st + i, k, B, load_taps(pp, k));
    }
  });
}

// ---- the brick kernels: one warp per active brick ---------------------------

// Loads issued where they are written (inline PTX the compiler does not move
// past the branch on the stop flag that follows them): in tolerance mode a
// pass reads the flag beside its first loads, one round trip instead of two.
__device__ __forceinline__ int4 ld_early(const int4 *p) {
  int4 v;
  asm volatile("ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_early(const int *p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// the stop flag (written by an earlier kernel, read-only in this one)
__device__ __forceinline__ bool stopped(const DomainDesc &d, int tol_mode) {
  return tol_mode && ld_early(&d.state->done);
}

// A warp stages up to SP_CHUNK pairs of its brick at a time: their brick-local
// weights and spread values.  96 pairs (6.9 KB of shared memory per warp)
// hold all pairs of 97 % of the bricks of a dense propeller array and leave
// room for 28 warps per SM (128 pairs: 23; measured 1.2 % faster per step).
constexpr int SP_CHUNK = 96;

struct BrickSmem {
  float4 swx[SP_CHUNK];
  float swy[SP_CHUNK][4], swz[SP_CHUNK][4];
  float4 sv[SP_CHUNK];
  float4 sF[3][16];  // U0 + G of the brick, rows of four x cells
};

// G(X) = sum over the brick's pairs of v(k) wx wy wz (Alg. 2 as a gather),
// for the 64 cells of the brick.  Lane l owns row l & 15 (an x-line of four
// cells, row = z_local * 4 + y_local); the two half-warps take alternate pairs
// (every lane of a half reads the same pair: shared-memory broadcasts) and
// are added as h0 + h1 in both.  Returns the row's four cells per component;
// on return the first chunk's pairs are staged (all of them when cnt <=
// SP_CHUNK).
// Packed FP32x2 multiply and fma (each half rounds as the scalar operation).
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

__device__ __forceinline__ void brick_gather(BrickSmem &sm, const PairMap &pm, int p0, int cnt,
                                             const float4 *__restrict__ vals, float4 out[3],
                                             bool scale_by_w = false) {
  const int t = threadIdx.x & 31;
  const int grp = t >> 4, tg = t & 15, yl = tg & 3, zl = tg >> 2;
  // cells 0, 1 and 2, 3 of the row per component, as packed pairs
  float2 A01[3], A23[3];
#pragma unroll
  for (int c = 0; c < 3; c++) A01[c] = A23[c] = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < cnt; c0 += SP_CHUNK) {
    __syncwarp();
    for (int q = t; q < SP_CHUNK; q += 32) {
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
        float4 v = vals[pm.k[p]];
        if (scale_by_w) {
          v.x *= v.w;
          v.y *= v.w;
          v.z *= v.w;
        }
        sm.sv[q] = v;
      }
    }
    __syncwarp();
    const int mm = min(SP_CHUNK, cnt - c0);
    for (int j = grp; j < mm; j += 2) {
      const float wyz = sm.swy[j][yl] * sm.swz[j][zl];
      const float4 wx = sm.swx[j];
      const float4 v = sm.sv[j];
      const float2 yz = make_float2(wyz, wyz);
      const float2 w01 = mul2(make_float2(wx.x, wx.y), yz), w23 = mul2(make_float2(wx.z, wx.w), yz);
      const float vc[3] = {v.x, v.y, v.z};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float2 vv = make_float2(vc[c], vc[c]);
        A01[c] = fma2(w01, vv, A01[c]);
        A23[c] = fma2(w23, vv, A23[c]);
      }
    }
  }
  __syncwarp();
  float acc[4][3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[0][c] = A01[c].x;
    acc[1][c] = A01[c].y;
    acc[2][c] = A23[c].x;
    acc[3][c] = A23[c].y;
  }
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float o = __shfl_xor_sync(0xffffffffu, acc[a][c], 16);
      acc[a][c] = grp == 0 ? acc[a][c] + o : o + acc[a][c];
    }
  out[0] = make_float4(acc[0][0], acc[1][0], acc[2][0], acc[3][0]);
  out[1] = make_float4(acc[0][1], acc[1][1], acc[2][1], acc[3][1]);
  out[2] = make_float4(acc[0][2], acc[1][2], acc[2][2], acc[3][2]);
}

// Each pair's share of I[F] for F = sm.sF: sum over the brick's cells of
// F(X) wx wy wz (one lane per pair; every lane reads the same F row at the same
// time, a shared-memory broadcast).  staged: the pair weights are still in
// sm.swx/swy/swz (the gather staged them and cnt <= SP_CHUNK).
__device__ __forceinline__ void brick_interp(BrickSmem &sm, const PairMap &pm, int p0, int cnt,
                                             bool staged) {
  for (int i = threadIdx.x & 31; i < cnt; i += 32) {
    // re-read F for every pair instead of holding all 192 values in registers
    asm volatile("" ::: "memory");
    const size_t p = (size_t)p0 + i;
    float4 wx;
    float wy[4], wz[4];
    if (staged) {
      wx = sm.swx[i];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        wy[c] = sm.swy[i][c];
        wz[c] = sm.swz[i][c];
      }
    } else {
      wx = pm.w[3 * p];
      const float4 wy4 = pm.w[3 * p + 1], wz4 = pm.w[3 * p + 2];
      wy[0] = wy4.x; wy[1] = wy4.y; wy[2] = wy4.z; wy[3] = wy4.w;
      wz[0] = wz4.x; wz[1] = wz4.y; wz[2] = wz4.z; wz[3] = wz4.w;
    }
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

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// U0 on every cell of every active brick: pull of Eq. 4 and Eq. 1 (the
// paper's kernel strategy of Sec. 5 without duplicated cells).  One thread per
// cell, 64 threads per brick, blockDim.x / 64 bricks per block.
template <typename S, bool WL>
__global__ void __launch_bounds__(256)
    brick_moments_kernel(const DomainDesc *__restrict__ D, int cur, const int *__restrict__ off,
                         int nd) {
  pdl_wait();
  const int t = threadIdx.x & 63, spb = blockDim.x >> 6;
  for_each_slot<WL, false>(D, off, nd, blockIdx.x * spb + (threadIdx.x >> 6), gridDim.x * spb,
                [&](const DomainDesc &dd, int s) {
    const S *__restrict__ f = (const S *)dd.f[cur];
    const Geometry &g = dd.g;
    const BrickMap &m = dd.m;
    float *__restrict__ U0s = dd.U0s;
    const int B = m.slot_brick[s];
    const int bx = B % g.nbx, rr = B / g.nbx;
    const int by = rr % g.nby, bz = rr / g.nby;
    const int x = bx * 4 + (t & 3), y = by * 4 + ((t >> 2) & 3), z = bz * 4 + (t >> 4);
    float *u = U0s + (size_t)s * SLOT_FLOATS + t;
    cell_velocity<S, true>(f, g, x, y, z, u[0], u[BRICK_CELLS], u[2 * BRICK_CELLS]);
  });
}

// The two U0 pre-computations that the paper compares in Sec. 5, as
// alternatives to the brick set above.
//
// Box strategy: U0 on every cell of each body's bounding box, the box of its
// points' rest positions moved by the body's rigid transform M(t) (Alg. 1)
// and widened by the support (taps floor(x) - 1 .. floor(x) + 2), rounded out
// to whole bricks so that it holds every active brick of the body; written to
// a full-lattice field like the paper's U, from which the active bricks take
// their cells.  Cells where boxes overlap are computed once per box.  One
// block row (blockIdx.y) per body, grid-stride over the box's cells, x
// fastest.
struct CellBox {
  int lo[3], ext[3];
};

__device__ CellBox body_cell_box(const DomainDesc &d, int b) {
  const double *rb = d.rest_box + 6 * b;
  double mn[3] = {rb[0], rb[1], rb[2]}, mx[3] = {rb[3], rb[4], rb[5]};
  if (d.nb > 0) {
    // the rest box's corners under M(t): a rotation about z through the
    // body's centre (Alg. 1); z is unchanged
    const double *c = d.centre + 3 * b;
    const double phi = d.phase[b] + d.omega[b] * (double)(*d.t);
    double sn, cs;
    sincos(phi, &sn, &cs);
    double lo0 = 1e300, lo1 = 1e300, hi0 = -1e300, hi1 = -1e300;
    for (int q = 0; q < 4; q++) {
      const double rx = ((q & 1) ? rb[3] : rb[0]) - c[0], ry = ((q & 2) ? rb[4] : rb[1]) - c[1];
      const double X = c[0] + (cs * rx - sn * ry), Y = c[1] + (sn * rx + cs * ry);
      lo0 = fmin(lo0, X);
      hi0 = fmax(hi0, X);
      lo1 = fmin(lo1, Y);
      hi1 = fmax(hi1, Y);
    }
    mn[0] = lo0;
    mx[0] = hi0;
    mn[1] = lo1;
    mx[1] = hi1;
  }
  // cells floor(min) - 1 .. floor(max) + 2, rounded out to whole bricks (the
  // bounds widened by 1e-6 first: a point's own rotation may round a last
  // bit past the moved corners); the first cell wrapped into the lattice (a
  // multiple of 4, as n is), the extent at most the lattice
  const int n[3] = {d.g.nx, d.g.ny, d.g.nz};
  CellBox cb;
  for (int a = 0; a < 3; a++) {
    const double lo = 4.0 * floor((floor(mn[a] - 1e-6) - 1.0) / 4.0);
    const double hi = 4.0 * floor((floor(mx[a] + 1e-6) + 2.0) / 4.0) + 3.0;
    const double w = lo - (double)n[a] * floor(lo / (double)n[a]);
    cb.lo[a] = min((int)w, n[a] - 4);
    cb.ext[a] = (int)fmin(hi - lo + 1.0, (double)n[a]);
  }
  return cb;
}

template <typename S>
__global__ void __launch_bounds__(256) box_moments_kernel(const DomainDesc *__restrict__ D,
                                                          int cur) {
  pdl_wait();
  const DomainDesc &d = D[0];
  const int b = blockIdx.y;
  if (b >= d.nbox) return;
  __shared__ CellBox sb;
  if (threadIdx.x == 0) sb = body_cell_box(d, b);
  __syncthreads();
  const CellBox cb = sb;
  const Geometry &g = d.g;
  const S *__restrict__ f = (const S *)d.f[cur];
  float *__restrict__ U = d.Ufull;
  const size_t N = (size_t)g.ncell;
  const int64_t cells = (int64_t)cb.ext[0] * cb.ext[1] * cb.ext[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % cb.ext[0]);
    const int64_t r = i / cb.ext[0];
    const int iy = (int)(r % cb.ext[1]), iz = (int)(r / cb.ext[1]);
    const int x = wrapi(cb.lo[0] + ix, g.nx), y = wrapi(cb.lo[1] + iy, g.ny),
              z = wrapi(cb.lo[2] + iz, g.nz);
    const size_t n = ((size_t)z * g.ny + y) * g.nx + x;
    cell_velocity<S>(f, g, x, y, z, U[n], U[N + n], U[2 * N + n]);
  }
}

// The active bricks' U0 from the full-lattice field of the box strategy: 64
// threads per slot.
__global__ void __launch_bounds__(256) box_gather_kernel(const DomainDesc *__restrict__ D) {
  pdl_wait();
  const int t = threadIdx.x & 63, spb = blockDim.x >> 6;
  for_each_slot<false, false>(D, nullptr, 1, blockIdx.x * spb + (threadIdx.x >> 6),
                              gridDim.x * spb, [&](const DomainDesc &d, int s) {
    const Geometry &g = d.g;
    const int B = d.m.slot_brick[s];
    const int bx = B % g.nbx, rr = B / g.nbx;
    const int by = rr % g.nby, bz = rr / g.nby;
    const int x = bx * 4 + (t & 3), y = by * 4 + ((t >> 2) & 3), z = bz * 4 + (t >> 4);
    const size_t N = (size_t)g.ncell, n = ((size_t)z * g.ny + y) * g.nx + x;
    float *u = d.U0s + (size_t)s * SLOT_FLOATS + t;
    u[0] = d.Ufull[n];
    u[BRICK_CELLS] = d.Ufull[N + n];
    u[2 * BRICK_CELLS] = d.Ufull[2 * N + n];
  });
}

// Kernel strategy: U0 on the 4 x 4 x 4 support of every point (the taps at
// which its weights can be non-zero; the paper's 5 x 5 x 5 block adds a fifth
// tap per axis of weight 0), 64 threads per point, written into the slots of
// the active bricks; a cell covered by several supports is computed and
// written once per support (the same value each time).  The other cells of
// an active brick keep finite values of earlier steps: every pair weighs them
// by exactly 0.
template <typename S>
__global__ void __launch_bounds__(256) point_moments_kernel(const DomainDesc *__restrict__ D,
                                                            int cur) {
  pdl_wait();
  const DomainDesc &d = D[0];
  const Geometry &g = d.g;
  const S *__restrict__ f = (const S *)d.f[cur];
  const int nact = active_slots(d.m);
  const int t = threadIdx.x & 63, ppb = blockDim.x >> 6;
  for (int64_t k = (int64_t)blockIdx.x * ppb + (threadIdx.x >> 6); k < d.np;
       k += (int64_t)gridDim.x * ppb) {
    const int4 b = d.pp.base[k];
    const int x = wrapi(b.x - 1 + (t & 3), g.nx), y = wrapi(b.y - 1 + ((t >> 2) & 3), g.ny),
              z = wrapi(b.z - 1 + (t >> 4), g.nz);
    const int s = d.m.brick_slot[((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2)];
    if (s < 0 || s >= nact) continue;
    float *u = d.U0s + (size_t)s * SLOT_FLOATS + brick_local(x, y, z);
    cell_velocity<S>(f, g, x, y, z, u[0], u[BRICK_CELLS], u[2 * BRICK_CELLS]);
  }
}


// First pass of a step over each active brick after the moments: G_0 = 0 or
// S[du_init] (warm start), and the pairs' shares of I[U0 + G_0] for the first
// iteration.  One warp per brick, grid-stride over the active bricks.
template <bool WL>
__global__ void __launch_bounds__(32, 32)
    brick_init_kernel(const DomainDesc *__restrict__ D, int use_du, const int *__restrict__ off,
                      int nd) {
  pdl_wait();
  __shared__ BrickSmem sm;
  const int t = threadIdx.x, r = t & 15;
  for_each_slot<WL, true>(D, off, nd, blockIdx.x, gridDim.x, [&](const DomainDesc &d, int s) {
    const PairMap &pm = d.pm;
    const float4 *__restrict__ du_init = use_du ? d.du : nullptr;
    const float *__restrict__ U0s = d.U0s;
    float *__restrict__ Gs = d.Gs;
    const int p0 = pm.start[s], cnt = pm.count[s];
    float4 G[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                   make_float4(0.f, 0.f, 0.f, 0.f)};
    if (du_init) brick_gather(sm, pm, p0, cnt, du_init, G);
    const size_t o = (size_t)s * SLOT_FLOATS + 4 * r;
    if (t < 16) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        *(float4 *)(Gs + o + c * BRICK_CELLS) = G[c];
        sm.sF[c][r] = add4(*(const float4 *)(U0s + o + c * BRICK_CELLS), G[c]);
      }
    }
    __syncwarp();
    brick_interp(sm, pm, p0, cnt, du_init != nullptr && cnt <= SP_CHUNK);
    __syncwarp();
  });
}

// One iteration's spreading over one active brick (slot s): G = S[du], the
// squared change of G into res[slot] (tolerance mode: res != nullptr), and,
// unless this is the last iteration, the pairs' shares of I[U0 + G] for the
// next one.
__device__ __forceinline__ void spread_brick(BrickSmem &sm, const PairMap &pm,
                                             const float4 *__restrict__ vals,
                                             const float *__restrict__ U0s, float *__restrict__ Gs,
                                             float *__restrict__ res, int s, int do_interp) {
  const int t = threadIdx.x, r = t & 15;
  const int p0 = pm.start[s], cnt = pm.count[s];
  float4 G[3];
  brick_gather(sm, pm, p0, cnt, vals, G);
  const size_t o = (size_t)s * SLOT_FLOATS + 4 * r;
  if (res) {
    float e = 0.f;
    if (t < 16) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float4 old = *(const float4 *)(Gs + o + c * BRICK_CELLS);
        const float a = G[c].x - old.x, b = G[c].y - old.y, cc = G[c].z - old.z,
                    dd = G[c].w - old.w;
        e += ((a * a + b * b) + cc * cc) + dd * dd;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (t == 0) res[s] = e;
  }
  if (t < 16) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      *(float4 *)(Gs + o + c * BRICK_CELLS) = G[c];
      if (do_interp)
        sm.sF[c][r] = add4(*(const float4 *)(U0s + o + c * BRICK_CELLS), G[c]);
    }
  }
  __syncwarp();
  if (do_interp) brick_interp(sm, pm, p0, cnt, cnt <= SP_CHUNK);
  __syncwarp();
}

// One iteration's spreading over each active brick (spread_brick; the single
// lattice's loop keeps the per-domain fields in registers across bricks).
template <bool WL>
__global__ void __launch_bounds__(32, 32)
    brick_spread_kernel(const DomainDesc *__restrict__ D, int do_interp, int tol_mode,
                        const int *__restrict__ off, int nd) {
  pdl_wait();
  __shared__ BrickSmem sm;
  if constexpr (WL) {
    // (tolerance mode: the bricks of a domain that has converged are skipped)
    for_each_slot<true, true>(D, off, nd, blockIdx.x, gridDim.x, [&](const DomainDesc &d, int s) {
      if (tol_mode && d.state->done) return;
      spread_brick(sm, d.pm, d.du, d.U0s, d.Gs, tol_mode ? d.res : nullptr, s, do_interp);
    });
  } else {
    const DomainDesc &d = D[blockIdx.y];
    const BrickMap m = d.m;
    const PairMap pm = d.pm;
    const float4 *__restrict__ vals = d.du;
    const float *__restrict__ U0s = d.U0s;
    float *__restrict__ Gs = d.Gs;
    float *__restrict__ res = tol_mode ? d.res : nullptr;
    // active_slots(m), its counters loaded beside the stop flag
    const int c0 = ld_early(m.counters), c1 = ld_early(m.counters + 1);
    if (stopped(d, tol_mode)) return;
    const int nslots = (c1 & 4) ? 0 : (c0 < m.max_slots ? c0 : m.max_slots);
    const int t = threadIdx.x, r = t & 15;
    for (int b = blockIdx.x; b < nslots; b += gridDim.x) {
      const int s = slot_in_order(m, b);
      const int p0 = pm.start[s], cnt = pm.count[s];
      float4 G[3];
      brick_gather(sm, pm, p0, cnt, vals, G);
      const size_t o = (size_t)s * SLOT_FLOATS + 4 * r;
      if (res) {
        float e = 0.f;
        if (t < 16) {
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const float4 old = *(const float4 *)(Gs + o + c * BRICK_CELLS);
            const float a = G[c].x - old.x, bb = G[c].y - old.y, cc = G[c].z - old.z,
                        dd = G[c].w - old.w;
            e += ((a * a + bb * bb) + cc * cc) + dd * dd;
          }
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) e += __shfl_xor_sync(0xffffffffu, e, sh);
        if (t == 0) res[s] = e;
      }
      if (t < 16) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          *(float4 *)(Gs + o + c * BRICK_CELLS) = G[c];
          if (do_interp)
            sm.sF[c][r] = add4(*(const float4 *)(U0s + o + c * BRICK_CELLS), G[c]);
        }
      }
      __syncwarp();
      if (do_interp) brick_interp(sm, pm, p0, cnt, cnt <= SP_CHUNK);
      __syncwarp();
    }
  }
}

// ||S[v]||^2 per active brick into res[slot] (v = vals, scaled by .w when
// scale_by_w): the denominators of the residual.
template <bool WL>
__global__ void __launch_bounds__(32, 32)
    brick_norm_kernel(const DomainDesc *__restrict__ D, int which, const int *__restrict__ off,
                      int nd) {
  pdl_wait();
  __shared__ BrickSmem sm;
  const int t = threadIdx.x;
  for_each_slot<WL, true>(D, off, nd, blockIdx.x, gridDim.x, [&](const DomainDesc &d, int s) {
    const PairMap &pm = d.pm;
    const float4 *__restrict__ vals = which == 0 ? d.pp.ut : d.uint;
    const int scale_by_w = which == 0;
    float *__restrict__ res = d.res;
    float4 G[3];
    brick_gather(sm, pm, pm.start[s], pm.count[s], vals, G, scale_by_w != 0);
    float e = 0.f;
    if (t < 16) {
#pragma unroll
      for (int c = 0; c < 3; c++)
        e += ((G[c].x * G[c].x + G[c].y * G[c].y) + G[c].z * G[c].z) + G[c].w * G[c].w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (t == 0) res[s] = e;
    __syncwarp();
  });
}

// Deterministic sum of res[0 .. nslots) over RES_BLOCKS blocks of 256
// threads: thread j of block b adds res[b*256 + j + k*RES_BLOCKS*256] in k
// order, the block adds its threads' sums in a fixed shuffle tree (FP32: FP64
// arithmetic runs at ~1/64 of the FP32 rate here and sat on the critical path
// of this per-iteration check), and the last block to finish adds the block
// sums in block order in FP64.  Returns true on that block's thread 0, with
// the sum in *total.  Every thread of every block calls it.
__device__ bool res_sum(const BrickMap &m, const float *__restrict__ res, IbmState *st,
                        double *total) {
  __shared__ float red[8];
  __shared__ bool last;
  const int nslots = active_slots(m), t = threadIdx.x, lane = t & 31, wid = t >> 5;
  float a = 0.f;
  for (int s = blockIdx.x * 256 + t; s < nslots; s += RES_BLOCKS * 256) a += res[s];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) red[wid] = a;
  __syncthreads();
  if (t == 0) {
    const float b = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    st->bsum[blockIdx.x] = (double)b;
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == (unsigned)RES_BLOCKS - 1;
  }
  __syncthreads();
  if (!last || t != 0) return false;
  __threadfence();
  double v = 0.0;
  for (int b = 0; b < RES_BLOCKS; b++) v += __ldcg(st->bsum + b);
  st->ticket = 0u;
  *total = v;
  return true;
}

// mode 0: den2 = sum res (||S[s u_k]||^2); mode 1: fallback den2 (used when
// the first is 0): sum res, or 1 if that is 0 as well; mode 2: as mode 0 where
// the surface velocities are known not to vanish (1 should the sum still be 0).
__global__ void __launch_bounds__(256) ibm_den_kernel(const DomainDesc *__restrict__ D,
                                                       int mode) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  if (d.np == 0) return;  // (a domain of a batch without points)
  IbmState *st = d.state;
  double v;
  if (!res_sum(d.m, d.res, st, &v)) return;
  if (mode == 0 || mode == 2) {
    st->den2 = mode == 2 && !(v > 0.0) ? 1.0 : v;
    st->done = 0;
    st->iters = 0;
  } else if (st->den2 == 0.0) {
    st->den2 = v > 0.0 ? v : 1.0;
  }
}

// After iteration `it`: eps = ||G_{it+1} - G_it|| / den (Eulerian residual of
// the fixed point); stop at the first eps <= tol or at max_iter iterations.
// (done is read before any block counts itself, and set after all have.)
__global__ void __launch_bounds__(256) ibm_check_kernel(const DomainDesc *__restrict__ D, int it,
                                                         double tol, int max_iter) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  if (d.np == 0) return;  // (a domain of a batch without points)
  IbmState *st = d.state;
  if (st->done) return;
  double v;
  if (!res_sum(d.m, d.res, st, &v)) return;
  const double eps = sqrt(v / st->den2);
  if (it < IbmState::HIST) st->eps[it] = eps;
  st->last_eps = eps;
  if (eps <= tol || it + 1 >= max_iter) {
    st->done = 1;
    st->iters = it + 1;
    st->capped = eps > tol;
  }
}

// Alg. 1 loop body per point: u_n(k) = sum of its bricks' shares (brick order),
// g = u_k - u_n, du += s g (du starts at 0 when first && !warm).
__global__ void __launch_bounds__(512)
    point_update_kernel(const DomainDesc *__restrict__ D, int first, int warm, int tol_mode) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.np) return;
  const PointPrep pp = d.pp;
  const PairMap pm = d.pm;
  float4 *__restrict__ du = d.du;
  float4 *__restrict__ uint = d.uint;
  const int4 *pk = (const int4 *)(pm.point_pairs + 8 * k);
  const int4 a = ld_early(pk), b = ld_early(pk + 1);
  if (stopped(d, tol_mode)) return;
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
  float4 dk = (first && !warm) ? make_float4(0.f, 0.f, 0.f, 0.f) : du[k];
  dk.x += ut.w * (ut.x - ux);
  dk.y += ut.w * (ut.y - uy);
  dk.z += ut.w * (ut.z - uz);
  du[k] = dk;
  uint[k] = make_float4(ux, uy, uz, 0.f);
}

// ---- conjugate gradients on the lattice form of the fixed point -----------
//
// The loop above is Richardson's iteration with unit step on B G = c, with
// B = S diag(s) I (symmetric positive semi-definite: S is the adjoint of I)
// and c = S[s (u_k - I[U0])]; its residual c - B G = S[s g] is the one eps
// measures.  These kernels run conjugate gradients on the same system, in
// the single-reduction form of Chronopoulos and Gear: with R_n the residual,
// W_n = B R_n, rho_n = R_n . R_n and delta_n = W_n . R_n,
//   beta_n  = rho_n / rho_{n-1},   alpha_n = rho_n / (delta_n - beta_n rho_n / alpha_{n-1})
//   P_n = R_n + beta_n P_{n-1},   B P_n = W_n + beta_n B P_{n-1}
//   G_{n+1} = G_n + alpha_n P_n,  R_{n+1} = R_n - alpha_n B P_n.
// Every lattice vector is a spread of point vectors (R = S[v] with v = s r and
// r the point residual, P = S[p], G = S[du]; B R = S[s a] with a = I[R], and
// B P = S[s y] with y = I[P]), so only point vectors are carried:
//   p = v + beta p,  y = a + beta y,  du += alpha p,  r -= alpha y,  v = s r,
// and G = S[du] is spread once after the last iteration.  rho_n = |S[v_n]|^2
// is summed per brick by the pass that gathers S[v_n] (and leaves the pair
// shares of I[R_n]); delta_n = sum_k s(k) |a_n(k)|^2 per block of the point
// pass that sums those shares (which also adds up slices of the brick sums),
// and every block of the update pass adds the block sums itself.  Point
// arrays d.cg: [0] r, [1] v, [2] p, [3] y, [4] a (np each).

constexpr int CG_BLOCK = 256;  // threads of the CG point kernels (fixed: the
                               // block sums of delta do not depend on the
                               // launch shape)

// the sum of a point's pair shares in brick order, from its eight pair
// indices (-1: none)
__device__ __forceinline__ float4 shares_of(const PairMap &pm, int4 a, int4 b) {
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
  return make_float4(ux, uy, uz, 0.f);
}

__device__ __forceinline__ float4 shares_sum(const PairMap &pm, int64_t k) {
  const int4 *pk = (const int4 *)(pm.point_pairs + 8 * k);
  return shares_of(pm, pk[0], pk[1]);
}

// r_0 = u_k - I[U0 + G_0] from the shares brick_init left, v_0 = s r_0,
// p = y = 0 (beta_0 = 0), du = 0 without a warm start.
__global__ void __launch_bounds__(CG_BLOCK) cg_start_kernel(const DomainDesc *__restrict__ D,
                                                            int warm) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) d.state->cg_stop = INT_MAX;
  if (k >= d.np) return;
  const int64_t np = d.np;
  float4 *__restrict__ cg = d.cg;
  const float4 u = shares_sum(d.pm, k);
  const float4 ut = d.pp.ut[k];
  const float4 r = make_float4(ut.x - u.x, ut.y - u.y, ut.z - u.z, 0.f);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  cg[k] = r;
  cg[np + k] = make_float4(ut.w * r.x, ut.w * r.y, ut.w * r.z, 0.f);
  cg[2 * np + k] = z;
  cg[3 * np + k] = z;
  if (!warm) d.du[k] = z;
}

// Residual replacement (tolerance mode, after the recursion reported
// convergence): r = u_k - I[U0 + S[du]] from the shares of the gather-and-
// interpolate pass, v = s r; the search directions p, y are kept.  The
// recursively updated r drifts from the true residual by FP32 rounding that
// CG amplifies, so the stop is confirmed by one more iteration on the true
// one.  Clears the stop flag for that iteration.
__global__ void __launch_bounds__(CG_BLOCK) cg_replace_kernel(const DomainDesc *__restrict__ D) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    d.state->done = 0;
    d.state->cg_stop = INT_MAX;
  }
  if (k >= d.np) return;
  const float4 u = shares_sum(d.pm, k);
  const float4 ut = d.pp.ut[k];
  const float4 r = make_float4(ut.x - u.x, ut.y - u.y, ut.z - u.z, 0.f);
  d.cg[k] = r;
  d.cg[d.np + k] = make_float4(ut.w * r.x, ut.w * r.y, ut.w * r.z, 0.f);
}

// R_n = S[v_n] on each active brick, |R_n|^2 into res[slot], and the pair
// shares of I[R_n].  One warp per brick.
template <bool WL>
__global__ void __launch_bounds__(32, 32)
    cg_brick_kernel(const DomainDesc *__restrict__ D, int tol_mode, const int *__restrict__ off,
                    int nd) {
  pdl_wait();
  __shared__ BrickSmem sm;
  const int t = threadIdx.x, r = t & 15;
  for_each_slot<WL, true>(D, off, nd, blockIdx.x, gridDim.x, [&](const DomainDesc &d, int s) {
    const PairMap &pm = d.pm;
    const int p0 = ld_early(pm.start + s), cnt = ld_early(pm.count + s);
    if (stopped(d, tol_mode)) return;
    float4 R[3];
    brick_gather(sm, pm, p0, cnt, d.cg + d.np, R);
    float e = 0.f;
    if (t < 16) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        e += ((R[c].x * R[c].x + R[c].y * R[c].y) + R[c].z * R[c].z) + R[c].w * R[c].w;
        sm.sF[c][r] = R[c];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (t == 0) d.res[s] = e;
    __syncwarp();
    brick_interp(sm, pm, p0, cnt, cnt <= SP_CHUNK);
    __syncwarp();
  });
}

// Sum over the block's threads of v in a fixed order: a shuffle tree within
// each warp, then, in every warp alike, a shuffle tree over the warps' sums.
// Every thread calls it and gets lane 0's result.  FP32: FP64 arithmetic is
// slow on this part (~1/64 of the FP32 rate) and sat on the critical path of
// these short kernels; a 256-term FP32 tree is within ~8 ulp, ample for the
// CG coefficients.  red: CG_BLOCK / 32 floats of shared memory.
__device__ __forceinline__ float block_sum256(float v, float *red) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // (red may still be read by a previous call)
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float w = lane < CG_BLOCK / 32 ? red[lane] : 0.f;
#pragma unroll
  for (int o = CG_BLOCK / 64; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  return __shfl_sync(0xffffffffu, w, 0);  // (lane 0's order: the same in every warp and block)
}

// a_n = I[R_n] per point (kept for the update); block b's sums of
// delta_n = sum_k s(k) |a_n(k)|^2 over its points and of rho_n over the
// bricks [b m, (b + 1) m) of res (m = ceil(nslots / blocks)), each in a fixed
// tree, into cg_part[b].
__global__ void __launch_bounds__(CG_BLOCK) cg_dot_kernel(const DomainDesc *__restrict__ D,
                                                          int tol_mode) {
  pdl_wait();
  __shared__ float red[CG_BLOCK / 32];
  const DomainDesc &d = D[blockIdx.y];
  const int nbk = (d.np + CG_BLOCK - 1) / CG_BLOCK;
  if ((int)blockIdx.x >= nbk) return;
  const int t = threadIdx.x, b = blockIdx.x;
  const int64_t k = (int64_t)b * CG_BLOCK + t;
  // the point's pair indices loaded beside the stop flag
  int4 pa = make_int4(-1, -1, -1, -1), pb = pa;
  if (k < d.np) {
    const int4 *pk = (const int4 *)(d.pm.point_pairs + 8 * k);
    pa = ld_early(pk);
    pb = ld_early(pk + 1);
  }
  if (stopped(d, tol_mode)) return;
  float e = 0.f;
  if (k < d.np) {
    const float4 a = shares_of(d.pm, pa, pb);
    d.cg[4 * (int64_t)d.np + k] = a;
    e = d.pp.ut[k].w * ((a.x * a.x + a.y * a.y) + a.z * a.z);
  }
  const int nslots = active_slots(d.m);
  const int m = (nslots + nbk - 1) / nbk;
  float f = 0.f;
  for (int j = b * m + t; j < min(nslots, (b + 1) * m); j += CG_BLOCK) f += d.res[j];
  const float bd = block_sum256(e, red);
  const float br = block_sum256(f, red);
  if (t == 0) {
    d.cg_part[2 * b] = bd;
    d.cg_part[2 * b + 1] = br;
  }
}

// The updates of iteration n, and u_interp = u_k - r_n (the velocity
// interpolated from the iterate).  Every block adds the block sums of
// cg_dot_kernel in block order (the same bits in every block) and forms
// alpha_n and beta_n from them and from rho_{n-1}, alpha_{n-1} (kept by
// iteration parity, so that no block reads a value this launch replaces; in
// FP32, like the sums);
// block 0 stores rho_n, alpha_n, and in tolerance mode records
// eps_n = sqrt(rho_n) / den and stops at the first eps_n <= tol or at
// max_iter iterations (this iteration's update still runs everywhere).
__global__ void __launch_bounds__(CG_BLOCK)
    cg_update_kernel(const DomainDesc *__restrict__ D, int it, double tol, int max_iter,
                     int tol_mode, int confirm) {
  pdl_wait();
  __shared__ float red[CG_BLOCK / 32];
  __shared__ float coef[2];
  __shared__ bool keep;
  const DomainDesc &d = D[blockIdx.y];
  IbmState *st = d.state;
  const int nbk = (d.np + CG_BLOCK - 1) / CG_BLOCK;
  if ((int)blockIdx.x >= nbk) return;
  // (cg_stop, one word, is the index of the iteration that converged; block
  // 0 of this launch may set it to it, which reads the same here as before)
  if (tol_mode && st->cg_stop < it) return;
  const int t = threadIdx.x;
  float a1 = 0.f, a2 = 0.f;
  for (int j = t; j < nbk; j += CG_BLOCK) {
    a1 += (float)d.cg_part[2 * j];  // (FP32 values held in the FP64 array)
    a2 += (float)d.cg_part[2 * j + 1];
  }
  const float delta = block_sum256(a1, red);
  const float rho = block_sum256(a2, red);
  if (t == 0) {
    const int cur = it & 1, prev = cur ^ 1;
    const float rho_prev = (float)st->cg_rho[prev], alpha_prev = (float)st->cg_alpha[prev];
    float beta = (it > 0 && rho_prev > 0.f) ? rho / rho_prev : 0.f;
    float den = delta;
    if (beta > 0.f && alpha_prev > 0.f) den = delta - beta * rho / alpha_prev;
    if (!(den > 0.f)) {  // rounding lost the conjugacy: restart from R_n
      beta = 0.f;
      den = delta;
    }
    const float alpha = (rho > 0.f && den > 0.f) ? rho / den : 0.f;
    coef[0] = alpha;
    coef[1] = beta;
    // a confirming iteration (r the true residual) that meets tol keeps its
    // iterate: the one whose residual was checked (the same test as the stop
    // below, so that a stop without the cap means a kept iterate)
    keep = confirm && tol_mode && sqrt((double)rho / st->den2) <= tol;
    if (blockIdx.x == 0) {
      st->cg_rho[cur] = rho;
      st->cg_alpha[cur] = alpha;
      if (tol_mode) {
        const double eps = sqrt((double)rho / st->den2);
        if (it < IbmState::HIST) st->eps[it] = eps;
        st->last_eps = eps;
        if (eps <= tol || it + 1 >= max_iter) {
          st->cg_stop = it;
          st->iters = it + 1;
          st->capped = eps > tol;
          st->done = 1;
        }
      }
    }
  }
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * CG_BLOCK + t;
  if (k >= d.np) return;
  const int64_t np = d.np;
  float4 *__restrict__ cg = d.cg;
  if (keep) {
    const float4 r = cg[k], ut = d.pp.ut[k];
    d.uint[k] = make_float4(ut.x - r.x, ut.y - r.y, ut.z - r.z, 0.f);
    return;
  }
  const float alpha = coef[0], beta = coef[1];
  float4 r = cg[k], p = cg[2 * np + k], y = cg[3 * np + k];
  const float4 a = cg[4 * np + k], ut = d.pp.ut[k];
  float4 dk = d.du[k];
  d.uint[k] = make_float4(ut.x - r.x, ut.y - r.y, ut.z - r.z, 0.f);
  p.x = fmaf(beta, p.x, ut.w * r.x);
  p.y = fmaf(beta, p.y, ut.w * r.y);
  p.z = fmaf(beta, p.z, ut.w * r.z);
  y.x = fmaf(beta, y.x, a.x);
  y.y = fmaf(beta, y.y, a.y);
  y.z = fmaf(beta, y.z, a.z);
  dk.x = fmaf(alpha, p.x, dk.x);
  dk.y = fmaf(alpha, p.y, dk.y);
  dk.z = fmaf(alpha, p.z, dk.z);
  r.x = fmaf(-alpha, y.x, r.x);
  r.y = fmaf(-alpha, y.y, r.y);
  r.z = fmaf(-alpha, y.z, r.z);
  cg[k] = r;
  cg[np + k] = make_float4(ut.w * r.x, ut.w * r.y, ut.w * r.z, 0.f);
  cg[2 * np + k] = p;
  cg[3 * np + k] = y;
  d.du[k] = dk;
}

// s(k) (u_k - u(k)) with u(k) the sum of the point's pair shares: the
// first increment from a zero start, for the fallback residual denominator.
__global__ void __launch_bounds__(512)
    point_residual0_kernel(const DomainDesc *__restrict__ D) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.np) return;
  const PointPrep pp = d.pp;
  const PairMap pm = d.pm;
  float4 *__restrict__ out = d.uint;
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
  out[k] = make_float4(ut.w * (ut.x - ux), ut.w * (ut.y - uy), ut.w * (ut.z - uz), 0.f);
}

// Features of the learned warm start, per point (velocities in units of
// MLP_VSCALE, lengths of MLP_LSCALE), from the pair shares of
// I[U0 + S[du_prev]] left by brick_init:
//   0-2  u_i = I[U0 + S[du_prev]](k), the fluid velocity interpolated at the
//        point with the previous step's force applied
//   3-5  u_k, the surface velocity
//   6-8  du_prev, the previous step's final velocity correction
//   9    local point density: pairs of the point's bricks per brick cell
//   10-12 body-relative rest position: radius and axial offset from the
//        body's axis, and the speed omega r (0 without bodies)
//   13-15 u_k - u_i, the slip left by the previous force
__global__ void __launch_bounds__(512)
    mlp_features_kernel(const DomainDesc *__restrict__ D, int use_prev) {
  pdl_wait();
  const DomainDesc &d = D[blockIdx.y];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.np) return;
  const PointPrep pp = d.pp;
  const PairMap pm = d.pm;
  const BrickMap m = d.m;
  const float4 *__restrict__ du_prev = use_prev ? d.du : nullptr;
  const PointsIn p{d.np, d.X, d.body, d.area, d.utarget};
  const Bodies bd{d.centre, d.omega, d.phase, d.nb};
  float *__restrict__ X = d.feat;
  const int4 *pk = (const int4 *)(pm.point_pairs + 8 * k);
  const int4 a = pk[0], b = pk[1];
  const int idx[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  float ux = 0.f, uy = 0.f, uz = 0.f, dens = 0.f;
  int nb = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    if (idx[j] >= 0) {
      const float4 v = pm.part[idx[j]];
      ux += v.x;
      uy += v.y;
      uz += v.z;
      dens += (float)pm.count[m.brick_slot[pm.brick[idx[j]]]];
      nb++;
    }
  }
  const float iv = 1.f / MLP_VSCALE;
  const float4 ut = pp.ut[k];
  const float4 dp = du_prev ? du_prev[k] : make_float4(0.f, 0.f, 0.f, 0.f);
  float r = 0.f, zr = 0.f, sp = 0.f;
  if (bd.nb > 0) {
    const int bi = p.body ? p.body[k] : 0;
    const double *c = bd.centre + 3 * bi;
    const double dx = p.X[3 * k] - c[0], dy = p.X[3 * k + 1] - c[1], dz = p.X[3 * k + 2] - c[2];
    r = (float)sqrt(dx * dx + dy * dy);
    zr = (float)dz;
    sp = (float)fabs(bd.omega[bi]) * r;
  }
  float *o = X + MLP_IN * k;
  o[0] = ux * iv;
  o[1] = uy * iv;
  o[2] = uz * iv;
  o[3] = ut.x * iv;
  o[4] = ut.y * iv;
  o[5] = ut.z * iv;
  o[6] = dp.x * iv;
  o[7] = dp.y * iv;
  o[8] = dp.z * iv;
  o[9] = nb > 0 ? dens / (64.f * nb) : 0.f;
  o[10] = r / MLP_LSCALE;
  o[11] = zr / MLP_LSCALE;
  o[12] = sp * iv;
  o[13] = (ut.x - ux) * iv;
  o[14] = (ut.y - uy) * iv;
  o[15] = (ut.z - uz) * iv;
}

__global__ void mlp_targets_kernel(int64_t np, const float *__restrict__ X,
                                   const float4 *__restrict__ du, float *__restrict__ T) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const float iv = 1.f / MLP_VSCALE;
  const float4 d = du[k];
  T[3 * k] = d.x * iv - X[MLP_IN * k + 6];
  T[3 * k + 1] = d.y * iv - X[MLP_IN * k + 7];
  T[3 * k + 2] = d.z * iv - X[MLP_IN * k + 8];
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

// Writes a descriptor passed by value into device memory: the descriptor is
// then part of the launch, not a copy from (pageable) host memory.
__global__ void store_desc_kernel(DomainDesc dd, DomainDesc *__restrict__ D) {
  if (threadIdx.x == 0) *D = dd;
}

__global__ void pack_points_kernel(int64_t n, const float4 *__restrict__ a, float *__restrict__ o) {
  pdl_wait();
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

inline unsigned xblocks(int64_t want, int nd, int cap) {
  int64_t b = std::min<int64_t>(want, std::max<int64_t>(1, cap / std::max(1, nd)));
  return (unsigned)std::max<int64_t>(1, b);
}

template <typename S>
cudaError_t brick_moments_typed(const DomainDesc *D, const BatchDims &dims, int cur,
                                cudaStream_t st) {
  const int spb = dims.ls.moments_spb;
  if (spb != 1 && spb != 2 && spb != 4) return cudaErrorInvalidValue;
  // a batch with a work list: one grid over all domains' slots
  const dim3 grid = dims.work_off
                        ? dim3(152 * 64 / spb)
                        : dim3(xblocks((dims.max_slots + spb - 1) / spb, dims.nd, 152 * 64 / spb),
                               dims.nd);
  return dims.work_off ? launch_pdl(brick_moments_kernel<S, true>, grid, dim3(64 * spb), 0, st, D,
                                    cur, dims.work_off, dims.nd)
                       : launch_pdl(brick_moments_kernel<S, false>, grid, dim3(64 * spb), 0, st, D,
                                    cur, dims.work_off, dims.nd);
}

}  // namespace

cudaError_t launch_prepare_points(const DomainDesc *D, const BatchDims &dims, cudaStream_t st,
                                  const double *Xsrc, const float *Usrc, long long t_step) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int pb = dims.ls.point_block;
  if (pb != 128 && pb != 256 && pb != 512) return cudaErrorInvalidValue;
  if ((Xsrc || Usrc) && dims.nd != 1) return cudaErrorInvalidValue;
  return launch_pdl(prepare_points_kernel, dim3(nblk(dims.max_points, pb), dims.nd), dim3(pb), 0,
                    st, D, Xsrc, Usrc, t_step);
}

cudaError_t launch_compact(const DomainDesc *D, const BatchDims &dims, cudaStream_t st) {
  return launch_pdl(compact_kernel, dim3(nblk(dims.max_bricks, COMPACT_TILE), dims.nd), dim3(256),
                    0, st, D);
}

cudaError_t launch_batch_worklist(const DomainDesc *D, const BatchDims &dims, cudaStream_t st) {
  if (!dims.work_off) return cudaSuccess;
  return launch_pdl(batch_worklist_kernel, dim3(1), dim3(1024), 0, st, D, dims.nd,
                    const_cast<int *>(dims.work_off));
}

cudaError_t launch_pair_lists(const DomainDesc *D, const BatchDims &dims, cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int pb = dims.ls.point_block;
  cudaError_t e =
      launch_pdl(pair_fill_kernel, dim3(nblk(dims.max_points, pb), dims.nd), dim3(pb), 0, st, D);
  // one warp per slot
  if (e == cudaSuccess)
    e = dims.work_off
            ? launch_pdl(pair_sort_kernel<true>, dim3(dims.ls.sort_blocks), dim3(128), 0, st, D,
                         dims.work_off, dims.nd)
            : launch_pdl(pair_sort_kernel<false>,
                         dim3(xblocks((dims.max_slots + 3) / 4, dims.nd, dims.ls.sort_blocks),
                              dims.nd),
                         dim3(128), 0, st, D, dims.work_off, dims.nd);
  return e;
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

cudaError_t launch_brick_moments(int storage, const DomainDesc *D, const BatchDims &dims, int cur,
                                 cudaStream_t st) {
  DISPATCH_STORAGE(storage, brick_moments_typed, D, dims, cur, st);
}

template <typename S>
cudaError_t box_moments_typed(const DomainDesc *D, int nbox, int cur, cudaStream_t st) {
  cudaError_t e = launch_pdl(box_moments_kernel<S>, dim3(std::max(1, 152 * 8 / std::max(1, nbox)),
                                                         nbox),
                             dim3(256), 0, st, D, cur);
  if (e == cudaSuccess)
    e = launch_pdl(box_gather_kernel, dim3(152 * 16), dim3(256), 0, st, D);
  return e;
}

template <typename S>
cudaError_t point_moments_typed(const DomainDesc *D, int64_t np, int cur, cudaStream_t st) {
  return launch_pdl(point_moments_kernel<S>, dim3(nblk(np, 4)), dim3(256), 0, st, D, cur);
}

cudaError_t launch_box_moments(int storage, const DomainDesc *D, int nbox, int cur,
                               cudaStream_t st) {
  if (nbox <= 0) return cudaSuccess;
  DISPATCH_STORAGE(storage, box_moments_typed, D, nbox, cur, st);
}

cudaError_t launch_point_moments(int storage, const DomainDesc *D, int64_t np, int cur,
                                 cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  DISPATCH_STORAGE(storage, point_moments_typed, D, np, cur, st);
}

// a batch with a work list: one grid over all domains' slots
static dim3 brick_grid(const BatchDims &dims) {
  if (dims.work_off) return dim3(dims.ls.brick_blocks);
  return dim3(xblocks(dims.max_slots, dims.nd, dims.ls.brick_blocks), dims.nd);
}

cudaError_t launch_brick_init(const DomainDesc *D, const BatchDims &dims, int use_du,
                              cudaStream_t st) {
  return dims.work_off ? launch_pdl(brick_init_kernel<true>, brick_grid(dims), dim3(32), 0, st, D,
                                    use_du, dims.work_off, dims.nd)
                       : launch_pdl(brick_init_kernel<false>, brick_grid(dims), dim3(32), 0, st, D,
                                    use_du, dims.work_off, dims.nd);
}

cudaError_t launch_brick_spread(const DomainDesc *D, const BatchDims &dims, int do_interp,
                                int tol_mode, cudaStream_t st) {
  return dims.work_off ? launch_pdl(brick_spread_kernel<true>, brick_grid(dims), dim3(32), 0, st, D,
                                    do_interp, tol_mode, dims.work_off, dims.nd)
                       : launch_pdl(brick_spread_kernel<false>, brick_grid(dims), dim3(32), 0, st, D,
                                    do_interp, tol_mode, dims.work_off, dims.nd);
}

cudaError_t launch_point_update(const DomainDesc *D, const BatchDims &dims, int first, int warm,
                                int tol_mode, cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int pb = dims.ls.point_block;
  return launch_pdl(point_update_kernel, dim3(nblk(dims.max_points, pb), dims.nd), dim3(pb), 0, st,
                    D, first, warm, tol_mode);
}

cudaError_t launch_cg_start(const DomainDesc *D, const BatchDims &dims, int warm,
                            cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  return launch_pdl(cg_start_kernel, dim3(nblk(dims.max_points, CG_BLOCK), dims.nd),
                    dim3(CG_BLOCK), 0, st, D, warm);
}

cudaError_t launch_cg_replace(const DomainDesc *D, const BatchDims &dims, cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  return launch_pdl(cg_replace_kernel, dim3(nblk(dims.max_points, CG_BLOCK), dims.nd),
                    dim3(CG_BLOCK), 0, st, D);
}

cudaError_t launch_cg_brick(const DomainDesc *D, const BatchDims &dims, int tol_mode,
                            cudaStream_t st) {
  return dims.work_off ? launch_pdl(cg_brick_kernel<true>, brick_grid(dims), dim3(32), 0, st, D,
                                    tol_mode, dims.work_off, dims.nd)
                       : launch_pdl(cg_brick_kernel<false>, brick_grid(dims), dim3(32), 0, st, D,
                                    tol_mode, dims.work_off, dims.nd);
}

cudaError_t launch_cg_dot(const DomainDesc *D, const BatchDims &dims, int tol_mode,
                          cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  return launch_pdl(cg_dot_kernel, dim3(nblk(dims.max_points, CG_BLOCK), dims.nd),
                    dim3(CG_BLOCK), 0, st, D, tol_mode);
}

cudaError_t launch_cg_update(const DomainDesc *D, const BatchDims &dims, int it, double tol,
                             int max_iter, int tol_mode, int confirm, cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  return launch_pdl(cg_update_kernel, dim3(nblk(dims.max_points, CG_BLOCK), dims.nd),
                    dim3(CG_BLOCK), 0, st, D, it, tol, max_iter, tol_mode, confirm);
}

cudaError_t launch_brick_norm(const DomainDesc *D, const BatchDims &dims, int which,
                              cudaStream_t st) {
  return dims.work_off ? launch_pdl(brick_norm_kernel<true>, brick_grid(dims), dim3(32), 0, st, D,
                                    which, dims.work_off, dims.nd)
                       : launch_pdl(brick_norm_kernel<false>, brick_grid(dims), dim3(32), 0, st, D,
                                    which, dims.work_off, dims.nd);
}

cudaError_t launch_ibm_den(const DomainDesc *D, const BatchDims &dims, int mode, cudaStream_t st) {
  return launch_pdl(ibm_den_kernel, dim3(RES_BLOCKS, dims.nd), dim3(256), 0, st, D, mode);
}

cudaError_t launch_ibm_check(const DomainDesc *D, const BatchDims &dims, int it, double tol,
                             int max_iter, cudaStream_t st) {
  return launch_pdl(ibm_check_kernel, dim3(RES_BLOCKS, dims.nd), dim3(256), 0, st, D, it, tol,
                    max_iter);
}


cudaError_t launch_point_residual0(const DomainDesc *D, const BatchDims &dims, cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int pb = dims.ls.point_block;
  return launch_pdl(point_residual0_kernel, dim3(nblk(dims.max_points, pb), dims.nd), dim3(pb), 0,
                    st, D);
}

cudaError_t launch_mlp_features(const DomainDesc *D, const BatchDims &dims, int use_prev,
                                cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int pb = dims.ls.point_block;
  return launch_pdl(mlp_features_kernel, dim3(nblk(dims.max_points, pb), dims.nd), dim3(pb), 0, st,
                    D, use_prev);
}

cudaError_t launch_mlp_targets(int64_t np, const float *X, const float4 *du, float *T,
                               cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  mlp_targets_kernel<<<nblk(np, 256), 256, 0, st>>>(np, X, du, T);
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

cudaError_t launch_store_desc(const DomainDesc &dd, DomainDesc *D, cudaStream_t st) {
  store_desc_kernel<<<1, 32, 0, st>>>(dd, D);
  return cudaGetLastError();
}

cudaError_t launch_slots_to_dense(const Geometry &g, const BrickMap &m, const float *Gs,
                                  float *F, cudaStream_t st) {
  slots_to_dense_kernel<<<PERSISTENT_BLOCKS, 64, 0, st>>>(g, m, Gs, F);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(int64_t n, const float4 *a, float *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl(pack_points_kernel, dim3(nblk(n, 256)), dim3(256), 0, st, n, a, out);
}

// n doubles from device memory to o (device or device-mapped host memory).
__global__ void copy_f64_kernel(int64_t n, const double *__restrict__ a, double *__restrict__ o) {
  pdl_wait();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) o[k] = a[k];
}

cudaError_t launch_copy_f64(int64_t n, const double *a, double *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl(copy_f64_kernel, dim3(nblk(n, 256)), dim3(256), 0, st, n, a, out);
}

}  // namespace lbmibm
