// Lattice Boltzmann kernels (Sec. 2): the fused pull-stream + BGK collision
// with the IBM force, moments on the active bricks, read-out kernels and the
// FP64 reduction of the global sums.
//
// Populations are stored structure-of-arrays, f[i][z][y][x], as deviations
// d_i = f_i - t_i in FP32, BF16 or FP16; all arithmetic is FP32.  Streaming
// is a pull: the kernel for step t reads d_i(X - e_i) from the source lattice
// (post-collision values of step t-1), which realises Eq. 4, and writes the
// post-collision value at X into the destination lattice, so every write is
// coalesced and each population is read and written exactly once per step.
// The FP64 mass and momentum need no sum over the 19 new values: the BGK
// collision conserves mass and adds exactly the force impulse rho G, so a
// cell's post-collision sums are rho and rho U + rho G from its moments.
#include <algorithm>

#include "kernels.h"
#include "lattice.cuh"

namespace lbmibm {

namespace {

// Arithmetic of the collision on one cell (float) or on two cells at once
// (float2, the packed FP32 instructions of this architecture): every operation
// is written out with explicit rounding (no contraction or reordering by the
// compiler), and each packed operation computes exactly the scalar one in
// each lane, so one-cell and two-cell kernels give bitwise the same values.
template <typename V>
__device__ __forceinline__ V vsplat(float a);
template <>
__device__ __forceinline__ float vsplat<float>(float a) {
  return a;
}
template <>
__device__ __forceinline__ float2 vsplat<float2>(float a) {
  return make_float2(a, a);
}
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// 1 / a by the approximate reciprocal instruction (at most one ulp from the
// rounded quotient; the same instruction in the one-cell and two-cell forms)
__device__ __forceinline__ float vrcp(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
// The packed operations in PTX with an explicit rounding mode: the code
// generator neither fuses nor reorders them (the packed intrinsics were
// fused, a multiply and a following add becoming one fma, which rounds
// once where the scalar form rounds twice).
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "add.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(vrcp(a.x), vrcp(a.y)); }
// j += e a for a component e of a direction in {-1, 0, 1}; the first term
// initialises j
template <typename V>
__device__ __forceinline__ void vacc(V &j, bool &first, int e, V a) {
  if (!e) return;
  if (first) j = e > 0 ? a : vsub(vsplat<V>(0.f), a);
  else j = e > 0 ? vadd(j, a) : vsub(j, a);
  first = false;
}

// The collision of one cell (V = float) or of two cells (V = float2) from its
// pulled deviations d (Eq. 4): Eq. 1 moments, U^G = U + tau G (Sec. 2 step 3)
// and the BGK relaxation towards Eq. 3 (om = 1 / tau), into dn.  G is the
// cell's force (body force plus its brick's IBM force).  st receives the
// cell's post-collision mass and momentum sums (the collision conserves mass
// and adds rho G of momentum, Eqs. 2-3, so they follow from the moments).
template <typename V>
__device__ __forceinline__ void collide_core(const V d[Q], V Gx, V Gy, V Gz, float tau,
                                             float om, V dn[Q], V st[4]) {
  // Eq. 1 in deviation form over the pairs of opposite directions (i, i + 1):
  // the pair's sum goes into the density, its difference times e_i into the
  // momentum (27 packed additions where the sums over single directions take
  // 48)
  V drho = d[0], jx = vsplat<V>(0.f), jy = vsplat<V>(0.f), jz = vsplat<V>(0.f);
  bool fx = true, fy = true, fz = true;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const V s = vadd(d[i], d[i + 1]), a = vsub(d[i], d[i + 1]);
    drho = vadd(drho, s);
    vacc(jx, fx, ex(i), a);
    vacc(jy, fy, ey(i), a);
    vacc(jz, fz, ez(i), a);
  }
  const V rho = vadd(vsplat<V>(1.f), drho);
  const V inv = vrcp(rho);
  const V vt = vsplat<V>(tau);
  const V ux = vfma(vt, Gx, vmul(jx, inv));
  const V uy = vfma(vt, Gy, vmul(jy, inv));
  const V uz = vfma(vt, Gz, vmul(jz, inv));
  st[0] = drho;
  st[1] = vfma(rho, Gx, jx);
  st[2] = vfma(rho, Gy, jy);
  st[3] = vfma(rho, Gz, jz);
  // Eq. 3 minus t_i: t_i (c0 + rho (3 e.u + 4.5 (e.u)^2)) with c0 the part
  // common to every direction; opposite directions share 4.5 rho (e.u)^2.
  // Every product that meets an addition is one fma (no separate multiply
  // and add that the code generator could contract in one form and not the
  // other): the relaxation is d + om (t_i E - d) with t_i E - d one fma.
  const V usq = vfma(uz, uz, vfma(uy, uy, vmul(ux, ux)));
  const V c0 = vfma(vmul(vsplat<V>(-1.5f), rho), usq, drho);
  const V r3 = vmul(vsplat<V>(3.f), rho), r45 = vmul(vsplat<V>(4.5f), rho);
  const V nr3 = vmul(vsplat<V>(-3.f), rho);
  // d + om (t_i E - d) as d - om (d - t_i E): negating both factors of the
  // outer product and the inner fma's result leaves every rounding as it was
  // (round-to-nearest is odd), and the packed form then needs no negated
  // copy of d
  const V nom = vsplat<V>(-om);
  dn[0] = vfma(nom, vfma(vsplat<V>(-wt(0)), c0, d[0]), d[0]);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    // e_i . u with the components of e_i in {-1, 0, 1}
    V eu = vsplat<V>(0.f);
    bool first = true;
    const V uc[3] = {ux, uy, uz};
    const int ec[3] = {ex(i), ey(i), ez(i)};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      if (!ec[c]) continue;
      if (first) eu = ec[c] > 0 ? uc[c] : vsub(vsplat<V>(0.f), uc[c]);
      else eu = ec[c] > 0 ? vadd(eu, uc[c]) : vsub(eu, uc[c]);
      first = false;
    }
    const V sym = vfma(r45, vmul(eu, eu), c0);
    const V ep = vfma(r3, eu, sym), em = vfma(nr3, eu, sym);  // E/t_i for e_i and -e_i
    const V nw = vsplat<V>(-wt(i));
    dn[i] = vfma(nom, vfma(nw, ep, d[i]), d[i]);
    dn[i + 1] = vfma(nom, vfma(nw, em, d[i + 1]), d[i + 1]);
  }
}

__device__ __forceinline__ void collide_math(const float d[Q], float Gx, float Gy, float Gz,
                                             float tau, float om, float dn[Q], float st[4]) {
  collide_core<float>(d, Gx, Gy, Gz, tau, om, dn, st);
}

// Two cells a, b at once with the packed instructions; bitwise two calls of
// collide_math.
__device__ __forceinline__ void collide_math2(const float da[Q], const float db[Q],
                                              const float Ga[3], const float Gb[3], float tau,
                                              float om, float dna[Q], float dnb[Q], float sta[4],
                                              float stb[4]) {
  float2 d[Q], dn[Q], st[4];
#pragma unroll
  for (int i = 0; i < Q; i++) d[i] = make_float2(da[i], db[i]);
  collide_core<float2>(d, make_float2(Ga[0], Gb[0]), make_float2(Ga[1], Gb[1]),
                       make_float2(Ga[2], Gb[2]), tau, om, dn, st);
#pragma unroll
  for (int i = 0; i < Q; i++) {
    dna[i] = dn[i].x;
    dnb[i] = dn[i].y;
  }
#pragma unroll
  for (int c = 0; c < 4; c++) {
    sta[c] = st[c].x;
    stb[c] = st[c].y;
  }
}

// One cell of the fused pull-stream + collision: the pull of Eq. 4 from src,
// collide_math, and the post-collision values written to dst at n.
template <typename S>
__device__ __forceinline__ void collide_cell(const S *__restrict__ src, S *__restrict__ dst,
                                             const Geometry &g, uint32_t n, int x, int y, int z,
                                             float Gx, float Gy, float Gz, float tau,
                                             float om, float st[4]) {
  float d[Q], dn[Q];
  pull<S, false, true>(src, g, x, y, z, d);
  collide_math(d, Gx, Gy, Gz, tau, om, dn, st);
  const size_t N = (size_t)g.ncell;
#pragma unroll
  for (int i = 0; i < Q; i++) Store<S>::st(dst + ((size_t)i * N + n), dn[i]);
}

// Warp sums of four values in 6 shuffles: the first exchange splits the
// components between the two half-warps (lanes with bit 4 keep 2, 3), the
// second between the quarter-warps (bit 3), then three exchanges finish one
// component per lane.  Lane l returns the sum of component
// ((l >> 4) & 1) * 2 + ((l >> 3) & 1): lanes 0, 8, 16 and 24 hold 0..3.
__device__ __forceinline__ float warp_sum4_split(const float a[4]) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  const float s0 = h16 ? a[0] : a[2], s1 = h16 ? a[1] : a[3];
  const float k0 = h16 ? a[2] : a[0], k1 = h16 ? a[3] : a[1];
  const float b0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
  const float b1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
  float c = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// One thread per cell.  dd is the domain of this block: a kernel parameter
// for a single lattice (constant bank, no dependent loads before the first
// population load), or a batch's domain from its block table; bx is the
// block's index within the domain.  SKIP: the cells of the
// step's active bricks are left to collide_active_kernel (they need the IBM
// force, the others do not); otherwise every cell, with its brick's force.
template <typename S, bool STATS, bool SKIP>
__device__ __forceinline__ void collide_stream_cells(const DomainDesc &dd, int cur,
                                                     uint32_t bx) {
  const Geometry g = dd.g;
  // blocks past this domain's cells (batches of unequal domains) leave at once
  if ((int64_t)bx * blockDim.x >= g.ncell) return;
  const S *__restrict__ src = (const S *)dd.f[cur];
  S *__restrict__ dst = (S *)dd.f[cur ^ 1];
  const int *__restrict__ brick_slot = dd.np > 0 ? dd.m.brick_slot : nullptr;
  const int nact = SKIP && brick_slot ? active_slots(dd.m) : 0;
  const float *__restrict__ Gs = dd.Gs;
  double *__restrict__ partial = dd.partial;
  float sv[4] = {0.f, 0.f, 0.f, 0.f};
  const uint32_t n = bx * blockDim.x + threadIdx.x;
  if (n < (uint32_t)g.ncell) {
    int x, y, z;
    cell_coords(n, g, x, y, z);
    float Gx = dd.gbody[0], Gy = dd.gbody[1], Gz = dd.gbody[2];
    bool mine = true;
    if (brick_slot) {
      const int b = ((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2);
      const int s = __ldg(brick_slot + b);
      if (SKIP) {
        mine = !(s >= 0 && s < nact);
      } else if (s >= 0) {
        const float *p = Gs + (size_t)s * SLOT_FLOATS + brick_local(x, y, z);
        Gx += __ldg(p);
        Gy += __ldg(p + BRICK_CELLS);
        Gz += __ldg(p + 2 * BRICK_CELLS);
      }
    }
    if (mine) {
      float st[4];
      collide_cell<S>(src, dst, g, n, x, y, z, Gx, Gy, Gz, dd.tau, dd.om, st);
      if (STATS)
        for (int c = 0; c < 4; c++) sv[c] = st[c];
    }
  }
  if (STATS) {
    const float ws = warp_sum4_split(sv);
    // one partial per PARTIAL_CELLS cells (four warps), whatever the block
    // size: the sums do not depend on the launch shape
    __shared__ double red[8][4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((lane & 7) == 0) red[w][lane >> 3] = ws;
    __syncthreads();
    const int groups = blockDim.x / PARTIAL_CELLS;
    if ((int)threadIdx.x < 4 * groups) {
      const int gi = threadIdx.x >> 2, c = threadIdx.x & 3;
      const double a = ((red[4 * gi][c] + red[4 * gi + 1][c]) + red[4 * gi + 2][c]) +
                       red[4 * gi + 3][c];
      const int64_t pidx = (int64_t)bx * groups + gi;
      if (pidx < dd.cblocks) partial[(size_t)pidx * 4 + c] = a;
    }
  }
}

template <typename S, bool STATS, bool SKIP>
__global__ void __launch_bounds__(256)
    collide_stream_kernel(const __grid_constant__ DomainDesc dd, int cur) {
  pdl_wait();
  collide_stream_cells<S, STATS, SKIP>(dd, cur, blockIdx.x);
}

// (five blocks of 256 per SM, as the single-lattice kernel gets with its
// descriptor in the parameter bank)
template <typename S, bool STATS, bool SKIP>
__global__ void __launch_bounds__(256, 5)
    collide_stream_batch_kernel(const DomainDesc *__restrict__ D, const int2 *__restrict__ blk,
                                int cur) {
  pdl_wait();
  const int2 e = blk[blockIdx.x];
  collide_stream_cells<S, STATS, SKIP>(D[e.x], cur, e.y);
}

// 16-bit storage: two x-neighbouring cells (x0 even, x0 + 1) per thread.
// The pulls are 32-bit words of two deviations: directions without an x
// component read one word (the two cells' values), the others the two words
// holding x0 - 1 and x0 (e_x = +1) or x0 + 1 and x0 + 2 (e_x = -1); each
// direction's two results go out as one word.  Rows, the brick's force and
// the stats are shared by the two cells; each cell's arithmetic is
// collide_math, so the results are those of collide_stream_cells.
template <typename S>
struct Word16;
template <>
struct Word16<__nv_bfloat16> {
  static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
  static __device__ __forceinline__ float hi(uint32_t w) {
    return __uint_as_float(w & 0xffff0000u);
  }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
  }
};
template <>
struct Word16<__half> {
  static __device__ __forceinline__ float lo(uint32_t w) {
    return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
  }
  static __device__ __forceinline__ float hi(uint32_t w) {
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
  }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
  }
};

template <typename S, bool STATS>
__device__ __forceinline__ void collide_pairs16(const DomainDesc &dd, int cur, uint32_t bx) {
  const Geometry g = dd.g;
  if ((int64_t)bx * blockDim.x * 2 >= g.ncell) return;
  const uint32_t *__restrict__ src = (const uint32_t *)dd.f[cur];
  uint32_t *__restrict__ dst = (uint32_t *)dd.f[cur ^ 1];
  const int *__restrict__ brick_slot = dd.np > 0 ? dd.m.brick_slot : nullptr;
  const float *__restrict__ Gs = dd.Gs;
  float sv[4] = {0.f, 0.f, 0.f, 0.f};
  const uint32_t n = 2 * (bx * blockDim.x + threadIdx.x);
  if (n < (uint32_t)g.ncell) {
    int x, y, z;
    cell_coords(n, g, x, y, z);
    float Ga[3] = {dd.gbody[0], dd.gbody[1], dd.gbody[2]};
    float Gb[3] = {Ga[0], Ga[1], Ga[2]};
    if (brick_slot) {
      const int b = ((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2);
      const int sl = __ldg(brick_slot + b);
      if (sl >= 0) {
        const float *p = Gs + (size_t)sl * SLOT_FLOATS + brick_local(x, y, z);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          Ga[c] += __ldg(p + c * BRICK_CELLS);
          Gb[c] += __ldg(p + c * BRICK_CELLS + 1);
        }
      }
    }
    // word offsets of the rows y - e_y, z - e_z and of x0 - 2, x0, x0 + 2
    const uint32_t nx = g.nx, ny = g.ny, hw = nx >> 1;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == (int)ny - 1 ? 0 : y + 1;
    const uint32_t zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    const uint32_t Y[3] = {yp, (uint32_t)y, ym}, Z[3] = {zp, (uint32_t)z, zm};
    const uint32_t w0 = (uint32_t)x >> 1;
    const uint32_t wl = w0 == 0 ? hw - 1 : w0 - 1, wr = w0 == hw - 1 ? 0 : w0 + 1;
    const size_t NW = (size_t)g.ncell >> 1;
    float da[Q], db[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const uint32_t row = (Z[ez(i) + 1] * ny + Y[ey(i) + 1]) * hw;
      const uint32_t *fi = src + (size_t)i * NW + row;
      if (ex(i) == 0) {
        const uint32_t w = ldw_stream(fi + w0);
        da[i] = Word16<S>::lo(w);
        db[i] = Word16<S>::hi(w);
      } else if (ex(i) > 0) {
        da[i] = Word16<S>::hi(ldw_stream(fi + wl));
        db[i] = Word16<S>::lo(ldw_stream(fi + w0));
      } else {
        da[i] = Word16<S>::hi(ldw_stream(fi + w0));
        db[i] = Word16<S>::lo(ldw_stream(fi + wr));
      }
    }
    float dna[Q], dnb[Q], sta[4], stb[4];
    collide_math2(da, db, Ga, Gb, dd.tau, dd.om, dna, dnb, sta, stb);
    const uint32_t wn = n >> 1;
#pragma unroll
    for (int i = 0; i < Q; i++) dst[(size_t)i * NW + wn] = Word16<S>::pack(dna[i], dnb[i]);
    if (STATS)
      for (int c = 0; c < 4; c++) sv[c] = sta[c] + stb[c];
  }
  if (STATS) {
    const float ws = warp_sum4_split(sv);
    // a warp covers 64 cells: one partial per PARTIAL_CELLS = two warps
    __shared__ double red[8][4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((lane & 7) == 0) red[w][lane >> 3] = ws;
    __syncthreads();
    const int groups = blockDim.x / (PARTIAL_CELLS / 2);
    if ((int)threadIdx.x < 4 * groups) {
      const int gi = threadIdx.x >> 2, c = threadIdx.x & 3;
      const double a = red[2 * gi][c] + red[2 * gi + 1][c];
      const int64_t pidx = (int64_t)bx * groups + gi;
      if (pidx < dd.cblocks) dd.partial[(size_t)pidx * 4 + c] = a;
    }
  }
}

// (at most 64 registers, four blocks of 256 per SM: the kernel is bound by the
// latency of its loads, and the extra warps pay for the few spilled values:
// 0.815 against 0.776 of the copy bandwidth at 75 registers; at 48 registers
// the spills dominate, 0.65)
template <typename S, bool STATS>
__global__ void __launch_bounds__(256, 4)
    collide_pairs16_kernel(const __grid_constant__ DomainDesc dd, int cur) {
  pdl_wait();
  collide_pairs16<S, STATS>(dd, cur, blockIdx.x);
}

template <typename S, bool STATS>
__global__ void __launch_bounds__(256, 4)
    collide_pairs16_batch_kernel(const DomainDesc *__restrict__ D, const int2 *__restrict__ blk,
                                 int cur) {
  pdl_wait();
  const int2 e = blk[blockIdx.x];
  collide_pairs16<S, STATS>(D[e.x], cur, e.y);
}

// 16-bit storage: four x-neighbouring cells (x0 a multiple of 4, so one
// brick) per thread, as two packed pairs A = (x0, x0 + 1) and
// B = (x0 + 2, x0 + 3).  A direction's pulls are the two words at x0 / 2 of
// its source row (one 8-byte load) and, for e_x = +1 / -1, the word before /
// after them; byte permutes assemble each pair's word of two deviations,
// which the pair reads as collide_pairs16 reads its words, and the two
// pairs' results leave as one 8-byte store per direction.  A warp covers the
// 128 cells of one FP64 partial and sums them in collide_pairs16's FP32 tree
// (pair q meets q ^ 16, q ^ 8, ..., q ^ 1; pairs 2L and 2L + 1 sit in lane L,
// so the lane exchanges are 8, 4, 2, 1 and the last level is within the
// lane): populations and sums are bitwise those of the two-cell kernel.
__device__ __forceinline__ uint2 ldw2_stream(const uint32_t *p) {
  uint2 v;
  asm("ld.global.nc.L2::256B.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

template <typename S>
__device__ __forceinline__ void pair_words(const uint32_t w[Q], const float Ga[3],
                                           const float Gb[3], float tau, float om,
                                           uint32_t r[Q], float sv[4]) {
  float da[Q], db[Q], dna[Q], dnb[Q], sta[4], stb[4];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    da[i] = Word16<S>::lo(w[i]);
    db[i] = Word16<S>::hi(w[i]);
  }
  collide_math2(da, db, Ga, Gb, tau, om, dna, dnb, sta, stb);
#pragma unroll
  for (int i = 0; i < Q; i++) r[i] = Word16<S>::pack(dna[i], dnb[i]);
#pragma unroll
  for (int c = 0; c < 4; c++) sv[c] = sta[c] + stb[c];
}

template <typename S, bool STATS>
__device__ __forceinline__ void collide_quads16(const DomainDesc &dd, int cur, uint32_t bx) {
  const Geometry g = dd.g;
  if ((int64_t)bx * blockDim.x * 4 >= g.ncell) return;
  const uint32_t *__restrict__ src = (const uint32_t *)dd.f[cur];
  uint32_t *__restrict__ dst = (uint32_t *)dd.f[cur ^ 1];
  const int *__restrict__ brick_slot = dd.np > 0 ? dd.m.brick_slot : nullptr;
  float vA[4] = {0.f, 0.f, 0.f, 0.f}, vB[4] = {0.f, 0.f, 0.f, 0.f};
  const uint32_t n = 4 * (bx * blockDim.x + threadIdx.x);
  if (n < (uint32_t)g.ncell) {
    int x, y, z;
    cell_coords(n, g, x, y, z);
    float G[4][3];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int c = 0; c < 3; c++) G[k][c] = dd.gbody[c];
    if (brick_slot) {
      const int b = ((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2);
      const int sl = __ldg(brick_slot + b);
      if (sl >= 0) {
        const float *p = dd.Gs + (size_t)sl * SLOT_FLOATS + brick_local(x, y, z);
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
          for (int c = 0; c < 3; c++) G[k][c] += __ldg(p + c * BRICK_CELLS + k);
      }
    }
    // word offsets of the rows y - e_y, z - e_z and of x0 - 2, x0, x0 + 4
    const uint32_t ny = g.ny, hw = (uint32_t)g.nx >> 1;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == (int)ny - 1 ? 0 : y + 1;
    const uint32_t zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    const uint32_t Y[3] = {yp, (uint32_t)y, ym}, Z[3] = {zp, (uint32_t)z, zm};
    const uint32_t w0 = (uint32_t)x >> 1;
    const uint32_t wl = w0 == 0 ? hw - 1 : w0 - 1, wr = w0 + 2 == hw ? 0 : w0 + 2;
    const size_t NW = (size_t)g.ncell >> 1;
    uint32_t wa[Q], wb[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const uint32_t row = (Z[ez(i) + 1] * ny + Y[ey(i) + 1]) * hw;
      const uint32_t *fi = src + (size_t)i * NW + row;
      const uint2 m = ldw2_stream(fi + w0);
      if (ex(i) == 0) {
        wa[i] = m.x;
        wb[i] = m.y;
      } else if (ex(i) > 0) {
        // cells x0 - 1 .. x0 + 2: the high half of each word, then the low
        // half of the next
        wa[i] = __byte_perm(ldw_stream(fi + wl), m.x, 0x5432);
        wb[i] = __byte_perm(m.x, m.y, 0x5432);
      } else {
        // cells x0 + 1 .. x0 + 4
        wa[i] = __byte_perm(m.x, m.y, 0x5432);
        wb[i] = __byte_perm(m.y, ldw_stream(fi + wr), 0x5432);
      }
    }
    const uint32_t wn = n >> 1;
    uint32_t ra[Q], rb[Q];
    pair_words<S>(wa, G[0], G[1], dd.tau, dd.om, ra, vA);
    pair_words<S>(wb, G[2], G[3], dd.tau, dd.om, rb, vB);
#pragma unroll
    for (int i = 0; i < Q; i++)
      *reinterpret_cast<uint2 *>(dst + (size_t)i * NW + wn) = make_uint2(ra[i], rb[i]);
  }
  if (STATS) {
    const int lane = threadIdx.x & 31;
    const bool h8 = lane & 8, h4 = lane & 4;
    // pair q ^ 16 (lane ^ 8): the half-warps' lanes with bit 3 keep
    // components 2, 3
    const float bA0 = (h8 ? vA[2] : vA[0]) + __shfl_xor_sync(0xffffffffu, h8 ? vA[0] : vA[2], 8);
    const float bA1 = (h8 ? vA[3] : vA[1]) + __shfl_xor_sync(0xffffffffu, h8 ? vA[1] : vA[3], 8);
    const float bB0 = (h8 ? vB[2] : vB[0]) + __shfl_xor_sync(0xffffffffu, h8 ? vB[0] : vB[2], 8);
    const float bB1 = (h8 ? vB[3] : vB[1]) + __shfl_xor_sync(0xffffffffu, h8 ? vB[1] : vB[3], 8);
    // q ^ 8 (lane ^ 4): lanes with bit 2 keep the second of the two
    float cA = (h4 ? bA1 : bA0) + __shfl_xor_sync(0xffffffffu, h4 ? bA0 : bA1, 4);
    float cB = (h4 ? bB1 : bB0) + __shfl_xor_sync(0xffffffffu, h4 ? bB0 : bB1, 4);
    // q ^ 4, q ^ 2 (lane ^ 2, lane ^ 1), then q ^ 1 within the lane
    cA += __shfl_xor_sync(0xffffffffu, cA, 2);
    cB += __shfl_xor_sync(0xffffffffu, cB, 2);
    cA += __shfl_xor_sync(0xffffffffu, cA, 1);
    cB += __shfl_xor_sync(0xffffffffu, cB, 1);
    const float c = cA + cB;
    // lanes 0, 4, 8, 12 hold components 0..3 of the first 64 cells, lanes
    // 16.. the same of the next 64; the partial is their FP64 sum
    const float o = __shfl_down_sync(0xffffffffu, c, 16);
    const int64_t pidx = ((int64_t)bx * blockDim.x + threadIdx.x) >> 5;
    if (lane < 16 && (lane & 3) == 0 && pidx < dd.cblocks)
      dd.partial[(size_t)pidx * 4 + (lane >> 2)] = (double)c + (double)o;
  }
}

// (at most 96 registers, five blocks of 128 per SM: 0.905 of the copy
// bandwidth at 384^3 against 0.851 at 128 registers (four blocks) and 0.744
// at 80 (six blocks, where the spills dominate))
template <typename S, bool STATS>
__global__ void __launch_bounds__(128, 5)
    collide_quads16_kernel(const __grid_constant__ DomainDesc dd, int cur) {
  pdl_wait();
  collide_quads16<S, STATS>(dd, cur, blockIdx.x);
}

template <typename S, bool STATS>
__global__ void __launch_bounds__(128, 5)
    collide_quads16_batch_kernel(const DomainDesc *__restrict__ D, const int2 *__restrict__ blk,
                                 int cur) {
  pdl_wait();
  const int2 e = blk[blockIdx.x];
  collide_quads16<S, STATS>(D[e.x], cur, e.y);
}

// 16-bit storage, single lattice: the pulls staged in shared memory by the
// bulk-copy engine.  A tile is R consecutive rows (y) of one z plane, whole
// rows in x; for each population the R source rows (the tile's rows shifted by
// -e_y, -e_z, wrapped) arrive as at most two contiguous bulk copies
// (cp.async.bulk, global -> shared, completing on the stage's "full"
// mbarrier).  A persistent grid walks the tiles; in each block one producer
// warp keeps NS stages in flight (it refills a stage once every consumer warp
// has arrived on its "empty" mbarrier) and R nx / 2 consumer threads take two
// x-neighbouring cells each, exactly as collide_pairs16 does (the same words,
// the same collide_math2, the same warps of 64 cells and the same FP64 partial
// per 128 cells, formed by the two warps of a pair at a named barrier of
// their own), so the results are bitwise those of collide_pairs16.  No
// block-wide barrier in the steady state.  Needs nx % 8 == 0 (16-byte rows),
// ny % R == 0 and R nx a multiple of 128; the launcher checks.  Every wait is
// bounded: past ROWS_SPIN_LIMIT polls the waiting warp sets bit 8 of the error
// flags and leaves (the producer stops issuing, so the others time out too).
constexpr unsigned ROWS_SPIN_LIMIT = 1u << 24;
constexpr int ROWS_MAX_CONSUMERS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// true once the phase of parity `phase` has completed; false after
// ROWS_SPIN_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase) {
  for (unsigned i = 0; i < ROWS_SPIN_LIMIT; i++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// barrier 1 + pair among the 64 threads of warps 2 pair and 2 pair + 1 (the
// ids are constants, so the block reserves only the barriers it uses)
__device__ __forceinline__ void pair_sync(int pair) {
  switch (pair) {
    case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
  }
}

struct RowsTiling {
  int R;            // rows per tile
  int NS;           // stages
  int tiles;        // nz * ny / R
  int stage_bytes;  // 19 R nx 2
};

// Issues the copies of tile t into stage buffer `buf`: called by the 32
// lanes of the producer warp, lane i < 19 copies population i (lane 0 first
// posts the stage's byte count).
__device__ __forceinline__ void rows_issue(const uint16_t *__restrict__ f, const Geometry &g,
                                           int R, int t, unsigned char *buf, uint64_t *bar,
                                           unsigned stage_bytes) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_expect_tx(bar, stage_bytes);
  __syncwarp();
  if (lane >= Q) return;
  const int i = lane;
  const int ny = g.ny, nx = g.nx;
  const int z = t / (ny / R), y0 = (t - z * (ny / R)) * R;
  const size_t N = (size_t)g.ncell;
  const unsigned rowb = (unsigned)nx * 2u;
  const int zs = wrapi(z - ez(i), g.nz);
  const int ya = wrapi(y0 - ey(i), ny);
  const int first = min(R, ny - ya);  // rows before the y seam
  unsigned char *d = buf + (size_t)i * R * rowb;
  const uint16_t *src = f + (size_t)i * N + ((size_t)zs * ny + ya) * nx;
  bulk_g2s(d, src, (unsigned)first * rowb, bar);
  if (first < R)
    bulk_g2s(d + (size_t)first * rowb, f + (size_t)i * N + (size_t)zs * ny * nx,
             (unsigned)(R - first) * rowb, bar);
}

template <typename S, bool STATS>
__global__ void __launch_bounds__(ROWS_MAX_CONSUMERS + 32, 2)
    collide_rows16_kernel(const __grid_constant__ DomainDesc dd, int cur, RowsTiling tl) {
  pdl_wait();
  extern __shared__ __align__(128) unsigned char smraw[];
  const int NS = tl.NS, R = tl.R;
  uint64_t *full = reinterpret_cast<uint64_t *>(smraw);
  uint64_t *empty = full + NS;
  unsigned char *stages = smraw + 256;
  __shared__ float red[2][ROWS_MAX_CONSUMERS / 32][4];
  __shared__ int pair_abort[2][ROWS_MAX_CONSUMERS / 64];  // by tile parity
  const Geometry g = dd.g;
  const int nx = g.nx, hw = nx >> 1;
  const int ncons = R * hw, cw = ncons >> 5;  // consumer threads and warps
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint16_t *__restrict__ f = (const uint16_t *)dd.f[cur];
  if (threadIdx.x < ROWS_MAX_CONSUMERS / 32) (&pair_abort[0][0])[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; q++) {
      mbar_init(full + q, 1);
      mbar_init(empty + q, cw);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == cw) {
    // producer: stage q of the k-th tile is refilled once the consumers have
    // released its previous use (the empty phase of use k / NS - 1)
    int k = 0;
    for (int t = blockIdx.x; t < tl.tiles; t += gridDim.x, k++) {
      const int q = k % NS;
      if (k >= NS && !mbar_wait(empty + q, (unsigned)(k / NS - 1) & 1u)) {
        if (lane == 0) atomicOr(dd.m.counters + 5, 8);
        return;
      }
      rows_issue(f, g, R, t, stages + (size_t)q * tl.stage_bytes, full + q,
                 (unsigned)tl.stage_bytes);
    }
    return;
  }
  uint32_t *__restrict__ dst = (uint32_t *)dd.f[cur ^ 1];
  const int *__restrict__ brick_slot = dd.np > 0 ? dd.m.brick_slot : nullptr;
  const float *__restrict__ Gs = dd.Gs;
  const unsigned rowb = (unsigned)nx * 2u;
  const size_t NW = (size_t)g.ncell >> 1;
  const int r = threadIdx.x / hw, j = threadIdx.x - r * hw;  // row, word of this thread
  const int x = 2 * j;
  const uint32_t wl = j == 0 ? hw - 1 : j - 1, wr = j == hw - 1 ? 0 : j + 1;
  const int pair = warp >> 1;
  int k = 0;
  for (int t = blockIdx.x; t < tl.tiles; t += gridDim.x, k++) {
    const int q = k % NS;
    // a wait that gives up marks the pair; both warps of a pair leave after
    // the same pair barrier (so neither is left waiting at it)
    if (!mbar_wait(full + q, (unsigned)(k / NS) & 1u)) {
      if (lane == 0) {
        atomicOr(dd.m.counters + 5, 8);
        pair_abort[k & 1][pair] = 1;
      }
      if (STATS) pair_sync(pair);
      break;
    }
    const int z = t / (g.ny / R), y = (t - z * (g.ny / R)) * R + r;
    const unsigned char *buf = stages + (size_t)q * tl.stage_bytes;
    float da[Q], db[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const uint32_t *row = (const uint32_t *)(buf + ((size_t)i * R + r) * rowb);
      if (ex(i) == 0) {
        const uint32_t w = row[j];
        da[i] = Word16<S>::lo(w);
        db[i] = Word16<S>::hi(w);
      } else if (ex(i) > 0) {
        da[i] = Word16<S>::hi(row[wl]);
        db[i] = Word16<S>::lo(row[j]);
      } else {
        da[i] = Word16<S>::hi(row[j]);
        db[i] = Word16<S>::lo(row[wr]);
      }
    }
    // this warp has read stage q
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + q);
    float Ga[3] = {dd.gbody[0], dd.gbody[1], dd.gbody[2]};
    float Gb[3] = {Ga[0], Ga[1], Ga[2]};
    if (brick_slot) {
      const int b = ((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2);
      const int sl = __ldg(brick_slot + b);
      if (sl >= 0) {
        const float *p = Gs + (size_t)sl * SLOT_FLOATS + brick_local(x, y, z);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          Ga[c] += __ldg(p + c * BRICK_CELLS);
          Gb[c] += __ldg(p + c * BRICK_CELLS + 1);
        }
      }
    }
    float dna[Q], dnb[Q], sta[4], stb[4];
    collide_math2(da, db, Ga, Gb, dd.tau, dd.om, dna, dnb, sta, stb);
    const size_t cell0 = ((size_t)z * g.ny + (y - r)) * nx;  // first cell of the tile
    const uint32_t wn = (uint32_t)((cell0 >> 1) + threadIdx.x);
#pragma unroll
    for (int i = 0; i < Q; i++) dst[(size_t)i * NW + wn] = Word16<S>::pack(dna[i], dnb[i]);
    if (STATS) {
      float sv[4];
      for (int c = 0; c < 4; c++) sv[c] = sta[c] + stb[c];
      const float ws = warp_sum4_split(sv);
      // a warp covers 64 cells: one partial per PARTIAL_CELLS = a pair of
      // warps, which meet at a barrier of their own (red double-buffered by
      // tile, so that the first warp may write the next tile's sums while
      // the second still reads these)
      if ((lane & 7) == 0) red[k & 1][warp][lane >> 3] = ws;
      pair_sync(pair);
      if (pair_abort[k & 1][pair]) break;
      if (!(warp & 1) && lane < 4) {
        const int c = lane;
        const double a = (double)red[k & 1][warp][c] + (double)red[k & 1][warp + 1][c];
        const int64_t pidx = (int64_t)(cell0 / PARTIAL_CELLS) + pair;
        if (pidx < dd.cblocks) dd.partial[(size_t)pidx * 4 + c] = a;
      }
    }
  }
}

// The cells of the active bricks, after the IBM loop: 64 threads per slot
// (one per cell), four slots per block, grid-stride over the slots; the same
// per-cell arithmetic as collide_stream_cells with G = body force + the
// slot's G.  STATS: one FP64 partial per slot (its two warps' FP32 sums).
template <typename S, bool STATS>
__global__ void __launch_bounds__(256)
    collide_active_kernel(const DomainDesc *__restrict__ D, int cur) {
  pdl_wait();
  const DomainDesc &dd = D[blockIdx.y];
  if (dd.np <= 0) return;
  const Geometry g = dd.g;
  const S *__restrict__ src = (const S *)dd.f[cur];
  S *__restrict__ dst = (S *)dd.f[cur ^ 1];
  const float *__restrict__ Gs = dd.Gs;
  const BrickMap m = dd.m;
  const int nact = active_slots(m);
  __shared__ float red[8][4];
  const int t = threadIdx.x & 63, w = threadIdx.x >> 5;
  // (every thread of a block takes the same number of trips)
  for (int s0 = blockIdx.x * 4; s0 < nact; s0 += gridDim.x * 4) {
    const int s = s0 + (threadIdx.x >> 6);
    float sv[4] = {0.f, 0.f, 0.f, 0.f};
    if (s < nact) {
      const int B = m.slot_brick[s];
      const int bx = B % g.nbx, rr = B / g.nbx;
      const int by = rr % g.nby, bz = rr / g.nby;
      const int x = bx * 4 + (t & 3), y = by * 4 + ((t >> 2) & 3), z = bz * 4 + (t >> 4);
      const uint32_t n = (uint32_t)(((size_t)z * g.ny + y) * g.nx + x);
      const float *p = Gs + (size_t)s * SLOT_FLOATS + t;
      float st[4];
      collide_cell<S>(src, dst, g, n, x, y, z, dd.gbody[0] + p[0],
                      dd.gbody[1] + p[BRICK_CELLS], dd.gbody[2] + p[2 * BRICK_CELLS], dd.tau, dd.om,
                      st);
      if (STATS)
        for (int c = 0; c < 4; c++) sv[c] = st[c];
    }
    if (STATS) {
      const float ws = warp_sum4_split(sv);
      const int lane = threadIdx.x & 31;
      if ((lane & 7) == 0) red[w][lane >> 3] = ws;
      __syncthreads();
      if ((threadIdx.x & 63) < 4) {
        const int c = threadIdx.x & 3, q = threadIdx.x >> 6;
        if (s < nact)
          dd.slot_partial[(size_t)s * 4 + c] = (double)red[2 * q][c] + (double)red[2 * q + 1][c];
      }
      __syncthreads();
    }
  }
}

// End of a step: the FP64 sum of the collide kernel's partials in a fixed
// order, and t += 1.  A domain with P partials takes nb = min(FINISH_MAX,
// ceil(P / 1024)) blocks of 256 threads, a function of its own size only (a
// domain sums the same way alone or in a batch): thread j of block b adds the
// partials b*256 + j + k*nb*256 in k order, the block adds its threads' sums
// in a fixed tree, and the last block to finish adds the nb block sums with
// the same tree (split: the active bricks' slot partials follow the cells'
// partials in the index range).  FP64 arithmetic is slow on this part, so each partial is
// added once and the trees use few warp instructions.  With stats off only the
// step counter advances.
constexpr int FINISH_MAX = 128;

__host__ __device__ __forceinline__ int finish_blocks(int partials) {
  const int nb = (partials + 1023) / 1024;
  return nb < 1 ? 1 : (nb > FINISH_MAX ? FINISH_MAX : nb);
}

// red[c][0] = sum of red[c][0..256) for c < 4 (pairwise tree, fixed order);
// every thread of the block calls it
__device__ __forceinline__ void block_tree4(double (*red)[256]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int o = 128; o > 0; o >>= 1) {
    __syncthreads();
    if (t < o)
#pragma unroll
      for (int c = 0; c < 4; c++) red[c][t] += red[c][t + o];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) finish_step_kernel(const DomainDesc *__restrict__ D,
                                                          int stats, int split) {
  pdl_wait();
  const DomainDesc &dd = D[blockIdx.y];
  if (!stats) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *dd.t += 1;
    return;
  }
  // the partials of the cells, then (split) those of the active bricks
  const int P0 = dd.cblocks, nb = finish_blocks(P0);
  if ((int)blockIdx.x >= nb) return;
  const int P = P0 + (split && dd.np > 0 ? active_slots(dd.m) : 0);
  const double4_32a *__restrict__ sp = (const double4_32a *)dd.slot_partial;
  __shared__ double red[4][256];
  __shared__ bool last;
  const int t = threadIdx.x;
  const double4_32a *__restrict__ partial = (const double4_32a *)dd.partial;
  double a[4] = {0, 0, 0, 0};
  const int stride = nb * 256;
  int p = blockIdx.x * 256 + t;
  // four loads in flight per trip; the adds stay in k order
  for (; p + 3 * stride < P; p += 4 * stride) {
    double4_32a v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int q = p + k * stride;
      v[k] = q < P0 ? partial[q] : sp[q - P0];
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      a[0] += v[k].x;
      a[1] += v[k].y;
      a[2] += v[k].z;
      a[3] += v[k].w;
    }
  }
  for (; p < P; p += stride) {
    const double4_32a v = p < P0 ? partial[p] : sp[p - P0];
    a[0] += v.x;
    a[1] += v.y;
    a[2] += v.z;
    a[3] += v.w;
  }
#pragma unroll
  for (int c = 0; c < 4; c++) red[c][t] = a[c];
  block_tree4(red);
  if (t < 4) {
    dd.red_scratch[blockIdx.x * 4 + t] = red[t][0];
    __threadfence();
  }
  __syncthreads();
  if (t == 0) last = atomicAdd(dd.ticket, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int c = 0; c < 4; c++) red[c][t] = t < nb ? __ldcg(dd.red_scratch + t * 4 + c) : 0.0;
  block_tree4(red);
  if (t < 4) dd.sums[t] = t == 0 ? (double)dd.g.ncell + red[0][0] : red[t][0];
  if (t == 0) {
    *dd.ticket = 0u;
    *dd.t += 1;
  }
}

template <typename S>
__global__ void __launch_bounds__(256)
    moments_dense_kernel(const S *__restrict__ f, Geometry g, float *__restrict__ rho,
                         float *__restrict__ U) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (uint32_t)g.ncell) return;
  int x, y, z;
  cell_coords(n, g, x, y, z);
  float d[Q];
  pull<S>(f, g, x, y, z, d);
  float drho, jx, jy, jz;
  moments(d, drho, jx, jy, jz);
  const float r = 1.f + drho, inv = 1.f / r;
  if (rho) rho[n] = r;
  if (U) {
    const size_t N = (size_t)g.ncell;
    U[n] = jx * inv;
    U[N + n] = jy * inv;
    U[2 * N + n] = jz * inv;
  }
}

template <typename S>
__global__ void read_pop_kernel(const S *__restrict__ f, Geometry g, float *__restrict__ out,
                                int deviations) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (uint32_t)g.ncell) return;
  int x, y, z;
  cell_coords(n, g, x, y, z);
  float d[Q];
  pull<S>(f, g, x, y, z, d);
  const size_t N = (size_t)g.ncell;
#pragma unroll
  for (int i = 0; i < Q; i++) out[(size_t)i * N + n] = deviations ? d[i] : wt(i) + d[i];
}

// inverse of the pull: stored_i(X) = f_i(X + e_i) - t_i
template <typename S>
__global__ void write_pop_kernel(const float *__restrict__ in, Geometry g, S *__restrict__ f) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (uint32_t)g.ncell) return;
  int x, y, z;
  cell_coords(n, g, x, y, z);
  const size_t N = (size_t)g.ncell;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int xs = wrapi(x + ex(i), g.nx), ys = wrapi(y + ey(i), g.ny),
              zs = wrapi(z + ez(i), g.nz);
    const size_t src = ((size_t)zs * g.ny + ys) * g.nx + xs;
    Store<S>::st(f + (size_t)i * N + n, in[(size_t)i * N + src] - wt(i));
  }
}

__global__ void force_dense_kernel(Geometry g, const int *__restrict__ brick_slot,
                                   const float *__restrict__ Gs, float gx, float gy, float gz,
                                   float *__restrict__ G) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (uint32_t)g.ncell) return;
  int x, y, z;
  cell_coords(n, g, x, y, z);
  float a = gx, b = gy, c = gz;
  if (brick_slot) {
    const int s = brick_slot[((z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2)];
    if (s >= 0) {
      const float *p = Gs + (size_t)s * SLOT_FLOATS + brick_local(x, y, z);
      a += p[0];
      b += p[BRICK_CELLS];
      c += p[2 * BRICK_CELLS];
    }
  }
  const size_t N = (size_t)g.ncell;
  G[n] = a;
  G[N + n] = b;
  G[2 * N + n] = c;
}

inline unsigned cell_blocks(const Geometry &g, int threads) {
  return (unsigned)((g.ncell + threads - 1) / threads);
}

// Tiling of the staged 16-bit collide: R the largest divisor of ny with
// R nx / 2 <= 256 consumer threads and R nx a multiple of 128 cells; as many
// stages (up to 8) as fit in ~74 KB (three blocks per SM), else in ~110 KB (two
// blocks), at least two.  False when no tiling applies (the two-cell kernel
// runs instead).
bool rows_tiling(const Geometry &g, RowsTiling &tl) {
  if (g.nx % 8 || g.nx / 2 > ROWS_MAX_CONSUMERS) return false;
  int R = 0;
  for (int r = 1; r <= g.ny && r * g.nx / 2 <= ROWS_MAX_CONSUMERS; r++)
    if (g.ny % r == 0 && (r * g.nx) % 128 == 0) R = r;
  if (!R) return false;
  const int stage = Q * R * g.nx * 2;
  int NS = std::min(8, (74 * 1024 - 256) / stage);
  if (NS < 2) NS = std::min(8, (110 * 1024 - 256) / stage);
  if (NS < 2) return false;
  tl.R = R;
  tl.NS = NS;
  tl.tiles = g.nz * (g.ny / R);
  tl.stage_bytes = stage;
  return true;
}

template <typename S, bool STATS>
cudaError_t launch_rows16(const DomainDesc &dd, int cur, const RowsTiling &tl, cudaStream_t st) {
  const size_t smem = 256 + (size_t)tl.NS * tl.stage_bytes;
  const int threads = tl.R * dd.g.nx / 2 + 32;
  static size_t set_for = 0;  // (the attribute is per kernel instantiation)
  if (smem > set_for) {
    cudaError_t e = cudaFuncSetAttribute(collide_rows16_kernel<S, STATS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set_for = smem;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, collide_rows16_kernel<S, STATS>, threads, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(tl.tiles, std::max(1, per_sm) * sms));
  return launch_pdl(collide_rows16_kernel<S, STATS>, dim3(grid), dim3(threads), smem, st, dd, cur,
                    tl);
}

// A batch's collide grid: one block per block of cells that some domain has
// (cpb cells each), from the batch's table; grid.x = 0 when it has none.
inline void batch_grid(const BatchDims &dims, int cpb, dim3 &grid, const int2 *&blk) {
  const int l = cpb == 128 ? 0 : (cpb == 256 ? 1 : 2);
  grid = dim3((unsigned)(dims.cblk[l] ? dims.ncblk[l] : 0));
  blk = dims.cblk[l];
}

template <typename S>
cudaError_t collide_typed(const DomainDesc *D, const DomainDesc *Dhost, const BatchDims &dims,
                          int cur, int stats, int skip_active, cudaStream_t st) {
  const int bs = dims.ls.collide_block;
  if (bs != 128 && bs != 256) return cudaErrorInvalidValue;
  const bool single = dims.nd == 1 && Dhost;
  const dim3 grid((unsigned)((dims.max_cells + bs - 1) / bs)), block(bs);
  dim3 bgrid;
  const int2 *blk = nullptr;
  if (!single) {
    batch_grid(dims, bs, bgrid, blk);
    if (!blk) return cudaErrorInvalidValue;
  }
#define LBM_COLLIDE(ST, SK)                                                                 \
  (single ? launch_pdl(collide_stream_kernel<S, ST, SK>, grid, block, 0, st, *Dhost, cur)   \
          : launch_pdl(collide_stream_batch_kernel<S, ST, SK>, bgrid, block, 0, st, D, blk, cur))
  if (skip_active) return stats ? LBM_COLLIDE(true, true) : LBM_COLLIDE(false, true);
#undef LBM_COLLIDE
  if constexpr (sizeof(S) == 2) {
    // a single lattice whose rows tile, with the staged kernel chosen (the
    // autotuner picks it where it is faster): pulls staged by bulk copies
    RowsTiling tl{};
    if (dims.ls.collide_staged == 1 && dims.nd == 1 && Dhost && rows_tiling(Dhost->g, tl))
      return stats ? launch_rows16<S, true>(*Dhost, cur, tl, st)
                   : launch_rows16<S, false>(*Dhost, cur, tl, st);
    // four cells per thread (nx is a multiple of 4), blocks of 128
    if (dims.ls.collide_staged == 2) {
      const dim3 grid4((unsigned)((dims.max_cells + 511) / 512)), block4(128);
      if (!single) batch_grid(dims, 512, bgrid, blk);
#define LBM_QUADS(ST)                                                                        \
  (single ? launch_pdl(collide_quads16_kernel<S, ST>, grid4, block4, 0, st, *Dhost, cur)     \
          : launch_pdl(collide_quads16_batch_kernel<S, ST>, bgrid, block4, 0, st, D, blk, cur))
      return stats ? LBM_QUADS(true) : LBM_QUADS(false);
#undef LBM_QUADS
    }
    // two cells per thread (nx is a multiple of 4)
    const dim3 grid2((unsigned)((dims.max_cells + 2 * bs - 1) / (2 * bs)));
    if (!single) batch_grid(dims, 2 * bs, bgrid, blk);
#define LBM_PAIRS(ST)                                                                        \
  (single ? launch_pdl(collide_pairs16_kernel<S, ST>, grid2, block, 0, st, *Dhost, cur)      \
          : launch_pdl(collide_pairs16_batch_kernel<S, ST>, bgrid, block, 0, st, D, blk, cur))
    return stats ? LBM_PAIRS(true) : LBM_PAIRS(false);
#undef LBM_PAIRS
  }
#define LBM_COLLIDE(ST, SK)                                                                 \
  (single ? launch_pdl(collide_stream_kernel<S, ST, SK>, grid, block, 0, st, *Dhost, cur)   \
          : launch_pdl(collide_stream_batch_kernel<S, ST, SK>, bgrid, block, 0, st, D, blk, cur))
  return stats ? LBM_COLLIDE(true, false) : LBM_COLLIDE(false, false);
#undef LBM_COLLIDE
}

template <typename S>
cudaError_t collide_active_typed(const DomainDesc *D, const BatchDims &dims, int cur, int stats,
                                 cudaStream_t st) {
  if (dims.max_slots <= 0) return cudaSuccess;
  const unsigned nb = (unsigned)std::min((dims.max_slots + 3) / 4, 152 * 16);
  const dim3 grid(nb, dims.nd);
  return stats ? launch_pdl(collide_active_kernel<S, true>, grid, dim3(256), 0, st, D, cur)
               : launch_pdl(collide_active_kernel<S, false>, grid, dim3(256), 0, st, D, cur);
}

}  // namespace

int collide_partials(const Geometry &g) { return (int)cell_blocks(g, PARTIAL_CELLS); }

#define DISPATCH_STORAGE(storage, FN, ...)                      \
  switch (storage) {                                            \
    case 0:                                                     \
      return FN<float>(__VA_ARGS__);                            \
    case 1:                                                     \
      return FN<__nv_bfloat16>(__VA_ARGS__);                    \
    case 2:                                                     \
      return FN<__half>(__VA_ARGS__);                           \
    default:                                                    \
      return cudaErrorInvalidValue;                             \
  }

cudaError_t launch_collide_stream(int storage, const DomainDesc *D, const DomainDesc *Dhost,
                                  const BatchDims &dims, int cur, int stats, int skip_active,
                                  cudaStream_t st) {
  DISPATCH_STORAGE(storage, collide_typed, D, Dhost, dims, cur, stats, skip_active, st);
}

cudaError_t launch_collide_active(int storage, const DomainDesc *D, const BatchDims &dims,
                                  int cur, int stats, cudaStream_t st) {
  DISPATCH_STORAGE(storage, collide_active_typed, D, dims, cur, stats, st);
}

cudaError_t launch_finish_step(const DomainDesc *D, const BatchDims &dims, int stats, int split,
                               cudaStream_t st) {
  Geometry big{};
  big.ncell = dims.max_cells;
  const int nb = stats ? finish_blocks(collide_partials(big)) : 1;
  return launch_pdl(finish_step_kernel, dim3(nb, dims.nd), dim3(256), 0, st, D, stats, split);
}

namespace {
template <typename S>
cudaError_t moments_dense_typed(const Geometry &g, const void *f, float *rho, float *U,
                                cudaStream_t st) {
  moments_dense_kernel<S><<<cell_blocks(g, 256), 256, 0, st>>>((const S *)f, g, rho, U);
  return cudaGetLastError();
}
template <typename S>
cudaError_t read_pop_typed(const Geometry &g, const void *f, float *out, int dev,
                           cudaStream_t st) {
  read_pop_kernel<S><<<cell_blocks(g, 256), 256, 0, st>>>((const S *)f, g, out, dev);
  return cudaGetLastError();
}
template <typename S>
cudaError_t write_pop_typed(const Geometry &g, const float *in, void *f, cudaStream_t st) {
  write_pop_kernel<S><<<cell_blocks(g, 256), 256, 0, st>>>(in, g, (S *)f);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_moments_dense(int storage, const Geometry &g, const void *f, float *rho,
                                 float *U, cudaStream_t st) {
  DISPATCH_STORAGE(storage, moments_dense_typed, g, f, rho, U, st);
}
cudaError_t launch_read_populations(int storage, const Geometry &g, const void *f,
                                    float *out, int deviations, cudaStream_t st) {
  DISPATCH_STORAGE(storage, read_pop_typed, g, f, out, deviations, st);
}
cudaError_t launch_write_populations(int storage, const Geometry &g, const float *in,
                                     void *f, cudaStream_t st) {
  DISPATCH_STORAGE(storage, write_pop_typed, g, in, f, st);
}
cudaError_t launch_force_dense(const Geometry &g, const int *brick_slot, const float *Gs,
                               const float gbody[3], float *G, cudaStream_t st) {
  force_dense_kernel<<<cell_blocks(g, 256), 256, 0, st>>>(g, brick_slot, Gs, gbody[0],
                                                          gbody[1], gbody[2], G);
  return cudaGetLastError();
}

}  // namespace lbmibm
