// Shared definitions of the CUDA library: the D3Q19 velocity set, population
// storage formats, the 4x4x4 brick geometry, and the device-side work
// descriptors passed from the host orchestration (api.cu) to the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmibm {

// ---- D3Q19 (Sec. 2): index 0 rest, 1-6 axis, 7-18 face diagonals ---------
// Order: +x -x +y -y +z -z, (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0),
// (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1), (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1).
__host__ __device__ constexpr int ex(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                               : 0;
}
__host__ __device__ constexpr int ey(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18)  ? -1
                                                               : 0;
}
__host__ __device__ constexpr int ez(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)  ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                : 0;
}
// lattice weights t_i of Eq. 3
__host__ __device__ constexpr float wt(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wtd(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
constexpr int Q = 19;

// ---- population storage: deviations d_i = f_i - t_i ----------------------
// Stored deviations keep the velocity moments well conditioned: rho - 1 and
// rho U are sums of O(1e-3) numbers instead of O(0.1) ones.
template <typename S>
struct Store;
// ld: read-only load.  ld_pf: the same with a 64-byte L2 prefetch size, for
// scattered short rows (an L2 miss then fills the whole 64 B that HBM
// delivers per access, so x-neighbouring rows read later hit L2).  ld_stream:
// with a 256-byte L2 prefetch size, for the collide's dense rows (a warp's
// miss also brings the next warp's line: 0.990 -> 0.996 of the copy
// bandwidth at 384^3 in FP32).
__device__ __forceinline__ uint32_t ldw_stream(const uint32_t *p) {
  uint32_t v;
  asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  }
  static __device__ __forceinline__ float ld_pf(const float *p) {
    float v;
    asm volatile("ld.global.nc.L2::64B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ float ld_stream(const __nv_bfloat16 *p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __bfloat162float(__ushort_as_bfloat16(v));
  }
  static __device__ __forceinline__ float ld_pf(const __nv_bfloat16 *p) {
    unsigned short v;
    asm volatile("ld.global.nc.L2::64B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __bfloat162float(__ushort_as_bfloat16(v));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
  }
};
template <>
struct Store<__half> {
  static __device__ __forceinline__ float ld(const __half *p) {
    return __half2float(__ldg(p));
  }
  static __device__ __forceinline__ float ld_stream(const __half *p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __half2float(__ushort_as_half(v));
  }
  static __device__ __forceinline__ float ld_pf(const __half *p) {
    unsigned short v;
    asm volatile("ld.global.nc.L2::64B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __half2float(__ushort_as_half(v));
  }
  static __device__ __forceinline__ void st(__half *p, float v) {
    *p = __float2half_rn(v);
  }
};

// ---- programmatic dependent launch --------------------------------------
// The step kernels are launched with programmatic stream serialization: a
// kernel may be scheduled while its predecessor in the stream drains.  Every
// step kernel calls pdl_wait() (which returns once the predecessor grid has
// completed and its writes are visible) before it touches anything the
// predecessor wrote, and pdl_wait() precedes every exit, so completion still
// chains through the stream.  No kernel triggers its dependents early
// (griddepcontrol.launch_dependents): blocks of the next kernel would sit
// resident at pdl_wait and take registers and shared memory from the running
// one (measured slower); the implicit trigger at block exit is kept.  A no-op
// for a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launches kern<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialization allowed.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  // the stream's priority goes with the launch (kept in captured graphs)
  int prio = 0;
  if (cudaStreamGetPriority(st, &prio) != cudaSuccess) prio = 0;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- bricks: 4x4x4 cells, the unit of point binning and force storage -----
constexpr int BRICK = 4;
constexpr int BRICK_CELLS = 64;
constexpr int SLOT_FLOATS = 3 * BRICK_CELLS;  // [3][64] per active brick

// Bricks per block of the compaction scan (256 threads x 4).
constexpr int COMPACT_TILE = 1024;

// Grid of the kernels that loop over the active bricks (grid-stride): 16
// blocks per SM of the 152-SM GB300.
constexpr int PERSISTENT_BLOCKS = 152 * 16;

struct Geometry {
  int nx, ny, nz;     // cells
  int nbx, nby, nbz;  // bricks
  int64_t ncell;      // nx*ny*nz
  int nbrick;         // nbx*nby*nbz
  // n / nx and r / ny as a multiply-high and shifts (unsigned division by an
  // invariant integer, Granlund and Montgomery 1994, Sec. 4): the multipliers
  // and the shift pairs (sh1 | sh2 << 8); mx == 0 means "not set, divide"
  uint32_t mx, my;
  int shx, shy;
};

// m' = floor(2^32 (2^l - d) / d) + 1 with l = ceil(log2 d), sh1 = min(l, 1),
// sh2 = l - sh1; then n / d = (t + ((n - t) >> sh1)) >> sh2 with
// t = (m' n) >> 32, exact for every 32-bit n (d in [1, 2^31]).
inline void divisor_magic(uint32_t d, uint32_t &m, int &sh) {
  int l = 0;
  while ((1ull << l) < d) l++;
  m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  const int s1 = l > 0 ? 1 : 0;
  sh = s1 | ((l - s1) << 8);
}

__host__ __device__ __forceinline__ uint32_t div_magic(uint32_t n, uint32_t m, int sh) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(n, m);
#else
  const uint32_t t = (uint32_t)(((uint64_t)n * m) >> 32);
#endif
  return (t + ((n - t) >> (sh & 0xff))) >> (sh >> 8);
}

// Fills the division constants of g from nx and ny.
inline void geometry_divisors(Geometry &g) {
  divisor_magic((uint32_t)g.nx, g.mx, g.shx);
  divisor_magic((uint32_t)g.ny, g.my, g.shy);
}

__host__ __device__ __forceinline__ int brick_local(int x, int y, int z) {
  return ((z & 3) * 4 + (y & 3)) * 4 + (x & 3);
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  // a in (-n, 2n)
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

constexpr int BRICK_COUNTERS = 16;
constexpr int ORDER_BUCKETS = 4;

// Sparse storage over the active bricks (those inside the support of some
// point).  brick_slot[b] = slot or -1; slot_brick[s] = b.  Per slot the fields
// U0 and G are [3][64] floats (component-major, brick-local cell order z,y,x).
struct BrickMap {
  int *brick_count;  // [nbrick] points whose support overlaps the brick (set
                     //           per step, cleared by the compaction)
  int *brick_slot;   // [nbrick]
  int *slot_brick;   // [max_slots]
  int *counters;     // [BRICK_COUNTERS]: 0 = active slots, 1 = error
                     //      flags of the step (1: slot overflow, 4:
                     //      compaction scan timed out), 3 = tile ticket, 4 =
                     //      scan epoch, 5 = error flags kept until the host
                     //      reads them, 8 + q = slots in bucket q of order
  int *order;        // [ORDER_BUCKETS][max_slots] the active slots in the
                     //             order the brick kernels take them, by
                     //             pair count, longest first (the long
                     //             bricks start early, the short ones fill
                     //             the end)
  unsigned long long *tiles;  // [compact tiles] look-back words of the
                              // compaction scan
  int max_slots;
};

// Active slots of this step (0 when the compaction did not complete).
__device__ __forceinline__ int active_slots(const BrickMap &m) {
  if (m.counters[1] & 4) return 0;
  const int n = m.counters[0];
  return n < m.max_slots ? n : m.max_slots;
}

// (brick, point) pairs: one per brick that a point's support overlaps (at most
// eight per point).  Grouped by slot, ascending point index inside a slot (a
// fixed summation order).  Built once per step; the points do not move inside
// the fixed point.
struct PairMap {
  int *count;        // [max_slots] pairs of each slot
  int *start;        // [max_slots + 1]
  int *cursor;       // [max_slots]
  int *k;            // [max_pairs] point of each pair
  int *brick;        // [max_pairs] brick of each pair
  float4 *w;         // [max_pairs][3] weights of the brick's cells 0..3 along
                     //                x, y, z (0 outside the support)
  float4 *part;      // [max_pairs] brick's share of the interpolated velocity
  int *point_pairs;  // [np][8] pair of each of the point's bricks, or -1;
                     //         index = (z hi) << 2 | (y hi) << 1 | (x hi)
  int64_t max_pairs;
};

// Per-point state prepared once per step: base cell floor(x) (wrapped) in
// .xyz, the four tap weights per axis for taps floor(x)-1 .. floor(x)+2, the
// surface velocity u_k with the area s(k) in .w.
struct PointPrep {
  int4 *base;    // [np]
  float *wts;    // [np][12]  wx[4] wy[4] wz[4]
  float4 *ut;    // [np]      (u_k, s_k)
};

// Per-point MLP of the learned warm start: 16 features -> 64 -> 64 -> 3.
constexpr int MLP_IN = 16, MLP_HIDDEN = 64, MLP_OUT = 3;
constexpr int MLP_NPARAM = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN +
                           MLP_HIDDEN + MLP_OUT * MLP_HIDDEN + MLP_OUT;
// feature scales: velocities in units of MLP_VSCALE, lengths of MLP_LSCALE
constexpr float MLP_VSCALE = 0.05f, MLP_LSCALE = 16.f;

// State of the tolerance-driven fixed point, on the device.
// Blocks of the multi-block residual sums (ibm_den / ibm_check).
constexpr int RES_BLOCKS = 16;

struct IbmState {
  static constexpr int HIST = 4096;
  int done;        // 1: converged or capped
  int iters;       // iterations taken this step
  int capped;      // 1: stopped at max_iter with eps > tol
  unsigned ticket; // blocks of the residual sum done (reset by the last)
  double den2;     // ||S[s u_k]||^2 (or the fallback)
  double last_eps;
  // conjugate gradients: rho_n and alpha_n of the iterations of either
  // parity (iteration n reads those of n - 1 and stores its own)
  double cg_rho[2], cg_alpha[2];
  int cg_stop;     // the iteration at which CG stopped this step, or INT_MAX
  int cg_pad;
  double bsum[RES_BLOCKS];  // block sums of the residual sum
  double eps[HIST];  // eps of every iteration of this step
};

// Passed to the loop kernels: state == nullptr in fixed-count mode; otherwise
// the kernels return at once when state->done is set.
struct IbmLoop {
  const IbmState *state;
};

// Everything a step kernel needs about one domain (lattice, points, force
// storage).  The step kernels read D[blockIdx.y]: one launch advances every
// domain of a batch, and a single lattice is a batch of one.  Pointers are
// fixed between steps (which keeps a captured step replayable); the step
// counter t lives on the device and is advanced by the last kernel of a step.
struct DomainDesc {
  Geometry g;
  int delta;          // weighting function
  int np;             // Lagrangian points
  float tau;
  float om;           // 1 / tau (FP32, rounded to nearest)
  float gbody[3];
  void *f[2];         // the two population lattices
  int64_t *t;         // [0] device step counter, [1] the step the last
                      // prepare_points computed
  const double *X;    // [np][3] rest or fixed positions
  const int *body;    // [np]
  const float *area;  // [np]
  const float *utarget;  // [np][3]
  const double *centre, *omega, *phase;
  int nb;
  int cblocks;        // FP64 partial sums of the collide kernel, one per
                      // PARTIAL_CELLS cells
  PointPrep pp;
  BrickMap m;
  PairMap pm;
  float *U0s, *Gs, *res;
  float4 *du, *uint;
  float4 *cg;              // [5][np] point vectors of conjugate gradients
  double *cg_part;         // [ceil(np / 256)][2] block sums of its dot products
  double *xpos;
  double *partial, *sums;  // collide partials [cblocks][4], FP64 sums [4]
  double *slot_partial;    // [max_slots][4] partials of the active bricks'
                           // collide when it runs apart from the others
  double *red_scratch;     // [128][4] block sums of the final reduction
  unsigned *ticket;        // blocks of the final reduction done (reset by
                           // the last one)
  IbmState *state;
  float *feat;
  const void *mlp_packed;
  int u0_mode;             // LBM_U0_* of the U0 pre-computation
  int nbox;                // bodies with a rest-pose bounding box (box mode)
  const double *rest_box;  // [nbox][6] min x, y, z, max x, y, z of the rest
                           // positions of each body's points
  float *Ufull;            // [3][ncell] full-lattice U0 of the box strategy
};

// Launch shapes of the step kernels, picked by the autotuner (lbm_autotune).
// None changes a result: they only spread the same work over the GPU
// differently (the collide kernel's FP64 partial sums stay one per 128 cells
// whatever its block size).
struct LaunchShape {
  int collide_block = 256;       // threads per block of the collide-stream
                                 // kernel: 128 or 256
  int brick_blocks = 152 * 64;   // grid of the brick kernels (grid-stride
                                 // over the active bricks in order, a warp
                                 // each; about one brick per block, which
                                 // the hardware balances across the SMs)
  int point_block = 256;         // threads per block of the per-point
                                 // kernels: 128, 256 or 512
  int moments_spb = 4;           // bricks per block of the moments kernel
                                 // (64 threads each): 1, 2 or 4
  int sort_blocks = 152 * 32;    // grid of the sort kernel (a warp per slot,
                                 // four per block)
  int collide_staged = 2;        // 16-bit storage: four cells per thread (2),
                                 // two cells per thread (0), or (single
                                 // lattice) the pulls staged in shared memory
                                 // by bulk copies (1)
  int sort_blocks_ahead = 152 * 4;  // grid of the sort of a step prepared
                                    // ahead (it runs beside the previous
                                    // step's collide: few blocks)
};

// Cells per FP64 partial sum of the collide kernel.
constexpr int PARTIAL_CELLS = 128;

// Grid extents of a batch: the largest domain along each work dimension.
struct BatchDims {
  int nd;              // domains (gridDim.y)
  int64_t max_cells;
  int max_points;
  int max_bodies;
  int max_bricks;
  int max_slots;
  LaunchShape ls;
  // a batch's work list (device, [(ORDER_BUCKETS + 1) * nd + 2]: the
  // bucket-major and the domain-major prefix of the active slots): the
  // per-brick kernels then run one grid over the active slots of all
  // domains; NULL for a single lattice
  const int *work_off = nullptr;
  // a batch's collide block tables for 128, 256 and 512 cells per block
  // (device, (domain, block within the domain) per block of cells that some
  // domain has, domain-major) and their lengths; NULL for a single lattice
  const int2 *cblk[3] = {nullptr, nullptr, nullptr};
  int ncblk[3] = {0, 0, 0};
};

}  // namespace lbmibm
