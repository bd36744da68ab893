// Per-point MLP of the learned warm start (not in the paper): inference and
// training kernels on the BF16 tensor cores with FP32 accumulation.
//
//   y = W3 s(W2 s(W1 x + b1) + b2) + b3,   s(v) = v / (1 + e^-v)   (SiLU)
//   x: 16 features, hidden 64 and 64, y: 3 outputs.
//
// Parameters (FP32 master copy, owned by the caller): one flat vector
// P = [W1 (64x16 row-major, out x in), b1 (64), W2 (64x64), b2 (64),
// W3 (3x64), b3 (3)].  The kernels read a packed BF16 copy made by
// launch_mlp_pack: W1, W2, W2 transposed and W3 zero-padded to 8 rows, each
// row padded for conflict-free shared-memory fragment loads, plus the FP32
// biases.
//
// One warp handles 16 samples with mma.sync.m16n8k16 (A row-major 16x16 BF16,
// B column-major 16x8 BF16, C 16x8 FP32).  The C fragment of one layer is
// re-packed in registers as the A fragment of the next.  The training kernel
// recomputes the forward pass, back-propagates the mean 0.5 |y - t|^2 loss
// and forms the weight gradients of its 128 samples as tensor-core products
// over the sample dimension; per-block partial gradients are summed by a
// second kernel in a fixed order.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"

namespace lbmibm {

namespace {

constexpr int IN = MLP_IN, H = MLP_HIDDEN, OUT = MLP_OUT;
// padded row lengths (BF16 elements) of the packed matrices
constexpr int LD1 = 24;   // W1 rows (16 used)
constexpr int LD2 = 72;   // W2, W2^T, W3 rows (64 used)
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + H * LD1;
constexpr int OFF_W2T = OFF_W2 + H * LD2;
constexpr int OFF_W3 = OFF_W2T + H * LD2;
constexpr int NB16 = OFF_W3 + 8 * LD2;            // BF16 elements
constexpr int OFF_B = NB16 * 2;                   // bytes: FP32 biases follow
constexpr int NBIAS = H + H + OUT;
// The same weights for the tcgen05 kernels, in the canonical K-major layout
// of the tensor-core shared-memory descriptors without swizzle: 8 x 8 BF16
// core matrices of 128 contiguous bytes (8 rows of 16 B), the K-blocks of an
// 8-row group next to each other (byte offset tc_ofs below).  W3 is padded
// to 16 rows (the smallest N of an M = 128 MMA).  Then a status word that a
// tensor-core kernel sets when one of its waits gives up.
constexpr int OFF_TC = ((OFF_B + NBIAS * 4) + 127) / 128 * 128;  // bytes
constexpr int TC_W1 = 0, TC_W2 = TC_W1 + H * IN * 2, TC_W3 = TC_W2 + H * H * 2;
constexpr int TC_BYTES = TC_W3 + 16 * H * 2;
constexpr int OFF_STATUS = OFF_TC + TC_BYTES;
constexpr int PACKED_BYTES = OFF_STATUS + 16;

// byte offset of element (row r, column k) of a K-major operand with kb
// 8-column blocks per row group
__host__ __device__ __forceinline__ int tc_ofs(int r, int k, int kb) {
  return ((r >> 3) * kb + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// parameter offsets in P
constexpr int P_W1 = 0, P_B1 = H * IN, P_W2 = P_B1 + H, P_B2 = P_W2 + H * H, P_W3 = P_B2 + H,
              P_B3 = P_W3 + OUT * H;

__device__ __forceinline__ float silu(float v) { return v / (1.f + __expf(-v)); }
__device__ __forceinline__ float silu_grad(float v) {
  const float sg = 1.f / (1.f + __expf(-v));
  return sg * (1.f + v * (1.f - sg));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two consecutive BF16 of a padded row in shared memory, as one register
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16 *s, int row, int ld, int col) {
  return *reinterpret_cast<const uint32_t *>(s + row * ld + col);
}

struct MlpSmem {
  __nv_bfloat16 w[NB16];
  float bias[NBIAS];
};

__device__ void load_weights(MlpSmem &sm, const void *packed) {
  const uint4 *src = (const uint4 *)packed;
  uint4 *dst = (uint4 *)sm.w;
  for (int i = threadIdx.x; i < NB16 * 2 / 16; i += blockDim.x) dst[i] = src[i];
  const float *b = (const float *)((const char *)packed + OFF_B);
  for (int i = threadIdx.x; i < NBIAS; i += blockDim.x) sm.bias[i] = b[i];
}

// Forward pass of the warp's 16 samples.  xa: A fragment of the inputs.
// z1, z2: pre-activations (C fragments, 8 n-tiles x 4), h1a, h2a: the
// activations as A fragments (4 k-chunks x 4), y: C fragment of the output.
struct Fwd {
  float z1[8][4], z2[8][4], y[4];
  uint32_t h1a[4][4], h2a[4][4];
};

__device__ __forceinline__ void c_to_a(const float h[8][4], uint32_t a[4][4]) {
#pragma unroll
  for (int kc = 0; kc < 4; kc++) {
    a[kc][0] = pack_bf16(h[2 * kc][0], h[2 * kc][1]);
    a[kc][1] = pack_bf16(h[2 * kc][2], h[2 * kc][3]);
    a[kc][2] = pack_bf16(h[2 * kc + 1][0], h[2 * kc + 1][1]);
    a[kc][3] = pack_bf16(h[2 * kc + 1][2], h[2 * kc + 1][3]);
  }
}

__device__ __forceinline__ void forward16(const MlpSmem &sm, const uint32_t xa[4], Fwd &f) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16 *W1 = sm.w + OFF_W1, *W2 = sm.w + OFF_W2, *W3 = sm.w + OFF_W3;
  float h[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16(c, xa, ld2(W1, nt * 8 + g, LD1, 2 * t), ld2(W1, nt * 8 + g, LD1, 2 * t + 8));
    const float bb0 = sm.bias[nt * 8 + 2 * t], bb1 = sm.bias[nt * 8 + 2 * t + 1];
    f.z1[nt][0] = c[0] + bb0;
    f.z1[nt][1] = c[1] + bb1;
    f.z1[nt][2] = c[2] + bb0;
    f.z1[nt][3] = c[3] + bb1;
#pragma unroll
    for (int q = 0; q < 4; q++) h[nt][q] = silu(f.z1[nt][q]);
  }
  c_to_a(h, f.h1a);
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kc = 0; kc < 4; kc++)
      mma_bf16(c, f.h1a[kc], ld2(W2, nt * 8 + g, LD2, kc * 16 + 2 * t),
               ld2(W2, nt * 8 + g, LD2, kc * 16 + 2 * t + 8));
    const float bb0 = sm.bias[H + nt * 8 + 2 * t], bb1 = sm.bias[H + nt * 8 + 2 * t + 1];
    f.z2[nt][0] = c[0] + bb0;
    f.z2[nt][1] = c[1] + bb1;
    f.z2[nt][2] = c[2] + bb0;
    f.z2[nt][3] = c[3] + bb1;
#pragma unroll
    for (int q = 0; q < 4; q++) h[nt][q] = silu(f.z2[nt][q]);
  }
  c_to_a(h, f.h2a);
  float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int kc = 0; kc < 4; kc++)
    mma_bf16(c, f.h2a[kc], ld2(W3, g, LD2, kc * 16 + 2 * t), ld2(W3, g, LD2, kc * 16 + 2 * t + 8));
  // columns 2t, 2t+1 of rows g, g+8; only columns 0..2 exist
  const float bb0 = 2 * t < OUT ? sm.bias[2 * H + 2 * t] : 0.f;
  const float bb1 = 2 * t + 1 < OUT ? sm.bias[2 * H + 2 * t + 1] : 0.f;
  f.y[0] = c[0] + bb0;
  f.y[1] = c[1] + bb1;
  f.y[2] = c[2] + bb0;
  f.y[3] = c[3] + bb1;
}

// A fragment of 16 samples x 16 features from FP32 rows in global memory
// (rows >= n read as zero).
__device__ __forceinline__ void load_x(const float *__restrict__ X, int64_t row0, int64_t n,
                                       uint32_t xa[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t r0 = row0 + g, r1 = row0 + g + 8;
  float2 v00 = make_float2(0.f, 0.f), v01 = v00, v10 = v00, v11 = v00;
  if (r0 < n) {
    v00 = *(const float2 *)(X + r0 * IN + 2 * t);
    v01 = *(const float2 *)(X + r0 * IN + 2 * t + 8);
  }
  if (r1 < n) {
    v10 = *(const float2 *)(X + r1 * IN + 2 * t);
    v11 = *(const float2 *)(X + r1 * IN + 2 * t + 8);
  }
  xa[0] = pack_bf16(v00.x, v00.y);
  xa[1] = pack_bf16(v10.x, v10.y);
  xa[2] = pack_bf16(v01.x, v01.y);
  xa[3] = pack_bf16(v11.x, v11.y);
}

// ---- inference on the fifth-generation tensor cores (tcgen05) -------------
//
// One block of 128 threads (four warps) takes tiles of 128 samples.  Per tile
// and layer, the activations are written to shared memory as BF16 in the
// canonical K-major layout (tc_ofs), one thread issues the layer's
// tcgen05.mma (M = 128 samples, N = 64 or 16 outputs, K = 16 per instruction,
// BF16 inputs, FP32 accumulation in tensor memory), a tcgen05.commit signals
// completion on an mbarrier, and each warp reads its 32 rows of the
// accumulator back with tcgen05.ld (thread t holds sample t) for the
// bias, SiLU and the next layer's operand.  Tensor memory: 128 columns per
// block (layer 1 in columns 0-63, layer 2 in 64-127, layer 3 in 0-15 again
// once layer 1 has been read).  Every wait is bounded: one that gives up sets
// the status word of the packed weights, and the block stops, waits (bounded)
// for its last MMA and frees its tensor memory.
constexpr unsigned TC_SPIN_LIMIT = 1u << 24;
constexpr int TC_COLS = 128;

struct TcSmem {
  __align__(128) unsigned char w[TC_BYTES];   // W1, W2, W3 (canonical layout)
  __align__(128) unsigned char a1[128 * IN * 2];  // layer-1 operand (K = 16)
  __align__(128) unsigned char a2[128 * H * 2];   // layer-2 and layer-3 operands
  float bias[NBIAS];
  uint64_t mbar;
  uint32_t tmem;
  int stop;
};

__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle: start address, byte distance
// between K-adjacent core matrices (lbo) and between 8-row groups (sbo),
// descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t tc_desc(const void *p, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((sm_addr(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          sm_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned phase) {
  for (unsigned i = 0; i < TC_SPIN_LIMIT; i++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(sm_addr(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy writes of shared memory made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// bias + SiLU of 64 accumulator columns (starting at column col) of this
// thread's row, as the next layer's BF16 operand row t
__device__ __forceinline__ void tc_hidden(uint32_t trow, int col, const float *bias,
                                          unsigned char *a2, int t) {
#pragma unroll
  for (int c = 0; c < H / 16; c++) {
    float z[16];
    tc_ld16(trow + col + 16 * c, z);
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
      w[i] = pack_bf16(silu(z[2 * i] + bias[16 * c + 2 * i]),
                       silu(z[2 * i + 1] + bias[16 * c + 2 * i + 1]));
    *(uint4 *)(a2 + tc_ofs(t, 16 * c, H / 8)) = make_uint4(w[0], w[1], w[2], w[3]);
    *(uint4 *)(a2 + tc_ofs(t, 16 * c + 8, H / 8)) = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// Inference.  mode 0: Y[n][3] = y.  mode 1 (warm start of the fixed point):
// du[k] = du_prev[k] + scale * y, with du_prev read from du itself (zero when
// !use_prev).
__device__ void mlp_tc_rows(int64_t n, const float *__restrict__ X, const void *packed,
                            float *__restrict__ Y, float4 *__restrict__ du, float scale, int mode,
                            int use_prev, TcSmem &sm) {
  const int t = threadIdx.x, warp = t >> 5;
  {
    const uint4 *src = (const uint4 *)((const char *)packed + OFF_TC);
    uint4 *dst = (uint4 *)sm.w;
    for (int i = t; i < TC_BYTES / 16; i += blockDim.x) dst[i] = src[i];
    const float *b = (const float *)((const char *)packed + OFF_B);
    for (int i = t; i < NBIAS; i += blockDim.x) sm.bias[i] = b[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sm_addr(&sm.tmem)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.stop = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes
  const uint64_t w1 = tc_desc(sm.w + TC_W1, 128, 256);
  unsigned phase = 0;
  bool pending = false;  // an MMA group whose completion was not observed
  for (int64_t row0 = (int64_t)blockIdx.x * 128; row0 < n; row0 += (int64_t)gridDim.x * 128) {
    const int64_t row = row0 + t;
    {
      // x (16 features) -> BF16 operand row t
      float4 v[4] = {};
      if (row < n) {
        const float4 *xr = (const float4 *)(X + row * IN);
#pragma unroll
        for (int i = 0; i < 4; i++) v[i] = xr[i];
      }
      *(uint4 *)(sm.a1 + tc_ofs(t, 0, IN / 8)) =
          make_uint4(pack_bf16(v[0].x, v[0].y), pack_bf16(v[0].z, v[0].w),
                     pack_bf16(v[1].x, v[1].y), pack_bf16(v[1].z, v[1].w));
      *(uint4 *)(sm.a1 + tc_ofs(t, 8, IN / 8)) =
          make_uint4(pack_bf16(v[2].x, v[2].y), pack_bf16(v[2].z, v[2].w),
                     pack_bf16(v[3].x, v[3].y), pack_bf16(v[3].z, v[3].w));
    }
    float y[4];
    bool ok = true;
#pragma unroll 1
    for (int layer = 0; layer < 3 && ok; layer++) {
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        if (layer == 0) {
          tc_mma(tmem, tc_desc(sm.a1, 128, 256), w1, tc_idesc(128, H), 0);
        } else {
          // K = 64 in four steps of 16 (two core matrices, 256 B, each)
          const unsigned char *wb = sm.w + (layer == 1 ? TC_W2 : TC_W3);
          const uint32_t d = tmem + (layer == 1 ? 64 : 0);
          const uint32_t idesc = tc_idesc(128, layer == 1 ? H : 16);
#pragma unroll
          for (int k = 0; k < 4; k++)
            tc_mma(d, tc_desc(sm.a2 + 256 * k, 128, 1024), tc_desc(wb + 256 * k, 128, 1024),
                   idesc, k > 0);
        }
        tc_commit(&sm.mbar);
      }
      pending = true;
      ok = __syncthreads_and(tc_wait(&sm.mbar, phase)) != 0;
      phase ^= 1u;
      if (!ok) break;
      pending = false;
      tc_fence_after();
      if (layer == 0) {
        tc_hidden(trow, 0, sm.bias, sm.a2, t);
      } else if (layer == 1) {
        tc_hidden(trow, 64, sm.bias + H, sm.a2, t);
      } else {
        float z[16];
        tc_ld16(trow, z);
#pragma unroll
        for (int i = 0; i < OUT; i++) y[i] = z[i] + sm.bias[2 * H + i];
      }
    }
    if (!ok) {
      if (t == 0) atomicOr((unsigned *)((char *)packed + OFF_STATUS), 1u);
      break;
    }
    if (row < n) {
      if (mode == 0) {
        Y[3 * row] = y[0];
        Y[3 * row + 1] = y[1];
        Y[3 * row + 2] = y[2];
      } else {
        float4 d = use_prev ? du[row] : make_float4(0.f, 0.f, 0.f, 0.f);
        d.x += scale * y[0];
        d.y += scale * y[1];
        d.z += scale * y[2];
        du[row] = d;
      }
    }
  }
  // the last MMA group must be done before the tensor memory is freed
  if (pending) (void)tc_wait(&sm.mbar, phase ^ 1u);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_COLS)
                 : "memory");
  }
}

__global__ void __launch_bounds__(128)
    mlp_forward_kernel(int64_t n, const float *__restrict__ X, const void *packed,
                       float *__restrict__ Y) {
  __shared__ TcSmem sm;
  mlp_tc_rows(n, X, packed, Y, nullptr, 0.f, 0, 0, sm);
}

__global__ void __launch_bounds__(128)
    mlp_warm_kernel(const DomainDesc *__restrict__ D, int use_prev) {
  pdl_wait();
  __shared__ TcSmem sm;
  const DomainDesc &d = D[blockIdx.y];
  if (d.np == 0 || !d.mlp_packed) return;
  mlp_tc_rows(d.np, d.feat, d.mlp_packed, nullptr, d.du, MLP_VSCALE, 1, use_prev, sm);
}

// Shared memory of the training kernel: weights plus the block's 128 samples
// of x, dz1, h1, dz2, h2 (BF16) and dy (FP32) for the weight gradients.
struct TrainSmem {
  MlpSmem m;
  float w3[OUT * H];                // W3 in FP32 for the first backward step
  __nv_bfloat16 x[128][IN + 8];
  __nv_bfloat16 h1[128][H + 8], dz1[128][H + 8];
  __nv_bfloat16 h2[128][H + 8], dz2[128][H + 8];
  float dy[128][4];
  float red[8][NBIAS];
  float loss[8];
};

// One block = 8 warps = 128 samples.  Writes its partial gradient (FP32,
// layout of P) and partial loss.
__global__ void __launch_bounds__(256)
    mlp_train_kernel(int64_t n, const float *__restrict__ X, const float *__restrict__ T,
                     const void *packed, const float *__restrict__ P, float *__restrict__ part,
                     float *__restrict__ part_loss, float inv_n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smraw);
  load_weights(sm.m, packed);
  for (int i = threadIdx.x; i < OUT * H; i += blockDim.x) sm.w3[i] = P[P_W3 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * 128 + w * 16;
  uint32_t xa[4];
  load_x(X, row0, n, xa);
  Fwd f;
  forward16(sm.m, xa, f);
  const int lr0 = w * 16 + g, lr1 = lr0 + 8;  // local rows
  const int64_t gr0 = row0 + g, gr1 = row0 + g + 8;
  // dy = (y - t) / n for valid rows and columns; loss
  float dy[4], loss = 0.f;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int col = 2 * t + (q & 1);
    const int64_t row = q < 2 ? gr0 : gr1;
    float e = 0.f;
    if (col < OUT && row < n) e = f.y[q] - T[3 * row + col];
    loss += 0.5f * e * e;
    dy[q] = e * inv_n;
  }
  if (t < 2) {
    sm.dy[lr0][2 * t] = dy[0];
    sm.dy[lr0][2 * t + 1] = dy[1];
    sm.dy[lr1][2 * t] = dy[2];
    sm.dy[lr1][2 * t + 1] = dy[3];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) sm.loss[w] = loss;
  // stage x, h1, h2 for the weight gradients
  {
    const float2 *xr0 = (const float2 *)(X + (gr0 < n ? gr0 : 0) * IN);
    const float2 *xr1 = (const float2 *)(X + (gr1 < n ? gr1 : 0) * IN);
    // x rows in BF16 (zero for rows >= n)
    const float2 a = gr0 < n ? xr0[t] : make_float2(0.f, 0.f),
                 b = gr0 < n ? xr0[t + 4] : make_float2(0.f, 0.f),
                 c = gr1 < n ? xr1[t] : make_float2(0.f, 0.f),
                 d = gr1 < n ? xr1[t + 4] : make_float2(0.f, 0.f);
    *(uint32_t *)&sm.x[lr0][2 * t] = pack_bf16(a.x, a.y);
    *(uint32_t *)&sm.x[lr0][2 * t + 8] = pack_bf16(b.x, b.y);
    *(uint32_t *)&sm.x[lr1][2 * t] = pack_bf16(c.x, c.y);
    *(uint32_t *)&sm.x[lr1][2 * t + 8] = pack_bf16(d.x, d.y);
  }
#pragma unroll
  for (int kc = 0; kc < 4; kc++) {
    *(uint32_t *)&sm.h1[lr0][kc * 16 + 2 * t] = f.h1a[kc][0];
    *(uint32_t *)&sm.h1[lr1][kc * 16 + 2 * t] = f.h1a[kc][1];
    *(uint32_t *)&sm.h1[lr0][kc * 16 + 2 * t + 8] = f.h1a[kc][2];
    *(uint32_t *)&sm.h1[lr1][kc * 16 + 2 * t + 8] = f.h1a[kc][3];
    *(uint32_t *)&sm.h2[lr0][kc * 16 + 2 * t] = f.h2a[kc][0];
    *(uint32_t *)&sm.h2[lr1][kc * 16 + 2 * t] = f.h2a[kc][1];
    *(uint32_t *)&sm.h2[lr0][kc * 16 + 2 * t + 8] = f.h2a[kc][2];
    *(uint32_t *)&sm.h2[lr1][kc * 16 + 2 * t + 8] = f.h2a[kc][3];
  }
  __syncwarp();
  // dh2 = dy W3 (K = 3, FP32), dz2 = dh2 s'(z2)
  const float dyr0[3] = {sm.dy[lr0][0], sm.dy[lr0][1], sm.dy[lr0][2]};
  const float dyr1[3] = {sm.dy[lr1][0], sm.dy[lr1][1], sm.dy[lr1][2]};
  float dz[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int col = nt * 8 + 2 * t + (q & 1);
      const float *dr = q < 2 ? dyr0 : dyr1;
      const float dh = dr[0] * sm.w3[col] + dr[1] * sm.w3[H + col] + dr[2] * sm.w3[2 * H + col];
      dz[nt][q] = dh * silu_grad(f.z2[nt][q]);
    }
  }
  uint32_t dz2a[4][4];
  c_to_a(dz, dz2a);
#pragma unroll
  for (int kc = 0; kc < 4; kc++) {
    *(uint32_t *)&sm.dz2[lr0][kc * 16 + 2 * t] = dz2a[kc][0];
    *(uint32_t *)&sm.dz2[lr1][kc * 16 + 2 * t] = dz2a[kc][1];
    *(uint32_t *)&sm.dz2[lr0][kc * 16 + 2 * t + 8] = dz2a[kc][2];
    *(uint32_t *)&sm.dz2[lr1][kc * 16 + 2 * t + 8] = dz2a[kc][3];
  }
  // dh1 = dz2 W2 (B[k=o][n=i] = W2[o][i] = W2T[i][o]), dz1 = dh1 s'(z1)
  const __nv_bfloat16 *W2T = sm.m.w + OFF_W2T;
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kc = 0; kc < 4; kc++)
      mma_bf16(c, dz2a[kc], ld2(W2T, nt * 8 + g, LD2, kc * 16 + 2 * t),
               ld2(W2T, nt * 8 + g, LD2, kc * 16 + 2 * t + 8));
#pragma unroll
    for (int q = 0; q < 4; q++) dz[nt][q] = c[q] * silu_grad(f.z1[nt][q]);
  }
  uint32_t dz1a[4][4];
  c_to_a(dz, dz1a);
#pragma unroll
  for (int kc = 0; kc < 4; kc++) {
    *(uint32_t *)&sm.dz1[lr0][kc * 16 + 2 * t] = dz1a[kc][0];
    *(uint32_t *)&sm.dz1[lr1][kc * 16 + 2 * t] = dz1a[kc][1];
    *(uint32_t *)&sm.dz1[lr0][kc * 16 + 2 * t + 8] = dz1a[kc][2];
    *(uint32_t *)&sm.dz1[lr1][kc * 16 + 2 * t + 8] = dz1a[kc][3];
  }
  __syncthreads();
  float *pb = part + (size_t)blockIdx.x * MLP_NPARAM;
  // Weight gradients over the block's 128 samples (K = sample):
  //   dW2[o][i] = sum_r dz2[r][o] h1[r][i], dW1[o][i] = sum_r dz1[r][o] x[r][i]
  // A[m = o][k = r] = dz[r][o], B[k = r][n = i] = h[r][i], both gathered from
  // the sample-major tiles.  Warp w owns output rows 16 (w >> 1) .. +15 and
  // half of the columns.
  {
    const int m0 = (w >> 1) * 16;
    auto afrag = [&](const __nv_bfloat16 (*dzt)[H + 8], int k0, uint32_t a[4]) {
      auto e = [&](int k, int m) { return dzt[k0 + k][m0 + m]; };
      a[0] = pack_bf16(__bfloat162float(e(2 * t, g)), __bfloat162float(e(2 * t + 1, g)));
      a[1] = pack_bf16(__bfloat162float(e(2 * t, g + 8)), __bfloat162float(e(2 * t + 1, g + 8)));
      a[2] = pack_bf16(__bfloat162float(e(2 * t + 8, g)), __bfloat162float(e(2 * t + 9, g)));
      a[3] = pack_bf16(__bfloat162float(e(2 * t + 8, g + 8)), __bfloat162float(e(2 * t + 9, g + 8)));
    };
    // dW2: 4 n-tiles per warp
    {
      float c[4][4] = {};
      const int n0 = (w & 1) * 32;
      for (int k0 = 0; k0 < 128; k0 += 16) {
        uint32_t a[4];
        afrag(sm.dz2, k0, a);
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int nn = n0 + j * 8 + g;
          const uint32_t b0 = pack_bf16(__bfloat162float(sm.h1[k0 + 2 * t][nn]),
                                        __bfloat162float(sm.h1[k0 + 2 * t + 1][nn]));
          const uint32_t b1 = pack_bf16(__bfloat162float(sm.h1[k0 + 2 * t + 8][nn]),
                                        __bfloat162float(sm.h1[k0 + 2 * t + 9][nn]));
          mma_bf16(c[j], a, b0, b1);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int col = n0 + j * 8 + 2 * t;
        pb[P_W2 + (m0 + g) * H + col] = c[j][0];
        pb[P_W2 + (m0 + g) * H + col + 1] = c[j][1];
        pb[P_W2 + (m0 + g + 8) * H + col] = c[j][2];
        pb[P_W2 + (m0 + g + 8) * H + col + 1] = c[j][3];
      }
    }
    // dW1: one n-tile per warp (N = 16)
    {
      float c[4] = {};
      const int n0 = (w & 1) * 8;
      for (int k0 = 0; k0 < 128; k0 += 16) {
        uint32_t a[4];
        afrag(sm.dz1, k0, a);
        const int nn = n0 + g;
        const uint32_t b0 = pack_bf16(__bfloat162float(sm.x[k0 + 2 * t][nn]),
                                      __bfloat162float(sm.x[k0 + 2 * t + 1][nn]));
        const uint32_t b1 = pack_bf16(__bfloat162float(sm.x[k0 + 2 * t + 8][nn]),
                                      __bfloat162float(sm.x[k0 + 2 * t + 9][nn]));
        mma_bf16(c, a, b0, b1);
      }
      const int col = n0 + 2 * t;
      pb[P_W1 + (m0 + g) * IN + col] = c[0];
      pb[P_W1 + (m0 + g) * IN + col + 1] = c[1];
      pb[P_W1 + (m0 + g + 8) * IN + col] = c[2];
      pb[P_W1 + (m0 + g + 8) * IN + col + 1] = c[3];
    }
  }
  // dW3[c][o] = sum_r dy[r][c] h2[r][o] (N = 3: FP32 dot products), biases
  for (int e = threadIdx.x; e < OUT * H; e += blockDim.x) {
    const int cc = e / H, o = e % H;
    float s = 0.f;
    for (int r = 0; r < 128; r++) s += sm.dy[r][cc] * __bfloat162float(sm.h2[r][o]);
    pb[P_W3 + e] = s;
  }
  for (int e = threadIdx.x; e < NBIAS; e += blockDim.x) {
    float s = 0.f;
    if (e < H) {
      for (int r = 0; r < 128; r++) s += __bfloat162float(sm.dz1[r][e]);
      pb[P_B1 + e] = s;
    } else if (e < 2 * H) {
      for (int r = 0; r < 128; r++) s += __bfloat162float(sm.dz2[r][e - H]);
      pb[P_B2 + e - H] = s;
    } else {
      for (int r = 0; r < 128; r++) s += sm.dy[r][e - 2 * H];
      pb[P_B3 + e - 2 * H] = s;
    }
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int q = 0; q < 8; q++) l += sm.loss[q];
    part_loss[blockIdx.x] = l * inv_n;
  }
}

// grad[j] = sum over blocks b of part[b][j], in block order; loss likewise.
__global__ void mlp_reduce_kernel(int nblocks, const float *__restrict__ part,
                                  const float *__restrict__ part_loss, float *__restrict__ grad,
                                  float *__restrict__ loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < MLP_NPARAM) {
    float s = 0.f;
    for (int b = 0; b < nblocks; b++) s += part[(size_t)b * MLP_NPARAM + j];
    grad[j] = s;
  }
  if (j == MLP_NPARAM && loss) {
    float s = 0.f;
    for (int b = 0; b < nblocks; b++) s += part_loss[b];
    *loss = s;
  }
}

// FP32 parameters -> packed BF16 matrices (padded rows, W2 also transposed,
// W3 zero-padded to 8 rows) + FP32 biases.
__global__ void mlp_pack_kernel(const float *__restrict__ P, void *packed) {
  __nv_bfloat16 *w = (__nv_bfloat16 *)packed;
  float *bias = (float *)((char *)packed + OFF_B);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NB16 + NBIAS;
       e += gridDim.x * blockDim.x) {
    if (e < OFF_W2) {
      const int r = e / LD1, c = e % LD1;
      w[e] = __float2bfloat16_rn(c < IN ? P[P_W1 + r * IN + c] : 0.f);
    } else if (e < OFF_W2T) {
      const int r = (e - OFF_W2) / LD2, c = (e - OFF_W2) % LD2;
      w[e] = __float2bfloat16_rn(c < H ? P[P_W2 + r * H + c] : 0.f);
    } else if (e < OFF_W3) {
      const int r = (e - OFF_W2T) / LD2, c = (e - OFF_W2T) % LD2;
      w[e] = __float2bfloat16_rn(c < H ? P[P_W2 + c * H + r] : 0.f);
    } else if (e < NB16) {
      const int r = (e - OFF_W3) / LD2, c = (e - OFF_W3) % LD2;
      w[e] = __float2bfloat16_rn(r < OUT && c < H ? P[P_W3 + r * H + c] : 0.f);
    } else {
      const int j = e - NB16;
      bias[j] = j < H ? P[P_B1 + j] : (j < 2 * H ? P[P_B2 + j - H] : P[P_B3 + j - 2 * H]);
    }
  }
  // the tensor-core copies (rows = outputs, K = inputs) and the status word
  unsigned char *tc = (unsigned char *)packed + OFF_TC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * IN + H * H + 16 * H;
       e += gridDim.x * blockDim.x) {
    float v;
    int ofs;
    if (e < H * IN) {
      const int r = e / IN, k = e % IN;
      v = P[P_W1 + r * IN + k];
      ofs = TC_W1 + tc_ofs(r, k, IN / 8);
    } else if (e < H * IN + H * H) {
      const int q = e - H * IN, r = q / H, k = q % H;
      v = P[P_W2 + r * H + k];
      ofs = TC_W2 + tc_ofs(r, k, H / 8);
    } else {
      const int q = e - H * IN - H * H, r = q / H, k = q % H;
      v = r < OUT ? P[P_W3 + r * H + k] : 0.f;
      ofs = TC_W3 + tc_ofs(r, k, H / 8);
    }
    *(__nv_bfloat16 *)(tc + ofs) = __float2bfloat16_rn(v);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *(unsigned *)((char *)packed + OFF_STATUS) = 0u;
}

// Adam (Kingma & Ba) on the FP32 master parameters, bias-corrected.
__global__ void mlp_adam_kernel(float *__restrict__ P, float *__restrict__ m,
                                float *__restrict__ v, const float *__restrict__ grad,
                                float lr, float b1, float b2, float eps, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= MLP_NPARAM) return;
  const float gj = grad[j];
  const float mj = b1 * m[j] + (1.f - b1) * gj;
  const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  P[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

}  // namespace

size_t mlp_packed_bytes() { return (size_t)PACKED_BYTES; }

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_pack(const float *P, void *packed, cudaStream_t st) {
  mlp_pack_kernel<<<16, 256, 0, st>>>(P, packed);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(int64_t n, const float *X, const void *packed, float *Y,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 127) / 128, 152 * 4);
  mlp_forward_kernel<<<(unsigned)blocks, 128, 0, st>>>(n, X, packed, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_warm(const DomainDesc *D, const BatchDims &dims, int use_prev,
                            cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int64_t want = (dims.max_points + 127) / 128;
  const int64_t cap = std::max<int64_t>(1, 152 * 4 / std::max(1, dims.nd));
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min(want, cap));
  return launch_pdl(mlp_warm_kernel, dim3(bx, dims.nd), dim3(128), 0, st, D, use_prev);
}

cudaError_t launch_mlp_loss_grad(int64_t n, const float *X, const float *T, const void *packed,
                                 const float *P, float *grad, float *loss, float *part,
                                 cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  const int nb = (int)((n + 127) / 128);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TrainSmem));
  if (e != cudaSuccess) return e;
  float *part_loss = part + (size_t)nb * MLP_NPARAM;
  mlp_train_kernel<<<nb, 256, sizeof(TrainSmem), st>>>(n, X, T, packed, P, part, part_loss,
                                                       1.f / (float)n);
  mlp_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(nb, part, part_loss, grad,
                                                                  loss);
  return cudaGetLastError();
}

size_t mlp_grad_scratch_floats(int64_t n) {
  const int64_t nb = (n + 127) / 128;
  return (size_t)nb * (MLP_NPARAM + 1);
}

cudaError_t launch_mlp_adam(float *P, float *m, float *v, const float *grad, int64_t step,
                            float lr, float b1, float b2, float eps, void *packed,
                            cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(P, m, v, grad, lr, b1, b2, eps, c1,
                                                            c2);
  if (packed) mlp_pack_kernel<<<16, 256, 0, st>>>(P, packed);
  return cudaGetLastError();
}

}  // namespace lbmibm
