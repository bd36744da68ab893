// Per-point MLP of the learned warm start (not in the paper): inference and
// training kernels on the fifth-generation (tcgen05) tensor cores, BF16
// operands, FP32 accumulation in tensor memory.
//
//   y = W3 s(W2 s(W1 x + b1) + b2) + b3,   s(v) = v / (1 + e^-v)   (SiLU)
//   x: 16 features, hidden 64 and 64, y: 3 outputs.
//
// Parameters (FP32 master copy, owned by the caller): one flat vector
// P = [W1 (64x16 row-major, out x in), b1 (64), W2 (64x64), b2 (64),
// W3 (3x64), b3 (3)].  The kernels read a packed copy made by
// launch_mlp_pack: the FP32 biases, then the BF16 weights in the canonical
// K-major layout of the tensor cores' shared-memory operands (W1, W2, W3
// padded to 16 rows, and W2 transposed for the backward pass), then a status
// word.
//
// A block takes 128 samples (one per thread, four warps): each layer is one
// to eight tcgen05.mma with M = 128 samples (K = 16 per instruction) whose
// accumulators live in tensor memory; the epilogues (bias, SiLU, the
// derivative) read them back with tcgen05.ld and write the next operand to
// shared memory.  The training kernel recomputes the forward pass,
// back-propagates the mean 0.5 |y - t|^2 loss and forms the weight gradients
// of its 128 samples as tensor-core products over the sample dimension (the
// operands transposed in shared memory, a row of ones giving the bias
// gradients); per-block partial gradients are summed by a second kernel in a
// fixed order.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"

namespace lbmibm {

namespace {

constexpr int IN = MLP_IN, H = MLP_HIDDEN, OUT = MLP_OUT;
constexpr int NBIAS = H + H + OUT;
// parameter offsets in P
constexpr int P_W1 = 0, P_B1 = H * IN, P_W2 = P_B1 + H, P_B2 = P_W2 + H * H, P_W3 = P_B2 + H,
              P_B3 = P_W3 + OUT * H;
// packed copy (bytes): FP32 biases [b1, b2, b3]; the BF16 weights in the
// canonical K-major layout of the tensor-core shared-memory descriptors
// without swizzle (8 x 8 core matrices of 128 contiguous bytes, 8 rows of
// 16 B; the K-blocks of an 8-row group next to each other: tc_ofs); a status
// word that a tensor-core kernel sets when one of its waits gives up
constexpr int OFF_B = 0;
constexpr int OFF_TC = (NBIAS * 4 + 127) / 128 * 128;
constexpr int TC_W1 = 0, TC_W2 = TC_W1 + H * IN * 2, TC_W3 = TC_W2 + H * H * 2;
constexpr int TC_FWD_BYTES = TC_W3 + 16 * H * 2;  // W1, W2, W3 (16 rows)
constexpr int TC_W2T = TC_FWD_BYTES;              // W2^T (rows = inputs)
constexpr int TC_BYTES = TC_W2T + H * H * 2;
constexpr int OFF_STATUS = OFF_TC + TC_BYTES;
constexpr int PACKED_BYTES = OFF_STATUS + 16;

// byte offset of element (row r, column k) of a K-major operand with kb
// 8-column blocks per row group
__host__ __device__ __forceinline__ int tc_ofs(int r, int k, int kb) {
  return ((r >> 3) * kb + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ float silu(float v) { return v / (1.f + __expf(-v)); }
__device__ __forceinline__ float silu_grad(float v) {
  const float sg = 1.f / (1.f + __expf(-v));
  return sg * (1.f + v * (1.f - sg));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
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
// bias, SiLU and the next layer's operand.  Tensor memory: 64 columns per
// block, each layer's accumulator in columns 0-63 (0-15 for layer 3) once
// the previous one has been read (its epilogue precedes the next issue).  Every wait is bounded: one that gives up sets
// the status word of the packed weights, and the block stops, waits (bounded)
// for its last MMA and frees its tensor memory.
constexpr unsigned TC_SPIN_LIMIT = 1u << 24;
constexpr int TC_COLS = 64;

struct TcSmem {
  __align__(128) unsigned char w[TC_FWD_BYTES];  // W1, W2, W3 (canonical layout)
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
    for (int i = t; i < TC_FWD_BYTES / 16; i += blockDim.x) dst[i] = src[i];
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
          const uint32_t d = tmem;
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
        tc_hidden(trow, 0, sm.bias + H, sm.a2, t);
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

// ---- training: forward, backward and weight gradients of 128 samples -----
//
// Tensor memory (256 columns): z1 = W1 x in 0-63, z2 = W2 h1 in 64-127 and y
// in 128-143 for the forward pass; then dh1 = dz2 W2 in 144-207, the weight
// gradient of layer 2 (with the bias gradient in its column 64) over 64-143
// once z2 and y have been read, and that of layer 1 (bias in column 16) in
// 208-239.  Shared-memory operands (BF16, canonical layout): x, h1, h2 and
// dz2 sample-major for the forward and backward products; x^T, h1^T (each
// with a row of ones) and dz^T (dz2^T, then dz1^T, 64 rows padded to 128
// with zeros) for the products over the samples.
constexpr int TR_COLS = 256;
constexpr int KB_S = 128 / 8;  // K-blocks of an operand whose K is the 128 samples

struct TrainSmem {
  __align__(128) unsigned char w[TC_BYTES];            // W1, W2, W3, W2^T
  __align__(128) unsigned char x[128 * IN * 2];        // [s][16]
  __align__(128) unsigned char xT[32 * 128 * 2];       // [16 + ones + pad][s]
  __align__(128) unsigned char h1[128 * H * 2];        // [s][64]
  __align__(128) unsigned char h1T[80 * 128 * 2];      // [64 + ones + pad][s]
  __align__(128) unsigned char h2[128 * H * 2];        // [s][64]
  __align__(128) unsigned char dz2[128 * H * 2];       // [s][64]
  __align__(128) unsigned char dzT[128 * 128 * 2];     // [64 + zero pad][s]
  float w3[OUT * H];                                   // W3 in FP32
  float bias[NBIAS];
  float dy[128][4];
  float loss[4];
  uint64_t mbar;
  uint32_t tmem;
};

// this thread's row of a sample-major operand with 64 columns, from 64
// FP32 values
__device__ __forceinline__ void put_row64(unsigned char *op, int s, const float v[H]) {
#pragma unroll
  for (int c = 0; c < H / 8; c++)
    *(uint4 *)(op + tc_ofs(s, 8 * c, H / 8)) =
        make_uint4(pack_bf16(v[8 * c], v[8 * c + 1]), pack_bf16(v[8 * c + 2], v[8 * c + 3]),
                   pack_bf16(v[8 * c + 4], v[8 * c + 5]), pack_bf16(v[8 * c + 6], v[8 * c + 7]));
}

// column s of a transposed operand (rows 0 .. m-1, K = the 128 samples)
template <int M>
__device__ __forceinline__ void put_col(unsigned char *op, int s, const float v[M]) {
#pragma unroll
  for (int r = 0; r < M; r++)
    *(__nv_bfloat16 *)(op + tc_ofs(r, s, KB_S)) = __float2bfloat16_rn(v[r]);
}

// 64 accumulator columns (from col) of this thread's row
__device__ __forceinline__ void tc_ld64(uint32_t trow, int col, float v[H]) {
#pragma unroll
  for (int c = 0; c < H / 16; c++) tc_ld16(trow + col + 16 * c, v + 16 * c);
}

// one tensor-core round of the block: thread 0 issues `issue` after every
// thread's shared-memory writes, and every thread waits for the products
template <typename Issue>
__device__ __forceinline__ bool tc_round(TrainSmem &sm, unsigned &phase, Issue issue) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue();
    tc_commit(&sm.mbar);
  }
  const bool ok = __syncthreads_and(tc_wait(&sm.mbar, phase)) != 0;
  phase ^= 1u;
  if (ok) tc_fence_after();
  return ok;
}

// One block = 128 samples (one per thread).  Writes its partial gradient
// (FP32, layout of P) and partial loss.
__global__ void __launch_bounds__(128)
    mlp_train_kernel(int64_t n, const float *__restrict__ X, const float *__restrict__ T,
                     const void *packed, const float *__restrict__ P, float *__restrict__ part,
                     float *__restrict__ part_loss, float inv_n) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smraw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  {
    const uint4 *src = (const uint4 *)((const char *)packed + OFF_TC);
    for (int i = t; i < TC_BYTES / 16; i += blockDim.x) ((uint4 *)sm.w)[i] = src[i];
    const float *b = (const float *)((const char *)packed + OFF_B);
    for (int i = t; i < NBIAS; i += blockDim.x) sm.bias[i] = b[i];
    for (int i = t; i < OUT * H; i += blockDim.x) sm.w3[i] = P[P_W3 + i];
    // the rows of ones (bias gradients) and the zero padding of the
    // transposed operands
    for (int i = t; i < 32 * 128 * 2 / 16; i += blockDim.x) ((uint4 *)sm.xT)[i] = make_uint4(0, 0, 0, 0);
    for (int i = t; i < 80 * 128 * 2 / 16; i += blockDim.x) ((uint4 *)sm.h1T)[i] = make_uint4(0, 0, 0, 0);
    for (int i = t; i < 128 * 128 * 2 / 16; i += blockDim.x) ((uint4 *)sm.dzT)[i] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sm_addr(&sm.tmem)),
                 "r"(TR_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  *(__nv_bfloat16 *)(sm.xT + tc_ofs(IN, t, KB_S)) = __float2bfloat16_rn(1.f);
  *(__nv_bfloat16 *)(sm.h1T + tc_ofs(H, t, KB_S)) = __float2bfloat16_rn(1.f);
  const uint32_t tmem = sm.tmem;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  const int64_t row = (int64_t)blockIdx.x * 128 + t;
  const bool valid = row < n;
  const unsigned char *W1 = sm.w + TC_W1, *W2 = sm.w + TC_W2, *W3 = sm.w + TC_W3,
                      *W2T = sm.w + TC_W2T;
  unsigned phase = 0;
  bool ok = true;
  {
    float x[IN] = {};
    if (valid)
#pragma unroll
      for (int i = 0; i < IN; i++) x[i] = X[row * IN + i];
    *(uint4 *)(sm.x + tc_ofs(t, 0, IN / 8)) =
        make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]),
                   pack_bf16(x[6], x[7]));
    *(uint4 *)(sm.x + tc_ofs(t, 8, IN / 8)) =
        make_uint4(pack_bf16(x[8], x[9]), pack_bf16(x[10], x[11]), pack_bf16(x[12], x[13]),
                   pack_bf16(x[14], x[15]));
    put_col<IN>(sm.xT, t, x);
  }
  // forward, layer 1: z1 = W1 x (columns 0-63)
  ok = tc_round(sm, phase, [&] {
    tc_mma(tmem, tc_desc(sm.x, 128, 256), tc_desc(W1, 128, 256), tc_idesc(128, H), 0);
  });
  if (ok) {
    float z[H];
    tc_ld64(trow, 0, z);
#pragma unroll
    for (int i = 0; i < H; i++) z[i] = silu(z[i] + sm.bias[i]);
    put_row64(sm.h1, t, z);
    put_col<H>(sm.h1T, t, z);
    // layer 2: z2 = W2 h1 (columns 64-127)
    ok = tc_round(sm, phase, [&] {
#pragma unroll
      for (int k = 0; k < 4; k++)
        tc_mma(tmem + 64, tc_desc(sm.h1 + 256 * k, 128, 1024),
               tc_desc(W2 + 256 * k, 128, 1024), tc_idesc(128, H), k > 0);
    });
  }
  if (ok) {
    float z[H];
    tc_ld64(trow, 64, z);
#pragma unroll
    for (int i = 0; i < H; i++) z[i] = silu(z[i] + sm.bias[H + i]);
    put_row64(sm.h2, t, z);
    // layer 3: y (columns 128-143)
    ok = tc_round(sm, phase, [&] {
#pragma unroll
      for (int k = 0; k < 4; k++)
        tc_mma(tmem + 128, tc_desc(sm.h2 + 256 * k, 128, 1024),
               tc_desc(W3 + 256 * k, 128, 1024), tc_idesc(128, 16), k > 0);
    });
  }
  float loss = 0.f;
  if (ok) {
    // dy = (y - t) / n; dh2 = dy W3 (FP32); dz2 = dh2 s'(z2)
    float yv[16];
    tc_ld16(trow + 128, yv);
    float dy[OUT];
#pragma unroll
    for (int c = 0; c < OUT; c++) {
      const float e = valid ? yv[c] + sm.bias[2 * H + c] - T[3 * row + c] : 0.f;
      loss += 0.5f * e * e;
      dy[c] = e * inv_n;
      sm.dy[t][c] = dy[c];
    }
    float z[H];
    tc_ld64(trow, 64, z);
#pragma unroll
    for (int i = 0; i < H; i++) {
      float dh = 0.f;
#pragma unroll
      for (int c = 0; c < OUT; c++) dh += dy[c] * sm.w3[c * H + i];
      z[i] = dh * silu_grad(z[i] + sm.bias[H + i]);
    }
    put_row64(sm.dz2, t, z);
    put_col<H>(sm.dzT, t, z);
    // dh1 = dz2 W2 (columns 144-207) and the layer-2 gradient
    // sum_s dz2^T [h1 | 1] (columns 64-143, over z2 and y)
    ok = tc_round(sm, phase, [&] {
#pragma unroll
      for (int k = 0; k < 4; k++)
        tc_mma(tmem + 144, tc_desc(sm.dz2 + 256 * k, 128, 1024),
               tc_desc(W2T + 256 * k, 128, 1024), tc_idesc(128, H), k > 0);
#pragma unroll
      for (int k = 0; k < 8; k++)
        tc_mma(tmem + 64, tc_desc(sm.dzT + 256 * k, 128, 2048),
               tc_desc(sm.h1T + 256 * k, 128, 2048), tc_idesc(128, 80), k > 0);
    });
  }
  if (ok) {
    // dz1 = dh1 s'(z1); the layer-1 gradient sum_s dz1^T [x | 1] (208-239)
    float dh[H], z[H];
    tc_ld64(trow, 144, dh);
    tc_ld64(trow, 0, z);
#pragma unroll
    for (int i = 0; i < H; i++) z[i] = dh[i] * silu_grad(z[i] + sm.bias[i]);
    put_col<H>(sm.dzT, t, z);
    ok = tc_round(sm, phase, [&] {
#pragma unroll
      for (int k = 0; k < 8; k++)
        tc_mma(tmem + 208, tc_desc(sm.dzT + 256 * k, 128, 2048),
               tc_desc(sm.xT + 256 * k, 128, 2048), tc_idesc(128, 32), k > 0);
    });
  }
  float *pb = part + (size_t)blockIdx.x * MLP_NPARAM;
  if (ok) {
    // rows 0-63 of the gradients (lanes of warps 0 and 1): one row per thread
    if (warp < 2) {
      float g[16];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        tc_ld16(trow + 64 + 16 * c, g);
#pragma unroll
        for (int i = 0; i < 16; i++) pb[P_W2 + t * H + 16 * c + i] = g[i];
      }
      tc_ld16(trow + 128, g);
      pb[P_B2 + t] = g[0];
      float g1[16], g2[16];
      tc_ld16(trow + 208, g1);
      tc_ld16(trow + 224, g2);
#pragma unroll
      for (int i = 0; i < IN; i++) pb[P_W1 + t * IN + i] = g1[i];
      pb[P_B1 + t] = g2[0];
    }
    // layer 3 in FP32 on the CUDA cores (N = 3): dW3 = dy^T h2, db3
    for (int e = t; e < OUT * H + OUT; e += blockDim.x) {
      float s = 0.f;
      if (e < OUT * H) {
        const int c = e / H, i = e % H;
        for (int r = 0; r < 128; r++)
          s += sm.dy[r][c] * __bfloat162float(*(const __nv_bfloat16 *)(sm.h2 + tc_ofs(r, i, H / 8)));
        pb[P_W3 + e] = s;
      } else {
        for (int r = 0; r < 128; r++) s += sm.dy[r][e - OUT * H];
        pb[P_B3 + e - OUT * H] = s;
      }
    }
  } else {
    if (t == 0) atomicOr((unsigned *)((char *)packed + OFF_STATUS), 1u);
    for (int e = t; e < MLP_NPARAM; e += blockDim.x) pb[e] = 0.f;
    // the last product group must be done before the tensor memory is freed
    (void)tc_wait(&sm.mbar, phase ^ 1u);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) sm.loss[warp] = loss;
  tc_fence_before();
  __syncthreads();
  if (t == 0) part_loss[blockIdx.x] = ((sm.loss[0] + sm.loss[1]) + (sm.loss[2] + sm.loss[3])) * inv_n;
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TR_COLS)
                 : "memory");
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


// FP32 parameters -> packed copy: FP32 biases, BF16 weights in the canonical
// layout (rows = outputs, K = inputs; W3 padded to 16 rows; W2^T with rows =
// inputs), status word cleared.
__global__ void mlp_pack_kernel(const float *__restrict__ P, void *packed) {
  float *bias = (float *)((char *)packed + OFF_B);
  unsigned char *tc = (unsigned char *)packed + OFF_TC;
  const int nw = H * IN + H * H + 16 * H + H * H;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw + NBIAS;
       e += gridDim.x * blockDim.x) {
    if (e >= nw) {
      const int j = e - nw;
      bias[j] = j < H ? P[P_B1 + j] : (j < 2 * H ? P[P_B2 + j - H] : P[P_B3 + j - 2 * H]);
      continue;
    }
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
    } else if (e < H * IN + H * H + 16 * H) {
      const int q = e - H * IN - H * H, r = q / H, k = q % H;
      v = r < OUT ? P[P_W3 + r * H + k] : 0.f;
      ofs = TC_W3 + tc_ofs(r, k, H / 8);
    } else {
      // W2^T: row r = input of layer 2, column k = output
      const int q = e - H * IN - H * H - 16 * H, r = q / H, k = q % H;
      v = P[P_W2 + k * H + r];
      ofs = TC_W2T + tc_ofs(r, k, H / 8);
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
  const int64_t blocks = std::min<int64_t>((n + 127) / 128, 152 * 6);
  mlp_forward_kernel<<<(unsigned)blocks, 128, 0, st>>>(n, X, packed, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_warm(const DomainDesc *D, const BatchDims &dims, int use_prev,
                            cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int64_t want = (dims.max_points + 127) / 128;
  const int64_t cap = std::max<int64_t>(1, 152 * 6 / std::max(1, dims.nd));
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
  mlp_train_kernel<<<nb, 128, sizeof(TrainSmem), st>>>(n, X, T, packed, P, part, part_loss,
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
