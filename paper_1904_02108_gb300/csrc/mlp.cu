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

// Inference.  mode 0: Y[n][3] = y.  mode 1 (warm start of the fixed point):
// du[k] = du_prev[k] + scale * y, with du_prev read from du itself (zero when
// !use_prev).  The domain variant takes n, X, the weights and du from
// D[blockIdx.y].
__device__ void mlp_forward_rows(int64_t n, const float *__restrict__ X, const void *packed,
                                 float *__restrict__ Y, float4 *__restrict__ du, float scale,
                                 int mode, int use_prev, MlpSmem &sm) {
  load_weights(sm, packed);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  for (int64_t row0 = ((int64_t)blockIdx.x * 8 + w) * 16; row0 < n;
       row0 += (int64_t)gridDim.x * 8 * 16) {
    uint32_t xa[4];
    load_x(X, row0, n, xa);
    Fwd f;
    forward16(sm, xa, f);
    // gather the three outputs of rows g and g+8 onto lane t == 0
    const int src0 = g * 4, src1 = g * 4 + 1;
    const float a0 = __shfl_sync(0xffffffffu, f.y[0], src0), a1 = __shfl_sync(0xffffffffu, f.y[1], src0),
                a2 = __shfl_sync(0xffffffffu, f.y[0], src1);
    const float c0 = __shfl_sync(0xffffffffu, f.y[2], src0), c1 = __shfl_sync(0xffffffffu, f.y[3], src0),
                c2 = __shfl_sync(0xffffffffu, f.y[2], src1);
    if (t == 0) {
      const int64_t r[2] = {row0 + g, row0 + g + 8};
      const float v[2][3] = {{a0, a1, a2}, {c0, c1, c2}};
#pragma unroll
      for (int q = 0; q < 2; q++) {
        if (r[q] >= n) continue;
        if (mode == 0) {
          Y[3 * r[q]] = v[q][0];
          Y[3 * r[q] + 1] = v[q][1];
          Y[3 * r[q] + 2] = v[q][2];
        } else {
          float4 d = use_prev ? du[r[q]] : make_float4(0.f, 0.f, 0.f, 0.f);
          d.x += scale * v[q][0];
          d.y += scale * v[q][1];
          d.z += scale * v[q][2];
          du[r[q]] = d;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256)
    mlp_forward_kernel(int64_t n, const float *__restrict__ X, const void *packed,
                       float *__restrict__ Y) {
  __shared__ MlpSmem sm;
  mlp_forward_rows(n, X, packed, Y, nullptr, 0.f, 0, 0, sm);
}

__global__ void __launch_bounds__(256)
    mlp_warm_kernel(const DomainDesc *__restrict__ D, int use_prev) {
  pdl_wait();
  __shared__ MlpSmem sm;
  const DomainDesc &d = D[blockIdx.y];
  if (d.np == 0 || !d.mlp_packed) return;
  mlp_forward_rows(d.np, d.feat, d.mlp_packed, nullptr, d.du, MLP_VSCALE, 1, use_prev, sm);
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

size_t mlp_packed_bytes() { return (size_t)OFF_B + NBIAS * sizeof(float); }

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_pack(const float *P, void *packed, cudaStream_t st) {
  mlp_pack_kernel<<<16, 256, 0, st>>>(P, packed);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(int64_t n, const float *X, const void *packed, float *Y,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 127) / 128, 152 * 8);
  mlp_forward_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, X, packed, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_warm(const DomainDesc *D, const BatchDims &dims, int use_prev,
                            cudaStream_t st) {
  if (dims.max_points <= 0) return cudaSuccess;
  const int64_t want = (dims.max_points + 127) / 128;
  const int64_t cap = std::max<int64_t>(1, 152 * 8 / std::max(1, dims.nd));
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min(want, cap));
  return launch_pdl(mlp_warm_kernel, dim3(bx, dims.nd), dim3(256), 0, st, D, use_prev);
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
