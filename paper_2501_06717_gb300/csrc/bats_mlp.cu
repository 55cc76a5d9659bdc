// bats_mlp.cu -- the learned flux correction's network on tensor cores:
// a 40 -> 64 -> 64 -> 8 MLP with tanh-form GELU (Hendrycks & Gimpel), BF16
// weights and activations, FP32 accumulation.
//
//  * k_mlp_infer: Y = MLP(X) for face feature rows X (BF16, 48 columns: the
//    40 features and 8 zeros) on the 5th-generation tensor cores: per CTA a
//    persistent loop over 128-row tiles; each layer is a tcgen05.mma chain
//    (M = 128, K = 16 per instruction) from shared-memory operands into a
//    tensor-memory accumulator, which eight warps read back (tcgen05.ld;
//    two warps per row, 32 columns each), add the bias to, pass through GELU
//    and store as the next layer's BF16 operand.
//  * k_mlp_train: the mean-squared-error loss and its gradient for a batch;
//    forward and the backward data products on tensor cores (warp-level
//    mma.sync m16n8k16 BF16, activations kept in registers), the weight
//    gradients (outer products over the tile's samples) on the CUDA cores,
//    accumulated per CTA in shared memory and once per CTA in global memory.
//  * k_mlp_adam, k_mlp_pack: the Adam update of the FP32 master weights and
//    the BF16 copies in the layouts the kernels read.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "bats.h"
#include "bats_internal.h"
#include "bats_tc.h"

namespace batsk {

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory weight layout (32-bit words = BF16 pairs), rows padded so the
// B-fragment loads of a warp fall in distinct banks.
constexpr int W1S = 28;  // W1 [64 out][48 in] -> 24 words + 4 pad
constexpr int W2S = 36;  // W2, W2T [64][64] -> 32 words + 4 pad
constexpr int W3S = 36;  // W3 [8][64]
constexpr int W3TS = 12; // W3T [64 in][16 out (8 + zeros)] -> 8 words + 4 pad
struct MlpSmem {
  uint32_t w1[64 * W1S];
  uint32_t w2[64 * W2S];
  uint32_t w3[8 * W3S];
  uint32_t w2t[64 * W2S];
  uint32_t w3t[64 * W3TS];
  float b1[64], b2[64], b3[8];
};

// Copy the packed device weights (MlpDev, unpadded rows) into shared memory.
__device__ void load_mlp_smem(const MlpDev& m, MlpSmem& s) {
  for (int e = threadIdx.x; e < 64 * 24; e += blockDim.x) s.w1[(e / 24) * W1S + e % 24] = m.w1[e];
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    s.w2[(e / 32) * W2S + e % 32] = m.w2[e];
    s.w2t[(e / 32) * W2S + e % 32] = m.w2t[e];
  }
  for (int e = threadIdx.x; e < 8 * 32; e += blockDim.x) s.w3[(e / 32) * W3S + e % 32] = m.w3[e];
  for (int e = threadIdx.x; e < 64 * 8; e += blockDim.x) s.w3t[(e / 8) * W3TS + e % 8] = m.w3t[e];
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    s.b1[e] = m.b1[e];
    s.b2[e] = m.b2[e];
  }
  for (int e = threadIdx.x; e < 8; e += blockDim.x) s.b3[e] = m.b3[e];
}

// Forward of one 16-row tile.  a1: A fragments of the inputs (3 k-tiles).
// Outputs: z1, z2 (pre-activations, C layout, 8 n-tiles x 4), a2, a3 (BF16
// A fragments of H1, H2, 4 k-tiles x 4), y (C layout of the 8 outputs).
template <bool KEEP>
__device__ __forceinline__ void mlp_tile_forward(const MlpSmem& s, const uint32_t a1[3][4], float z1[8][4],
                                                 float z2[8][4], uint32_t a2[4][4], uint32_t a3[4][4],
                                                 float y[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    const float bl = s.b1[nt * 8 + 2 * t], bh = s.b1[nt * 8 + 2 * t + 1];
    acc[nt][0] = bl; acc[nt][1] = bh; acc[nt][2] = bl; acc[nt][3] = bh;
#pragma unroll
    for (int kt = 0; kt < 3; kt++)
      mma_bf16(acc[nt], a1[kt], s.w1[(nt * 8 + g) * W1S + kt * 8 + t], s.w1[(nt * 8 + g) * W1S + kt * 8 + 4 + t]);
  }
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    if (KEEP) {
#pragma unroll
      for (int r = 0; r < 4; r++) z1[nt][r] = acc[nt][r];
    }
    const int kt = nt >> 1, hi = nt & 1;
    a2[kt][hi * 2 + 0] = gelu2_pack(acc[nt][0], acc[nt][1]);
    a2[kt][hi * 2 + 1] = gelu2_pack(acc[nt][2], acc[nt][3]);
  }
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    const float bl = s.b2[nt * 8 + 2 * t], bh = s.b2[nt * 8 + 2 * t + 1];
    acc[nt][0] = bl; acc[nt][1] = bh; acc[nt][2] = bl; acc[nt][3] = bh;
#pragma unroll
    for (int kt = 0; kt < 4; kt++)
      mma_bf16(acc[nt], a2[kt], s.w2[(nt * 8 + g) * W2S + kt * 8 + t], s.w2[(nt * 8 + g) * W2S + kt * 8 + 4 + t]);
  }
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    if (KEEP) {
#pragma unroll
      for (int r = 0; r < 4; r++) z2[nt][r] = acc[nt][r];
    }
    const int kt = nt >> 1, hi = nt & 1;
    a3[kt][hi * 2 + 0] = gelu2_pack(acc[nt][0], acc[nt][1]);
    a3[kt][hi * 2 + 1] = gelu2_pack(acc[nt][2], acc[nt][3]);
  }
  const float bl = s.b3[2 * t], bh = s.b3[2 * t + 1];
  y[0] = bl; y[1] = bh; y[2] = bl; y[3] = bh;
#pragma unroll
  for (int kt = 0; kt < 4; kt++) mma_bf16(y, a3[kt], s.w3[g * W3S + kt * 8 + t], s.w3[g * W3S + kt * 8 + 4 + t]);
}

constexpr int TC_TILE = 128;             // rows per tile (MMA M = tensor-memory lanes)
constexpr int TC_TMEM_COLS = 64;         // one FP32 accumulator of N = 64 (reused by all three layers)
struct TcSmem {
  alignas(128) uint8_t x[TC_TILE * 96];  // X tile, K = 48
  alignas(128) uint8_t h[TC_TILE * 128]; // hidden activations, K = 64 (H1, then H2)
  alignas(128) uint8_t w1[64 * 96];      // B of layer 1: N = 64, K = 48
  alignas(128) uint8_t w2[64 * 128];     // B of layer 2: N = 64, K = 64
  alignas(128) uint8_t w3[16 * 128];     // B of layer 3: N = 16 (8 outputs, 8 zero rows), K = 64
  float b1[64], b2[64], b3[8];
  uint64_t bar;
  uint32_t tmem;
};

// Bias, GELU and BF16 rounding of 32 accumulator columns c0..c0+31 of this
// thread's lane (at taddr) into row `row` of the canonical K = 64 tile h.
__device__ __forceinline__ void tc_hidden_cols(uint32_t taddr, const float* bias, uint8_t* h, int row, int c0) {
#pragma unroll
  for (int q = 0; q < 2; q++) {
    float v[16];
    tmem_ld16(taddr + 16 * q, v);
#pragma unroll
    for (int c = 0; c < 2; c++) {
      uint4 o;
      const float* b = bias + c0 + 16 * q + 8 * c;
      const float* z = v + 8 * c;
      o.x = gelu2_pack(z[0] + b[0], z[1] + b[1]);
      o.y = gelu2_pack(z[2] + b[2], z[3] + b[3]);
      o.z = gelu2_pack(z[4] + b[4], z[5] + b[5]);
      o.w = gelu2_pack(z[6] + b[6], z[7] + b[7]);
      *reinterpret_cast<uint4*>(h + cm_off(row, c0 / 8 + 2 * q + c, SBO_K64)) = o;
    }
  }
}

// Y[n][8] = MLP(X[n][48] BF16), 256 threads per CTA, persistent over tiles.
// Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (the tile rows it may
// access) and accumulator columns 32 (w / 4) .. + 31, so two warps share each
// row's epilogue.  Thread 0 issues the MMAs; every wait is bounded
// (ERR_TIMEOUT in err), after which the CTA waits once more for its MMAs,
// frees its tensor memory and returns.
constexpr int TC_THREADS = 256;
__global__ void __launch_bounds__(TC_THREADS, 4) k_mlp_infer(const uint32_t* __restrict__ X, float* __restrict__ Y,
                                                             int64_t n, MlpDev m, int32_t* err) {
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(tc_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int lg = warp & 3, ch = warp >> 2;   // lane group, column half
  const int trow = 32 * lg + (tid & 31);     // the tile row of this thread's lane
  // weights into the canonical layouts (16-byte chunks), biases
  for (int e = tid; e < 64 * 6; e += TC_THREADS) {
    const int r = e / 6, kc = e % 6;
    *reinterpret_cast<uint4*>(s.w1 + cm_off(r, kc, SBO_K48)) = *reinterpret_cast<const uint4*>(m.w1 + r * 24 + kc * 4);
  }
  for (int e = tid; e < 64 * 8; e += TC_THREADS) {
    const int r = e / 8, kc = e % 8;
    *reinterpret_cast<uint4*>(s.w2 + cm_off(r, kc, SBO_K64)) = *reinterpret_cast<const uint4*>(m.w2 + r * 32 + kc * 4);
  }
  for (int e = tid; e < 16 * 8; e += TC_THREADS) {
    const int r = e / 8, kc = e % 8;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(s.w3 + cm_off(r, kc, SBO_K64)) =
        r < 8 ? *reinterpret_cast<const uint4*>(m.w3 + r * 32 + kc * 4) : z;
  }
  if (tid < 64) {
    s.b1[tid] = m.b1[tid];
    s.b2[tid] = m.b2[tid];
  }
  if (tid < 8) s.b3[tid] = m.b3[tid];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&s.tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init_tc(&s.bar);
  proxy_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem;
  const uint32_t tlanes = tmem + (static_cast<uint32_t>(32 * lg) << 16);  // this warp's 32 lanes
  const uint32_t xs = tc_saddr(s.x), hs = tc_saddr(s.h);
  const uint32_t w1s = tc_saddr(s.w1), w2s = tc_saddr(s.w2), w3s = tc_saddr(s.w3);
  constexpr uint32_t ID64 = umma_idesc_bf16(TC_TILE, 64), ID16 = umma_idesc_bf16(TC_TILE, 16);
  uint32_t phase = 0;
  bool failed = false;
  const int64_t ntiles = (n + TC_TILE - 1) / TC_TILE;
  // input: thread tid carries half (three 16-byte chunks) of row tid % 128,
  // loaded one tile ahead (zeros past n)
  const int xr = tid & (TC_TILE - 1), xk0 = 3 * (tid / TC_TILE);
  auto load_part = [&](int64_t r, uint4 xv[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) xv[k] = make_uint4(0u, 0u, 0u, 0u);
    if (r < n) {
      const uint4* src = reinterpret_cast<const uint4*>(X + r * 24) + xk0;
#pragma unroll
      for (int k = 0; k < 3; k++) xv[k] = src[k];
    }
  };
  uint4 xn[3];
  load_part(static_cast<int64_t>(blockIdx.x) * TC_TILE + xr, xn);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // the input chunks into the canonical K = 48 tile; the next tile's on
    // their way while this tile runs through the three layers
#pragma unroll
    for (int k = 0; k < 3; k++) *reinterpret_cast<uint4*>(s.x + cm_off(xr, xk0 + k, SBO_K48)) = xn[k];
    load_part(tile * TC_TILE + xr + static_cast<int64_t>(gridDim.x) * TC_TILE, xn);
#pragma unroll 1
    for (int layer = 0; layer < 3; layer++) {
      // operands written by the threads -> visible to the tensor cores
      proxy_fence_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        if (layer == 0) {
#pragma unroll
          for (int k = 0; k < 3; k++)
            umma_bf16(tmem, umma_sdesc(xs + 256 * k, 128, SBO_K48), umma_sdesc(w1s + 256 * k, 128, SBO_K48), ID64,
                      k > 0);
        } else {
          const uint32_t ws = layer == 1 ? w2s : w3s;
#pragma unroll
          for (int k = 0; k < 4; k++)
            umma_bf16(tmem, umma_sdesc(hs + 256 * k, 128, SBO_K64), umma_sdesc(ws + 256 * k, 128, SBO_K64),
                      layer == 1 ? ID64 : ID16, k > 0);
        }
        umma_commit(&s.bar);
      }
      const bool got = mbar_wait_bounded_tc(&s.bar, phase, err);
      if (__syncthreads_or(!got)) {
        failed = true;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      if (layer < 2) {
        tc_hidden_cols(tlanes + 32 * ch, layer == 0 ? s.b1 : s.b2, s.h, trow, 32 * ch);
      } else if (ch == 0) {
        float v[16];
        tmem_ld16(tlanes, v);
        const int64_t row = tile * TC_TILE + trow;
        if (row < n) {
          float4* dst = reinterpret_cast<float4*>(Y + row * 8);
          dst[0] = make_float4(v[0] + s.b3[0], v[1] + s.b3[1], v[2] + s.b3[2], v[3] + s.b3[3]);
          dst[1] = make_float4(v[4] + s.b3[4], v[5] + s.b3[5], v[6] + s.b3[6], v[7] + s.b3[7]);
        }
      }
    }
    if (failed) break;
  }
  // an MMA may still run after a timed-out wait: wait for it once more
  if (failed && tid == 0) mbar_wait_bounded_tc(&s.bar, phase, err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// Loss sum and gradient of L = (1/(8 n_total)) sum (y - t)^2 over rows
// [0, n) of X (FP32 [n][40], rounded to BF16 on load) and T (FP32 [n][8]).
// grad (FP32 [NPARAM], zeroed by the caller) and loss_sum accumulate.
constexpr int TRAIN_WARPS = 4;
struct TrainTile {           // per-warp staging of one 16-sample tile, FP32
  float x[16][40];
  float h1[16][64];
  float h2[16][64];
  float dz1[16][64];
  float dz2[16][64];
  float dy[16][8];
};

__global__ void __launch_bounds__(TRAIN_WARPS * 32) k_mlp_train(const float* __restrict__ X,
                                                                const float* __restrict__ T, int64_t n,
                                                                double inv_count, MlpDev m,
                                                                float* __restrict__ grad,
                                                                double* __restrict__ loss_sum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
  TrainTile* tiles = reinterpret_cast<TrainTile*>(smem_raw + sizeof(MlpSmem));
  float* sgrad = reinterpret_cast<float*>(smem_raw + sizeof(MlpSmem) + TRAIN_WARPS * sizeof(TrainTile));
  load_mlp_smem(m, s);
  for (int e = threadIdx.x; e < MLP_NPARAM; e += blockDim.x) sgrad[e] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  TrainTile& tt = tiles[w];
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const float scale = static_cast<float>(2.0 * inv_count);
  double lsum = 0.0;
  for (int64_t r0 = warp * 16; r0 < n; r0 += nwarps * 16) {
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    // inputs as BF16 A fragments (and their FP32 values for the W1 gradient)
    uint32_t a1[3][4];
#pragma unroll
    for (int kt = 0; kt < 3; kt++) {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int64_t r = (q & 1) ? rb : ra;
        const int col = kt * 16 + (q >> 1) * 8 + 2 * t;
        float v0 = 0.f, v1 = 0.f;
        if (r < n && col < MLP_IN) {
          v0 = X[r * MLP_IN + col];
          v1 = X[r * MLP_IN + col + 1];
        }
        a1[kt][q] = pack_bf16(v0, v1);
        if (col < MLP_IN) {
          const int rr = (q & 1) ? g + 8 : g;
          tt.x[rr][col] = bf16_lo(a1[kt][q]);
          tt.x[rr][col + 1] = bf16_hi(a1[kt][q]);
        }
      }
    }
    float z1[8][4], z2[8][4], y[4];
    uint32_t a2[4][4], a3[4][4];
    mlp_tile_forward<true>(s, a1, z1, z2, a2, a3, y);
    // dL/dy
    float dy[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t r = q < 2 ? ra : rb;
      const int col = 2 * t + (q & 1);
      float e = 0.f;
      if (r < n) e = y[q] - T[r * 8 + col];
      lsum += static_cast<double>(e) * e;
      dy[q] = scale * e;
      tt.dy[q < 2 ? g : g + 8][col] = dy[q];
    }
    // stage H1, H2 (the BF16 values the next layers saw)
#pragma unroll
    for (int kt = 0; kt < 4; kt++)
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int rr = (q & 1) ? g + 8 : g;
        const int col = kt * 16 + (q >> 1) * 8 + 2 * t;
        tt.h1[rr][col] = bf16_lo(a2[kt][q]);
        tt.h1[rr][col + 1] = bf16_hi(a2[kt][q]);
        tt.h2[rr][col] = bf16_lo(a3[kt][q]);
        tt.h2[rr][col + 1] = bf16_hi(a3[kt][q]);
      }
    // dH2 = dY W3 (K = 8 outputs, zero-padded to 16), dZ2 = dH2 * gelu'(Z2)
    uint32_t ady[4] = {pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), 0u, 0u};
    uint32_t adz2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, ady, s.w3t[(nt * 8 + g) * W3TS + t], s.w3t[(nt * 8 + g) * W3TS + 4 + t]);
#pragma unroll
      for (int q = 0; q < 4; q++) c[q] *= gelu_grad_f(z2[nt][q]);
      const int kt = nt >> 1, hi = nt & 1;
      adz2[kt][hi * 2 + 0] = pack_bf16(c[0], c[1]);
      adz2[kt][hi * 2 + 1] = pack_bf16(c[2], c[3]);
      const int col = nt * 8 + 2 * t;
      tt.dz2[g][col] = c[0];
      tt.dz2[g][col + 1] = c[1];
      tt.dz2[g + 8][col] = c[2];
      tt.dz2[g + 8][col + 1] = c[3];
    }
    // dH1 = dZ2 W2, dZ1 = dH1 * gelu'(Z1)
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < 4; kt++)
        mma_bf16(c, adz2[kt], s.w2t[(nt * 8 + g) * W2S + kt * 8 + t], s.w2t[(nt * 8 + g) * W2S + kt * 8 + 4 + t]);
      const int col = nt * 8 + 2 * t;
      tt.dz1[g][col] = c[0] * gelu_grad_f(z1[nt][0]);
      tt.dz1[g][col + 1] = c[1] * gelu_grad_f(z1[nt][1]);
      tt.dz1[g + 8][col] = c[2] * gelu_grad_f(z1[nt][2]);
      tt.dz1[g + 8][col + 1] = c[3] * gelu_grad_f(z1[nt][3]);
    }
    __syncwarp();
    // weight and bias gradients: sums over the tile's 16 samples
    for (int e = lane; e < MLP_NPARAM; e += 32) {
      float acc = 0.f;
      if (e < 2560) {
        const int o = e / 40, i = e % 40;
#pragma unroll 4
        for (int r = 0; r < 16; r++) acc += tt.dz1[r][o] * tt.x[r][i];
      } else if (e < 2624) {
        const int o = e - 2560;
        for (int r = 0; r < 16; r++) acc += tt.dz1[r][o];
      } else if (e < 6720) {
        const int o = (e - 2624) >> 6, i = (e - 2624) & 63;
#pragma unroll 4
        for (int r = 0; r < 16; r++) acc += tt.dz2[r][o] * tt.h1[r][i];
      } else if (e < 6784) {
        const int o = e - 6720;
        for (int r = 0; r < 16; r++) acc += tt.dz2[r][o];
      } else if (e < 7296) {
        const int o = (e - 6784) >> 6, i = (e - 6784) & 63;
#pragma unroll 4
        for (int r = 0; r < 16; r++) acc += tt.dy[r][o] * tt.h2[r][i];
      } else {
        const int o = e - 7296;
        for (int r = 0; r < 16; r++) acc += tt.dy[r][o];
      }
      atomicAdd(&sgrad[e], acc);
    }
    __syncwarp();
  }
  // loss: warp sum, then one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(loss_sum, lsum);
  __syncthreads();
  for (int e = threadIdx.x; e < MLP_NPARAM; e += blockDim.x) atomicAdd(&grad[e], sgrad[e]);
}

// Adam (Kingma & Ba 2015) on the FP32 master weights, bias-corrected.
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= MLP_NPARAM) return;
  float gv = gr[e];
  float a = b1 * m1[e] + (1.f - b1) * gv;
  float b = b2 * m2[e] + (1.f - b2) * gv * gv;
  m1[e] = a;
  m2[e] = b;
  p[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// FP32 master weights (W1 [64][40], b1, W2 [64][64], b2, W3 [8][64], b3) ->
// BF16 pair layouts: w1 [64][24] (inputs 40..47 zero), w2 [64][32],
// w3 [8][32], w2t [64][32] (transposed), w3t [64][8] (transposed, outputs
// 8..15 zero), and the FP32 biases.
__global__ void k_mlp_pack(const float* __restrict__ P, MlpDev m) {
  const float* W1 = P;
  const float* B1 = W1 + 64 * 40;
  const float* W2 = B1 + 64;
  const float* B2 = W2 + 64 * 64;
  const float* W3 = B2 + 64;
  const float* B3 = W3 + 8 * 64;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 32; e += gridDim.x * blockDim.x) {
    const int r = e / 32, c = e % 32;
    if (c < 24) {
      float v0 = 2 * c < 40 ? W1[r * 40 + 2 * c] : 0.f, v1 = 2 * c + 1 < 40 ? W1[r * 40 + 2 * c + 1] : 0.f;
      m.w1[r * 24 + c] = pack_bf16(v0, v1);
    }
    m.w2[r * 32 + c] = pack_bf16(W2[r * 64 + 2 * c], W2[r * 64 + 2 * c + 1]);
    m.w2t[r * 32 + c] = pack_bf16(W2[(2 * c) * 64 + r], W2[(2 * c + 1) * 64 + r]);
    if (r < 8) m.w3[r * 32 + c] = pack_bf16(W3[r * 64 + 2 * c], W3[r * 64 + 2 * c + 1]);
    if (c < 8) {
      float v0 = 2 * c < 8 ? W3[(2 * c) * 64 + r] : 0.f, v1 = 2 * c + 1 < 8 ? W3[(2 * c + 1) * 64 + r] : 0.f;
      m.w3t[r * 8 + c] = pack_bf16(v0, v1);
    }
    if (e < 64) {
      m.b1[e] = B1[e];
      m.b2[e] = B2[e];
    }
    if (e < 8) m.b3[e] = B3[e];
  }
}

// FP32 rows of 40 -> BF16 rows of 48 (24 words, the last 4 words zero).
__global__ void k_rows_to_bf16(const float* __restrict__ X, uint32_t* __restrict__ Xb, int64_t n) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * 24;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / 24;
    const int c = static_cast<int>(e % 24);
    Xb[e] = c < 20 ? pack_bf16(X[r * 40 + 2 * c], X[r * 40 + 2 * c + 1]) : 0u;
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers.

size_t mlp_train_smem() { return sizeof(MlpSmem) + TRAIN_WARPS * sizeof(TrainTile) + MLP_NPARAM * sizeof(float); }

cudaError_t mlp_setup() {
  return cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(mlp_train_smem()));
}
cudaError_t launch_mlp_pack(const float* P, const MlpDev& m, cudaStream_t st) {
  k_mlp_pack<<<8, 256, 0, st>>>(P, m);
  return cudaGetLastError();
}
// X: n rows of 24 words (16-byte aligned), Y: n rows of 8 floats (16-byte
// aligned); 4 CTAs per SM at most (shared memory 45 KB, tensor memory 64 of
// the SM's 512 columns each).
cudaError_t launch_mlp_infer(const uint32_t* X, float* Y, int64_t n, const MlpDev& m, int nsm, int32_t* err,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) return cudaErrorInvalidValue;
  const int64_t tiles = (n + TC_TILE - 1) / TC_TILE;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(nsm) * 4));
  k_mlp_infer<<<grid, TC_THREADS, sizeof(TcSmem), st>>>(X, Y, n, m, err);
  return cudaGetLastError();
}
cudaError_t launch_mlp_train(const float* X, const float* T, int64_t n, const MlpDev& m, float* grad, double* loss,
                             int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t tiles = (n + 15) / 16;
  int grid = static_cast<int>(std::min<int64_t>((tiles + TRAIN_WARPS - 1) / TRAIN_WARPS, static_cast<int64_t>(nsm)));
  k_mlp_train<<<grid, TRAIN_WARPS * 32, mlp_train_smem(), st>>>(X, T, n, 1.0 / (8.0 * static_cast<double>(n)), m,
                                                                 grad, loss);
  return cudaGetLastError();
}
cudaError_t launch_mlp_adam(float* p, const float* g, float* m1, float* m2, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float c1 = 1.f - powf(b1, static_cast<float>(step)), c2 = 1.f - powf(b2, static_cast<float>(step));
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(p, g, m1, m2, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_rows_to_bf16(const float* X, uint32_t* Xb, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = static_cast<int>(std::min<int64_t>((n * 24 + 255) / 256, 4096));
  k_rows_to_bf16<<<grid, 256, 0, st>>>(X, Xb, n);
  return cudaGetLastError();
}

// Device weight set: one allocation holding the BF16 layouts and biases.
cudaError_t mlp_alloc(MlpDev* w) {
  const size_t words = 64 * 24 + 64 * 32 + 8 * 32 + 64 * 32 + 64 * 8;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, words * 4 + (64 + 64 + 8) * 4);
  if (e != cudaSuccess) return e;
  uint32_t* u = static_cast<uint32_t*>(p);
  w->w1 = u;
  w->w2 = w->w1 + 64 * 24;
  w->w3 = w->w2 + 64 * 32;
  w->w2t = w->w3 + 8 * 32;
  w->w3t = w->w2t + 64 * 32;
  float* f = reinterpret_cast<float*>(w->w3t + 64 * 8);
  w->b1 = f;
  w->b2 = f + 64;
  w->b3 = f + 128;
  return cudaMemsetAsync(p, 0, words * 4 + (64 + 64 + 8) * 4);
}
void mlp_free(MlpDev* w) {
  if (w->w1) cudaFree(w->w1);
  std::memset(w, 0, sizeof(*w));
}

// Seeded initialisation: hidden layers N(0, 1/fan_in), biases and the output
// layer zero (the initial network adds nothing).
void mlp_init_params(uint64_t seed, float* P) {
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::memset(P, 0, sizeof(float) * MLP_NPARAM);
  for (int e = 0; e < 64 * 40; e++) P[e] = static_cast<float>(nd(rng) / std::sqrt(40.0));
  float* W2 = P + 64 * 40 + 64;
  for (int e = 0; e < 64 * 64; e++) W2[e] = static_cast<float>(nd(rng) / std::sqrt(64.0));
}

}  // namespace batsk

using namespace batsk;

struct bats_mlp {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nsm = 1;
  float *P = nullptr, *M1 = nullptr, *M2 = nullptr, *G = nullptr;
  double* loss = nullptr;
  MlpDev w{};
  int step = 0;
  float *X = nullptr, *T = nullptr, *Y = nullptr;
  uint32_t* Xb = nullptr;
  int64_t cap = 0;
  int32_t* errw = nullptr;  // device error bits of the inference kernel (ERR_TIMEOUT)
};

namespace {

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int mlp_reserve(bats_mlp_t* m, int64_t n) {
  if (n <= m->cap) return BATS_OK;
  cudaFree(m->X);
  cudaFree(m->T);
  cudaFree(m->Y);
  cudaFree(m->Xb);
  m->X = m->T = m->Y = nullptr;
  m->Xb = nullptr;
  m->cap = 0;
  if (cudaMalloc(&m->X, n * 40 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->T, n * 8 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->Y, n * 8 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->Xb, n * 24 * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return BATS_ERR_OUT_OF_MEMORY;
  }
  m->cap = n;
  return BATS_OK;
}

int copy_in(bats_mlp_t* m, float* dst, const float* src, size_t count) {
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(float),
                                  dev_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream);
  return e == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

int grad_pass(bats_mlp_t* m, const float* X, const float* T, int64_t n) {
  if (!X || !T || n <= 0) return BATS_ERR_INVALID_ARG;
  int rc = mlp_reserve(m, n);
  if (rc) return rc;
  if ((rc = copy_in(m, m->X, X, static_cast<size_t>(n) * 40)) || (rc = copy_in(m, m->T, T, static_cast<size_t>(n) * 8)))
    return rc;
  if (cudaMemsetAsync(m->G, 0, sizeof(float) * MLP_NPARAM, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream) != cudaSuccess ||
      launch_mlp_train(m->X, m->T, n, m->w, m->G, m->loss, m->nsm, m->stream) != cudaSuccess)
    return BATS_ERR_CUDA;
  return BATS_OK;
}

}  // namespace

extern "C" {

int bats_mlp_create(const float* params, uint64_t seed, void* cuda_stream, bats_mlp_t** out) {
  if (!out) return BATS_ERR_INVALID_ARG;
  *out = nullptr;
  bats_mlp_t* m = new bats_mlp_t();
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && !m->stream) {
    e = cudaStreamCreate(&m->stream);
    m->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = mlp_setup();
  if (e == cudaSuccess) e = cudaMalloc(&m->P, sizeof(float) * MLP_NPARAM * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->errw, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(m->errw, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = mlp_alloc(&m->w);
  if (e != cudaSuccess) {
    bats_mlp_destroy(m);
    return BATS_ERR_CUDA;
  }
  m->M1 = m->P + MLP_NPARAM;
  m->M2 = m->P + 2 * MLP_NPARAM;
  m->G = m->P + 3 * MLP_NPARAM;
  int rc;
  if (params) {
    rc = bats_mlp_set_params(m, params);
  } else {
    std::vector<float> h(MLP_NPARAM);
    mlp_init_params(seed, h.data());
    rc = bats_mlp_set_params(m, h.data());
  }
  if (rc) {
    bats_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return BATS_OK;
}

void bats_mlp_destroy(bats_mlp_t* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  cudaFree(m->P);
  cudaFree(m->loss);
  cudaFree(m->errw);
  cudaFree(m->X);
  cudaFree(m->T);
  cudaFree(m->Y);
  cudaFree(m->Xb);
  mlp_free(&m->w);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

int bats_mlp_set_params(bats_mlp_t* m, const float* params) {
  if (!m || !params) return BATS_ERR_INVALID_ARG;
  if (copy_in(m, m->P, params, MLP_NPARAM)) return BATS_ERR_CUDA;
  if (cudaMemsetAsync(m->M1, 0, sizeof(float) * 2 * MLP_NPARAM, m->stream) != cudaSuccess) return BATS_ERR_CUDA;
  m->step = 0;
  if (launch_mlp_pack(m->P, m->w, m->stream) != cudaSuccess) return BATS_ERR_CUDA;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

int bats_mlp_get_params(bats_mlp_t* m, float* params) {
  if (!m || !params) return BATS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(params, m->P, sizeof(float) * MLP_NPARAM,
                                  dev_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

// GELU self-check: y[i] = the kernels' packed-pair GELU (BF16 results) of x[i].
__global__ void k_debug_gelu(const float* x, int n, float* y) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float x1 = i + 1 < n ? x[i + 1] : 0.f;
  const uint32_t r = gelu2_pack(x[i], x1);
  y[i] = bf16_lo(r);
  if (i + 1 < n) y[i + 1] = bf16_hi(r);
}

int bats_debug_gelu(const float* x, int n, float* y) {
  if (!x || !y || n <= 0) return BATS_ERR_INVALID_ARG;
  float *xd = nullptr, *yd = nullptr;
  cudaError_t e = cudaMalloc(&xd, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&yd, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(xd, x, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_debug_gelu<<<(n / 2 + 256) / 256, 256>>>(xd, n, yd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y, yd, n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(xd);
  cudaFree(yd);
  return e == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

int bats_mlp_forward(bats_mlp_t* m, const float* X, int64_t n, float* Y) {
  if (!m || !X || !Y || n <= 0) return BATS_ERR_INVALID_ARG;
  int rc = mlp_reserve(m, n);
  if (rc) return rc;
  if ((rc = copy_in(m, m->X, X, static_cast<size_t>(n) * 40))) return rc;
  cudaError_t e = launch_rows_to_bf16(m->X, m->Xb, n, m->stream);
  if (e == cudaSuccess) e = launch_mlp_infer(m->Xb, m->Y, n, m->w, m->nsm, m->errw, m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Y, m->Y, sizeof(float) * n * 8, dev_ptr(Y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        m->stream);
  int32_t eb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&eb, m->errw, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return BATS_ERR_CUDA;
  if (eb) {
    cudaMemsetAsync(m->errw, 0, sizeof(int32_t), m->stream);
    return BATS_ERR_TIMEOUT;
  }
  return BATS_OK;
}

int bats_mlp_loss_grad(bats_mlp_t* m, const float* X, const float* T, int64_t n, float* grad, double* loss) {
  if (!m) return BATS_ERR_INVALID_ARG;
  int rc = grad_pass(m, X, T, n);
  if (rc) return rc;
  double ls = 0.0;
  cudaError_t e = cudaMemcpyAsync(&ls, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, m->G, sizeof(float) * MLP_NPARAM,
                        dev_ptr(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return BATS_ERR_CUDA;
  if (loss) *loss = ls / (8.0 * static_cast<double>(n));
  return BATS_OK;
}

int bats_mlp_train_step(bats_mlp_t* m, const float* X, const float* T, int64_t n, float lr, double* loss) {
  if (!m || !(lr >= 0.f)) return BATS_ERR_INVALID_ARG;
  int rc = grad_pass(m, X, T, n);
  if (rc) return rc;
  m->step++;
  if (launch_mlp_adam(m->P, m->G, m->M1, m->M2, lr, m->step, m->stream) != cudaSuccess ||
      launch_mlp_pack(m->P, m->w, m->stream) != cudaSuccess)
    return BATS_ERR_CUDA;
  if (loss) {
    double ls = 0.0;
    if (cudaMemcpyAsync(&ls, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
      return BATS_ERR_CUDA;
    *loss = ls / (8.0 * static_cast<double>(n));
  }
  return BATS_OK;
}

}  // extern "C"
