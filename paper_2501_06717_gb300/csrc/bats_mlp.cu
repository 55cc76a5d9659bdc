// bats_mlp.cu -- the learned flux correction's network on tensor cores:
// a 40 -> 64 -> 64 -> 8 MLP with tanh-form GELU (Hendrycks & Gimpel), BF16
// weights and activations, FP32 accumulation.
//
//  * k_mlp_infer: Y = MLP(X) for face feature rows X (BF16, 48 columns: the
//    40 features and 8 zeros) on the 5th-generation tensor cores: one
//    persistent CTA per SM with four streams of 128-row tiles; each layer is
//    a tcgen05.mma chain (M = 128, K = 16 per instruction) with the A operand
//    (the inputs, then the activations) in tensor memory and the weights in
//    shared memory, into a tensor-memory accumulator that the stream's
//    threads read back (tcgen05.ld, one row per thread) and write over with
//    the next layer's BF16 operand (tcgen05.st); biases folded into the
//    products.
//  * k_mlp_train_tc, k_mlp_grad_reduce: the mean-squared-error loss and its
//    gradient for a batch, every product on tcgen05 (the weight gradients
//    with the samples as K), per-CTA partial sums added in a fixed order.
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

constexpr int TC_TILE = 128;        // rows per tile (MMA M = tensor-memory lanes)
constexpr int TC_STREAMS = 4;       // tiles in flight per CTA (one CTA per SM)
constexpr int TC_THREADS = 32 * 4 * TC_STREAMS;  // four warps per stream
constexpr int TC_TMEM_COLS = 512;   // two regions of 64 columns per stream
struct TcSmem {
  alignas(128) uint8_t w1[64 * 96];   // B of layer 1: N = 64, K = 48
  alignas(128) uint8_t w2[64 * 160];  // B of layer 2: N = 64, K = 80 (weights halved)
  alignas(128) uint8_t w3[16 * 160];  // B of layer 3: N = 16 (8 outputs, 8 zero rows), K = 80 (halved)
  uint64_t accready[TC_STREAMS];      // tcgen05.commit: the stream's layer is in tensor memory
  uint32_t tmem;
};

__device__ __forceinline__ void mbar_init_count(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_saddr(bar)), "r"(count) : "memory");
}
// D[tmem] (+)= A B^T for one K = 16 slice, A (M = 128 rows = lanes, K packed
// two BF16 per 32-bit column, 8 columns per slice) in tensor memory
__device__ __forceinline__ void umma_bf16_ts(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
      "r"(atmem), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// 16 + 8 (x24) or 32 + 8 (x40) words into consecutive columns of this
// thread's lane, waiting for the stores
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Twice the GELU of the 64 accumulator columns of this thread's lane at taddr
// (the biases came in through the products), as 32 BF16 pairs written back
// over the first 32 of those columns, then the bias column pair (ones) and
// zeros: the next layer's A, K = 80.
__device__ __forceinline__ void tc_hidden_row(uint32_t taddr) {
  uint32_t h[40];
#pragma unroll
  for (int q = 0; q < 2; q++) {
    float z[32];
    tmem_ld32(taddr + 32 * q, z);
#pragma unroll
    for (int c = 0; c < 16; c++) h[16 * q + c] = gelu2x_pack(z[2 * c], z[2 * c + 1]);
  }
  h[32] = pack_bf16(1.f, 1.f);
#pragma unroll
  for (int c = 33; c < 40; c++) h[c] = 0u;
  tmem_st16(taddr, h);
  tmem_st16(taddr + 16, h + 16);
  tmem_st8(taddr + 32, h + 32);
  tmem_st_wait();
}

// Y[n][8] = MLP(X[n][48] BF16), one persistent CTA per SM: TC_STREAMS
// streams of four warps, each stream with a tile of its own in flight (the
// CTA's tiles k = s, s + TC_STREAMS, ..), thread t of the stream owning row t
// (tensor-memory lane t; warp w reads and writes lanes 32 (w % 4) ..).  Every
// A operand lives in tensor memory, written by the stream's threads
// (tcgen05.st): the inputs, then each layer's activations over the
// accumulator they came from, so shared memory carries only the weights.  A
// stream's two 64-column regions alternate: layer 1 reads X from region 1
// into region 0, layer 2 reads H1 (region 0) into region 1, layer 3 reads H2
// (region 1) into region 0.  Each stream issues its own MMAs (one elected
// thread of its first warp, after a barrier of the stream's 128 threads) and
// commits them to its own mbarrier, so a stream waits for its own products
// only.  The biases ride in the products (ones in the bias columns, the bias
// pairs in the weights); the hidden activations are twice the GELU (the next
// layer's weights halved), a hidden pair costing one packed-FP32 chain
// around two tanh.approx.f32.  Every wait is bounded (ERR_TIMEOUT in err); a
// stream whose wait ran out (in any of its threads: the stream's barrier
// carries the flag) waits once more for its MMAs in flight and stops, and
// the CTA frees its tensor memory and returns.
__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_infer(const uint32_t* __restrict__ X, float* __restrict__ Y,
                                                             int64_t n, MlpDev m, int32_t* err) {
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~uintptr_t(127));
  const int t = threadIdx.x, warp = t >> 5;
  // weights into the canonical layouts (16-byte chunks)
  for (int e = t; e < 64 * 6; e += TC_THREADS) {
    const int r = e / 6, kc = e % 6;
    *reinterpret_cast<uint4*>(s.w1 + cm_off(r, kc, SBO_K48)) = *reinterpret_cast<const uint4*>(m.w1b + r * 24 + kc * 4);
  }
  for (int e = t; e < 64 * 10; e += TC_THREADS) {
    const int r = e / 10, kc = e % 10;
    *reinterpret_cast<uint4*>(s.w2 + cm_off(r, kc, SBO_K80)) = *reinterpret_cast<const uint4*>(m.w2b + r * 40 + kc * 4);
  }
  for (int e = t; e < 16 * 10; e += TC_THREADS) {
    const int r = e / 10, kc = e % 10;
    *reinterpret_cast<uint4*>(s.w3 + cm_off(r, kc, SBO_K80)) = *reinterpret_cast<const uint4*>(m.w3b + r * 40 + kc * 4);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&s.tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int q = 0; q < TC_STREAMS; q++) mbar_init_count(&s.accready[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  proxy_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem;
  const int64_t ntiles = (n + TC_TILE - 1) / TC_TILE;
  auto tile_of = [&](int64_t k) { return static_cast<int64_t>(blockIdx.x) + k * gridDim.x; };
  const int st = warp >> 2;                     // this warp's stream
  const int trow = 32 * (warp & 3) + (t & 31);  // the tile row of this thread's lane
  const uint32_t lanes = static_cast<uint32_t>(32 * (warp & 3)) << 16;
  const uint32_t r0 = tmem + lanes + 128 * st, r1 = r0 + 64;  // this lane in the stream's two regions
  const uint32_t m0 = tmem + 128 * st, m1 = m0 + 64;          // the regions as MMA operands (lane 0)
  const uint64_t bd1 = umma_sdesc(tc_saddr(s.w1), 128, SBO_K48), bd2 = umma_sdesc(tc_saddr(s.w2), 128, SBO_K80),
                 bd3 = umma_sdesc(tc_saddr(s.w3), 128, SBO_K80);
  constexpr uint32_t ID64 = umma_idesc_bf16(TC_TILE, 64), ID16 = umma_idesc_bf16(TC_TILE, 16);
  uint64_t* bar = &s.accready[st];
  uint32_t aph = 0;
  bool pending = false;  // an MMA group of this stream not yet waited for (issuing thread's view)
  // operands of layer l in tensor memory (stores waited for) in every thread
  // of the stream -> its MMAs, issued by one thread; false if some thread of
  // the stream saw a wait run out
  auto issue = [&](int l, bool ok) -> bool {
    tc_fence_before();
    uint32_t any_bad;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.eq.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(any_bad)
        : "r"(ok ? 1u : 0u), "r"(1 + st), "r"(TC_TILE)
        : "memory");
    if (any_bad) return false;
    if ((warp & 3) == 0) {
      if (elect_one()) {
        tc_fence_after();
        // K slice k: A 8 columns further, B 256 bytes further (16 in the
        // descriptor's address field)
        if (l == 0) {
#pragma unroll
          for (int k = 0; k < 3; k++) umma_bf16_ts(m0, m1 + 8 * k, bd1 + 16 * k, ID64, k);
        } else if (l == 1) {
#pragma unroll
          for (int k = 0; k < 5; k++) umma_bf16_ts(m1, m0 + 8 * k, bd2 + 16 * k, ID64, k);
        } else {
#pragma unroll
          for (int k = 0; k < 5; k++) umma_bf16_ts(m0, m1 + 8 * k, bd3 + 16 * k, ID16, k);
        }
        umma_commit(bar);
      }
      __syncwarp();
    }
    pending = true;
    return true;
  };
  auto wait_acc = [&]() -> bool {
    const bool got = mbar_wait_bounded_tc(bar, aph, err);
    if (got) {
      aph ^= 1u;
      pending = false;
    }
    tc_fence_after();
    return got;
  };
  // the 40 inputs (20 words) of this row of tile k, zeros past n
  auto load_row = [&](int64_t k, uint4 xv[5]) {
    const int64_t r = tile_of(k) * TC_TILE + trow;
#pragma unroll
    for (int c = 0; c < 5; c++) xv[c] = make_uint4(0u, 0u, 0u, 0u);
    if (r < n) {
      const uint4* src = reinterpret_cast<const uint4*>(X + r * 24);
#pragma unroll
      for (int c = 0; c < 5; c++) xv[c] = src[c];
    }
  };
  uint4 xv[5];
  load_row(st, xv);
  bool ok = true;
  for (int64_t k = st; tile_of(k) < ntiles; k += TC_STREAMS) {
    {  // X (K = 48: 20 words of inputs, the bias column pair, zeros) into region 1
      uint32_t w[24];
#pragma unroll
      for (int c = 0; c < 5; c++) {
        w[4 * c] = xv[c].x;
        w[4 * c + 1] = xv[c].y;
        w[4 * c + 2] = xv[c].z;
        w[4 * c + 3] = xv[c].w;
      }
      w[20] = pack_bf16(1.f, 1.f);
      w[21] = w[22] = w[23] = 0u;
      tmem_st16(r1, w);
      tmem_st8(r1 + 16, w + 16);
      tmem_st_wait();
    }
    load_row(k + TC_STREAMS, xv);
    if (!issue(0, ok)) break;
    ok = wait_acc();
    tc_hidden_row(r0);
    if (!issue(1, ok)) break;
    ok = wait_acc();
    tc_hidden_row(r1);
    if (!issue(2, ok)) break;
    ok = wait_acc();
    float v[32];
    tmem_ld32(r0, v);
    const int64_t row = tile_of(k) * TC_TILE + trow;
    if (ok && row < n) {
      float4* dst = reinterpret_cast<float4*>(Y + row * 8);
      dst[0] = make_float4(v[0], v[1], v[2], v[3]);
      dst[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
  // after a timed-out wait this stream's MMAs may still run: wait once more
  if (pending && !ok) mbar_wait_bounded_tc(bar, aph, err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
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
// A bias as the BF16 pair (hi, lo): hi = BF16(b), lo = BF16(b - hi); with
// 1.0 in both matching input columns the product adds b to 2^-16 relative.
__device__ __forceinline__ uint32_t bias_pair(float b) {
  const float hi = __bfloat162float(__float2bfloat16_rn(b));
  return pack_bf16(hi, b - hi);
}
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
  // folded-bias layouts of the inference kernel
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * 40; e += gridDim.x * blockDim.x) {
    const int r = e / 40, c = e % 40;
    if (c < 24) {
      uint32_t w1 = 0u;
      if (c < 20) w1 = pack_bf16(W1[r * 40 + 2 * c], W1[r * 40 + 2 * c + 1]);
      else if (c == 20) w1 = bias_pair(B1[r]);
      m.w1b[r * 24 + c] = w1;
    }
    uint32_t w = 0u;
    if (c < 32) w = pack_bf16(0.5f * W2[r * 64 + 2 * c], 0.5f * W2[r * 64 + 2 * c + 1]);
    else if (c == 32) w = bias_pair(B2[r]);
    m.w2b[r * 40 + c] = w;
    if (r < 16) {
      uint32_t w3 = 0u;
      if (r < 8 && c < 32) w3 = pack_bf16(0.5f * W3[r * 64 + 2 * c], 0.5f * W3[r * 64 + 2 * c + 1]);
      else if (r < 8 && c == 32) w3 = bias_pair(B3[r]);
      m.w3b[r * 40 + c] = w3;
    }
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
// Training on tcgen05.  One CTA of 128 threads per SM, persistent over
// 128-sample tiles; thread t owns sample t of the tile (tensor-memory lane t).
// Every product is a tcgen05.mma with the FP32 accumulator in tensor memory:
//   forward   Z1 = X W1^T, Z2 = H1 W2^T, Y = H2 W3^T          (M = samples)
//   backward  dH2 = dY W3, dH1 = dZ2 W2                         (M = samples)
//   weights   dW1|db1 = dZ1^T [X | 1], dW2|db2 = dZ2^T [H1 | 1],
//             dW3^T|db3 = [H2 | 1]^T dY                         (K = samples)
// For the weight products the threads store the per-sample factors
// transposed (a column per sample), which makes them K-major operands with
// the samples along K; a row of ones appended to one factor gives the bias
// gradient in an extra accumulator row or column.  The weight accumulators
// live in tensor memory across all of a CTA's tiles (a fixed order of
// accumulation), each CTA writes its partial gradient, and a second kernel
// sums the partials in CTA order: the gradient is the same bit for bit from
// run to run.

constexpr int TT = 128;              // samples per tile
constexpr uint32_t SBO_KT = 16 * TT; // K = 128 samples: 2048 bytes per 8-row group
constexpr uint32_t SBO_K16 = 256;    // K = 16
struct TrainTc {
  alignas(128) uint8_t a1[TT * 128];   // X (K = 48), then H1 (K = 64), then dZ2 (K = 64): A operands, M = samples
  alignas(128) uint8_t a2[TT * 128];   // H2 (K = 64), then dY (K = 16)
  alignas(128) uint8_t xt[48 * 256];   // [X | 1]^T: rows 0-39 features, 40 ones, 41-47 zero; K = samples
  alignas(128) uint8_t h1t[80 * 256];  // [H1 | 1]^T: rows 0-63, 64 ones, 65-79 zero
  alignas(128) uint8_t h2t[128 * 256]; // [H2 | 1]^T as the A of dW3^T: rows 0-63, 64 ones, 65-127 zero
  alignas(128) uint8_t dyt[16 * 256];  // dY^T: rows 0-7, 8-15 zero
  alignas(128) uint8_t dz2t[128 * 256];// dZ2^T: rows 0-63, 64-127 zero
  alignas(128) uint8_t dz1t[128 * 256];// dZ1^T: rows 0-63, 64-127 zero
  alignas(128) uint8_t w1[64 * 96];    // B of Z1: N = 64, K = 48
  alignas(128) uint8_t w2[64 * 128];   // B of Z2: N = 64, K = 64
  alignas(128) uint8_t w3[16 * 128];   // B of Y: N = 16 (8 zero rows), K = 64
  alignas(128) uint8_t w3t[64 * 32];   // B of dH2: N = 64, K = 16 (W3^T, 8 zero columns)
  alignas(128) uint8_t w2t[64 * 128];  // B of dH1: N = 64, K = 64 (W2^T)
  float b1[64], b2[64], b3[8];
  double wloss[4];
  uint64_t bar;
  uint32_t tmem;
};
// tensor-memory columns of the accumulators
constexpr uint32_t TM_Z1 = 0, TM_Z2 = 64, TM_Y = 128, TM_DH2 = 160, TM_DH1 = 224, TM_D1 = 288, TM_D2 = 352,
                   TM_D3 = 448, TM_COLS = 512;

// one BF16 (bits) of a K = 128-sample transposed operand: row r, sample k
__device__ __forceinline__ void st_t(uint8_t* buf, int r, int k, uint16_t v) {
  *reinterpret_cast<uint16_t*>(buf + cm_off(r, k >> 3, SBO_KT) + (k & 7) * 2) = v;
}
__device__ __forceinline__ uint16_t bf16_bits(float v) {
  return static_cast<uint16_t>(pack_bf16(v, 0.f) & 0xffffu);
}

// The MMAs of one group (issued by thread 0, committed, waited for by all
// threads, bounded): false when the wait ran out.
template <class F>
__device__ __forceinline__ bool tt_group(TrainTc& s, int t, uint32_t& phase, int32_t* err, F issue) {
  proxy_fence_smem();
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
    issue();
    umma_commit(&s.bar);
  }
  const bool got = mbar_wait_bounded_tc(&s.bar, phase, err);
  if (__syncthreads_or(!got)) return false;
  phase ^= 1u;
  tc_fence_after();
  return true;
}

__global__ void __launch_bounds__(TT, 1) k_mlp_train_tc(const float* __restrict__ X, const float* __restrict__ T,
                                                       const int64_t* __restrict__ idx, int64_t nrows,
                                                       int64_t n, double inv_count, MlpDev m,
                                                       float* __restrict__ partial, double* __restrict__ partial_loss,
                                                       int32_t* err) {
  extern __shared__ __align__(128) unsigned char tt_smem_raw[];
  TrainTc& s = *reinterpret_cast<TrainTc*>((reinterpret_cast<uintptr_t>(tt_smem_raw) + 127) & ~uintptr_t(127));
  const int t = threadIdx.x, warp = t >> 5;
  // weights in the canonical layouts; the constant rows and columns of the
  // transposed operands (ones, zeros)
  for (int e = t; e < 64 * 6; e += TT) {
    const int r = e / 6, kc = e % 6;
    *reinterpret_cast<uint4*>(s.w1 + cm_off(r, kc, SBO_K48)) = *reinterpret_cast<const uint4*>(m.w1 + r * 24 + kc * 4);
  }
  for (int e = t; e < 64 * 8; e += TT) {
    const int r = e / 8, kc = e % 8;
    *reinterpret_cast<uint4*>(s.w2 + cm_off(r, kc, SBO_K64)) = *reinterpret_cast<const uint4*>(m.w2 + r * 32 + kc * 4);
    *reinterpret_cast<uint4*>(s.w2t + cm_off(r, kc, SBO_K64)) = *reinterpret_cast<const uint4*>(m.w2t + r * 32 + kc * 4);
  }
  for (int e = t; e < 16 * 8; e += TT) {
    const int r = e / 8, kc = e % 8;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(s.w3 + cm_off(r, kc, SBO_K64)) =
        r < 8 ? *reinterpret_cast<const uint4*>(m.w3 + r * 32 + kc * 4) : z;
  }
  for (int e = t; e < 64 * 2; e += TT) {
    const int r = e / 2, kc = e % 2;
    *reinterpret_cast<uint4*>(s.w3t + cm_off(r, kc, SBO_K16)) = *reinterpret_cast<const uint4*>(m.w3t + r * 8 + kc * 4);
  }
  if (t < 64) {
    s.b1[t] = m.b1[t];
    s.b2[t] = m.b2[t];
  }
  if (t < 8) s.b3[t] = m.b3[t];
  {
    const uint16_t one = bf16_bits(1.f);
    for (int r = 40; r < 48; r++) st_t(s.xt, r, t, r == 40 ? one : 0);
    for (int r = 64; r < 80; r++) st_t(s.h1t, r, t, r == 64 ? one : 0);
    for (int r = 64; r < 128; r++) {
      st_t(s.h2t, r, t, r == 64 ? one : 0);
      st_t(s.dz2t, r, t, 0);
      st_t(s.dz1t, r, t, 0);
    }
    for (int r = 8; r < 16; r++) st_t(s.dyt, r, t, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&s.tmem)),
                 "r"(TM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) mbar_init_tc(&s.bar);
  proxy_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = s.tmem;
  const uint32_t tl = tm + (static_cast<uint32_t>(32 * warp) << 16);  // this warp's lanes
  const uint32_t a1s = tc_saddr(s.a1), a2s = tc_saddr(s.a2), xts = tc_saddr(s.xt), h1ts = tc_saddr(s.h1t);
  const uint32_t h2ts = tc_saddr(s.h2t), dyts = tc_saddr(s.dyt), dz2ts = tc_saddr(s.dz2t), dz1ts = tc_saddr(s.dz1t);
  const uint32_t w1s = tc_saddr(s.w1), w2s = tc_saddr(s.w2), w3s = tc_saddr(s.w3), w3ts = tc_saddr(s.w3t),
                 w2ts = tc_saddr(s.w2t);
  const float scale = static_cast<float>(2.0 * inv_count);
  uint32_t phase = 0;
  bool failed = false, any = false;
  double lsum = 0.0;
  const int64_t ntiles = (n + TT - 1) / TT;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t rt = tile * TT + t;
    int64_t r = rt < n && idx ? idx[rt] : rt;  // the sample's row of X and T
    if (idx && rt < n && (r < 0 || r >= nrows)) {  // an index outside X: no contribution, flagged
      atomicOr(err, ERR_BOUNDS);
      r = -1;
    }
    const bool valid = rt < n && r >= 0;
    // X row t (BF16) as the A of Z1, and its column of [X | 1]^T
    {
      float x[40];
#pragma unroll
      for (int i = 0; i < 40; i++) x[i] = valid ? X[r * 40 + i] : 0.f;
#pragma unroll
      for (int kc = 0; kc < 6; kc++) {
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (kc < 5)
          o = make_uint4(pack_bf16(x[8 * kc], x[8 * kc + 1]), pack_bf16(x[8 * kc + 2], x[8 * kc + 3]),
                         pack_bf16(x[8 * kc + 4], x[8 * kc + 5]), pack_bf16(x[8 * kc + 6], x[8 * kc + 7]));
        *reinterpret_cast<uint4*>(s.a1 + cm_off(t, kc, SBO_K48)) = o;
      }
#pragma unroll
      for (int i = 0; i < 40; i++) st_t(s.xt, i, t, bf16_bits(x[i]));
    }
    const uint32_t I64 = umma_idesc_bf16(TT, 64), I16 = umma_idesc_bf16(TT, 16), I48 = umma_idesc_bf16(TT, 48),
                   I80 = umma_idesc_bf16(TT, 80);
    // Z1 = X W1^T
    if (!tt_group(s, t, phase, err, [&]() {
          for (int k = 0; k < 3; k++)
            umma_bf16(tm + TM_Z1, umma_sdesc(a1s + 256 * k, 128, SBO_K48), umma_sdesc(w1s + 256 * k, 128, SBO_K48),
                      I64, k > 0);
        })) { failed = true; break; }
    // H1 = GELU(Z1 + b1): the A of Z2 (into a1) and a column of [H1 | 1]^T
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float v[16];
      tmem_ld16(tl + TM_Z1 + 16 * q, v);
#pragma unroll
      for (int c = 0; c < 2; c++) {
        const float* b = s.b1 + 16 * q + 8 * c;
        const float* z = v + 8 * c;
        uint4 o;
        o.x = gelu2_pack(z[0] + b[0], z[1] + b[1]);
        o.y = gelu2_pack(z[2] + b[2], z[3] + b[3]);
        o.z = gelu2_pack(z[4] + b[4], z[5] + b[5]);
        o.w = gelu2_pack(z[6] + b[6], z[7] + b[7]);
        *reinterpret_cast<uint4*>(s.a1 + cm_off(t, 2 * q + c, SBO_K64)) = o;
        const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
          st_t(s.h1t, 16 * q + 8 * c + 2 * j, t, static_cast<uint16_t>(w[j] & 0xffffu));
          st_t(s.h1t, 16 * q + 8 * c + 2 * j + 1, t, static_cast<uint16_t>(w[j] >> 16));
        }
      }
    }
    // Z2 = H1 W2^T
    if (!tt_group(s, t, phase, err, [&]() {
          for (int k = 0; k < 4; k++)
            umma_bf16(tm + TM_Z2, umma_sdesc(a1s + 256 * k, 128, SBO_K64), umma_sdesc(w2s + 256 * k, 128, SBO_K64),
                      I64, k > 0);
        })) { failed = true; break; }
    // H2 = GELU(Z2 + b2): the A of Y (into a2) and a column of [H2 | 1]^T
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float v[16];
      tmem_ld16(tl + TM_Z2 + 16 * q, v);
#pragma unroll
      for (int c = 0; c < 2; c++) {
        const float* b = s.b2 + 16 * q + 8 * c;
        const float* z = v + 8 * c;
        uint4 o;
        o.x = gelu2_pack(z[0] + b[0], z[1] + b[1]);
        o.y = gelu2_pack(z[2] + b[2], z[3] + b[3]);
        o.z = gelu2_pack(z[4] + b[4], z[5] + b[5]);
        o.w = gelu2_pack(z[6] + b[6], z[7] + b[7]);
        *reinterpret_cast<uint4*>(s.a2 + cm_off(t, 2 * q + c, SBO_K64)) = o;
        const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
          st_t(s.h2t, 16 * q + 8 * c + 2 * j, t, static_cast<uint16_t>(w[j] & 0xffffu));
          st_t(s.h2t, 16 * q + 8 * c + 2 * j + 1, t, static_cast<uint16_t>(w[j] >> 16));
        }
      }
    }
    // Y = H2 W3^T (N = 16: the 8 outputs and 8 zero columns)
    if (!tt_group(s, t, phase, err, [&]() {
          for (int k = 0; k < 4; k++)
            umma_bf16(tm + TM_Y, umma_sdesc(a2s + 256 * k, 128, SBO_K64), umma_sdesc(w3s + 256 * k, 128, SBO_K64),
                      I16, k > 0);
        })) { failed = true; break; }
    // dL/dY = 2 (y - t) / (8 n): the A of dH2 (into a2, K = 16) and dY^T
    {
      float v[16];
      tmem_ld16(tl + TM_Y, v);
      float dy[8];
#pragma unroll
      for (int o = 0; o < 8; o++) {
        const float e = valid ? (v[o] + s.b3[o]) - T[r * 8 + o] : 0.f;
        lsum += static_cast<double>(e) * e;
        dy[o] = scale * e;
      }
      *reinterpret_cast<uint4*>(s.a2 + cm_off(t, 0, SBO_K16)) =
          make_uint4(pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), pack_bf16(dy[4], dy[5]), pack_bf16(dy[6], dy[7]));
      *reinterpret_cast<uint4*>(s.a2 + cm_off(t, 1, SBO_K16)) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int o = 0; o < 8; o++) st_t(s.dyt, o, t, bf16_bits(dy[o]));
    }
    // dH2 = dY W3
    if (!tt_group(s, t, phase, err, [&]() {
          umma_bf16(tm + TM_DH2, umma_sdesc(a2s, 128, SBO_K16), umma_sdesc(w3ts, 128, SBO_K16), I64, 0);
        })) { failed = true; break; }
    // dZ2 = dH2 GELU'(Z2 + b2): the A of dH1 (into a1) and a column of dZ2^T
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float dh[16], z[16];
      tmem_ld16(tl + TM_DH2 + 16 * q, dh);
      tmem_ld16(tl + TM_Z2 + 16 * q, z);
#pragma unroll
      for (int c = 0; c < 2; c++) {
        float g[8];
#pragma unroll
        for (int j = 0; j < 8; j++) g[j] = dh[8 * c + j] * gelu_grad_f(z[8 * c + j] + s.b2[16 * q + 8 * c + j]);
        *reinterpret_cast<uint4*>(s.a1 + cm_off(t, 2 * q + c, SBO_K64)) =
            make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]), pack_bf16(g[6], g[7]));
#pragma unroll
        for (int j = 0; j < 8; j++) st_t(s.dz2t, 16 * q + 8 * c + j, t, bf16_bits(g[j]));
      }
    }
    // dH1 = dZ2 W2
    if (!tt_group(s, t, phase, err, [&]() {
          for (int k = 0; k < 4; k++)
            umma_bf16(tm + TM_DH1, umma_sdesc(a1s + 256 * k, 128, SBO_K64), umma_sdesc(w2ts + 256 * k, 128, SBO_K64),
                      I64, k > 0);
        })) { failed = true; break; }
    // dZ1 = dH1 GELU'(Z1 + b1): a column of dZ1^T
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float dh[16], z[16];
      tmem_ld16(tl + TM_DH1 + 16 * q, dh);
      tmem_ld16(tl + TM_Z1 + 16 * q, z);
#pragma unroll
      for (int j = 0; j < 16; j++)
        st_t(s.dz1t, 16 * q + j, t, bf16_bits(dh[j] * gelu_grad_f(z[j] + s.b1[16 * q + j])));
    }
    // the weight gradients of this tile, added to the CTA's accumulators:
    // [dW1 | db1] += dZ1^T [X | 1], [dW2 | db2] += dZ2^T [H1 | 1],
    // [dW3^T ; db3] += [H2 | 1]^T dY (K = the tile's 128 samples)
    const uint32_t acc0 = any ? 1u : 0u;
    if (!tt_group(s, t, phase, err, [&]() {
          for (int k = 0; k < 8; k++) {
            const uint32_t acc = k > 0 ? 1u : acc0;
            umma_bf16(tm + TM_D1, umma_sdesc(dz1ts + 256 * k, 128, SBO_KT), umma_sdesc(xts + 256 * k, 128, SBO_KT),
                      I48, acc);
            umma_bf16(tm + TM_D2, umma_sdesc(dz2ts + 256 * k, 128, SBO_KT), umma_sdesc(h1ts + 256 * k, 128, SBO_KT),
                      I80, acc);
            umma_bf16(tm + TM_D3, umma_sdesc(h2ts + 256 * k, 128, SBO_KT), umma_sdesc(dyts + 256 * k, 128, SBO_KT),
                      I16, acc);
          }
        })) { failed = true; break; }
    any = true;
  }
  // this CTA's partial gradient in the parameter order W1, b1, W2, b2, W3, b3
  float* pg = partial + static_cast<int64_t>(blockIdx.x) * MLP_NPARAM;
  if (!failed) {
    float d1[48], d2[80], d3[16];
#pragma unroll
    for (int q = 0; q < 3; q++) tmem_ld16(tl + TM_D1 + 16 * q, d1 + 16 * q);
#pragma unroll
    for (int q = 0; q < 5; q++) tmem_ld16(tl + TM_D2 + 16 * q, d2 + 16 * q);
    tmem_ld16(tl + TM_D3, d3);
    if (!any) {
#pragma unroll
      for (int i = 0; i < 48; i++) d1[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 80; i++) d2[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 16; i++) d3[i] = 0.f;
    }
    if (t < 64) {
#pragma unroll
      for (int i = 0; i < 40; i++) pg[t * 40 + i] = d1[i];
      pg[2560 + t] = d1[40];
#pragma unroll
      for (int i = 0; i < 64; i++) pg[2624 + t * 64 + i] = d2[i];
      pg[6720 + t] = d2[64];
#pragma unroll
      for (int o = 0; o < 8; o++) pg[6784 + o * 64 + t] = d3[o];
    } else if (t == 64) {
#pragma unroll
      for (int o = 0; o < 8; o++) pg[7296 + o] = d3[o];
    }
  }
  // the CTA's loss: each thread's samples in tile order, then the threads in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) s.wloss[warp] = lsum;
  // an MMA may still run after a timed-out wait: wait for it once more
  if (failed && t == 0) mbar_wait_bounded_tc(&s.bar, phase, err);
  tc_fence_before();
  __syncthreads();
  if (t == 0) partial_loss[blockIdx.x] = ((s.wloss[0] + s.wloss[1]) + s.wloss[2]) + s.wloss[3];
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TM_COLS) : "memory");
  }
}

// grad[e] = sum over the CTAs c = 0, 1, ... of partial[c][e] (a fixed
// order); *loss = the same sum of the partial losses.
__global__ void k_mlp_grad_reduce(const float* __restrict__ partial, const double* __restrict__ partial_loss,
                                  int nparts, float* __restrict__ grad, double* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < MLP_NPARAM) {
    float acc = 0.f;
    for (int c = 0; c < nparts; c++) acc += partial[static_cast<int64_t>(c) * MLP_NPARAM + e];
    grad[e] = acc;
  }
  if (e == 0) {
    double l = 0.0;
    for (int c = 0; c < nparts; c++) l += partial_loss[c];
    *loss = l;
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers.


constexpr size_t kTrainTcSmem = sizeof(TrainTc) + 128;
constexpr size_t kInferSmem = sizeof(TcSmem) + 128;
cudaError_t mlp_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kTrainTcSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kInferSmem));
  return e;
}
cudaError_t launch_mlp_pack(const float* P, const MlpDev& m, cudaStream_t st) {
  k_mlp_pack<<<8, 256, 0, st>>>(P, m);
  return cudaGetLastError();
}
// X: n rows of 24 words (16-byte aligned), Y: n rows of 8 floats (16-byte
// aligned); one CTA per SM (all 512 tensor-memory columns, 19 KB of shared
// memory).
cudaError_t launch_mlp_infer(const uint32_t* X, float* Y, int64_t n, const MlpDev& m, int nsm, int32_t* err,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) return cudaErrorInvalidValue;
  const int64_t tiles = (n + TC_TILE - 1) / TC_TILE;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(nsm)));
  k_mlp_infer<<<grid, TC_THREADS, kInferSmem, st>>>(X, Y, n, m, err);
  return cudaGetLastError();
}
// The loss sum and the gradient on the tensor cores: one CTA per SM (at most
// one per tile), each writing a partial gradient and loss, then their sum in
// CTA order (the result is the same bit for bit from run to run).  partial:
// nsm x MLP_NPARAM floats, partial_loss: nsm doubles.
// idx (nullable, device): sample i is row idx[i] of X and T (nrows rows);
// without it sample i is row i.
cudaError_t launch_mlp_train(const float* X, const float* T, const int64_t* idx, int64_t nrows, int64_t n,
                             const MlpDev& m, float* grad, double* loss, float* partial, double* partial_loss,
                             int32_t* err, int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + TT - 1) / TT;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(nsm)));
  k_mlp_train_tc<<<grid, TT, kTrainTcSmem, st>>>(X, T, idx, nrows, n, 1.0 / (8.0 * static_cast<double>(n)), m,
                                                  partial, partial_loss, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mlp_grad_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(partial, partial_loss, grid, grad, loss);
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
  const size_t words = 64 * 24 + 64 * 32 + 8 * 32 + 64 * 32 + 64 * 8 + 64 * 24 + 64 * 40 + 16 * 40;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, words * 4 + (64 + 64 + 8) * 4);
  if (e != cudaSuccess) return e;
  uint32_t* u = static_cast<uint32_t*>(p);
  w->w1 = u;
  w->w2 = w->w1 + 64 * 24;
  w->w3 = w->w2 + 64 * 32;
  w->w2t = w->w3 + 8 * 32;
  w->w3t = w->w2t + 64 * 32;
  w->w1b = w->w3t + 64 * 8;
  w->w2b = w->w1b + 64 * 24;
  w->w3b = w->w2b + 64 * 40;
  float* f = reinterpret_cast<float*>(w->w3b + 16 * 40);
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
  int32_t* errw = nullptr;  // device error bits of the inference and training kernels (ERR_TIMEOUT)
  float* partial = nullptr;          // per-CTA partial gradients of a training pass [nsm][NPARAM]
  double* partial_loss = nullptr;    // and losses [nsm]
  double* step_loss = nullptr;       // per-step losses of an epoch [step_cap]
  int64_t step_cap = 0;
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
  if (launch_mlp_train(m->X, m->T, nullptr, n, n, m->w, m->G, m->loss, m->partial, m->partial_loss, m->errw,
                       m->nsm, m->stream) != cudaSuccess)
    return BATS_ERR_CUDA;
  return BATS_OK;
}

// The error bits of the kernels since the last check (cleared): a bounded
// tensor-core wait that ran out is BATS_ERR_TIMEOUT, a sample index outside
// the training set BATS_ERR_INVALID_ARG.
int mlp_check_err(bats_mlp_t* m) {
  int32_t eb = 0;
  if (cudaMemcpyAsync(&eb, m->errw, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return BATS_ERR_CUDA;
  if (eb) {
    cudaMemsetAsync(m->errw, 0, sizeof(int32_t), m->stream);
    return (eb & ERR_TIMEOUT) ? BATS_ERR_TIMEOUT : BATS_ERR_INVALID_ARG;
  }
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
  if (e == cudaSuccess) e = cudaMalloc(&m->partial, sizeof(float) * MLP_NPARAM * m->nsm);
  if (e == cudaSuccess) e = cudaMalloc(&m->partial_loss, sizeof(double) * m->nsm);
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
  cudaFree(m->partial);
  cudaFree(m->partial_loss);
  cudaFree(m->step_loss);
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
__global__ void k_debug_gelu(const float* x, int n, int variant, float* y) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float x1 = i + 1 < n ? x[i + 1] : 0.f;
  const uint32_t r = variant ? gelu2x_pack(x[i], x1) : gelu2_pack(x[i], x1);
  const float sc = variant ? 0.5f : 1.f;
  y[i] = sc * bf16_lo(r);
  if (i + 1 < n) y[i + 1] = sc * bf16_hi(r);
}

int bats_debug_gelu(const float* x, int n, int variant, float* y) {
  if (!x || !y || n <= 0 || variant < 0 || variant > 1) return BATS_ERR_INVALID_ARG;
  float *xd = nullptr, *yd = nullptr;
  cudaError_t e = cudaMalloc(&xd, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&yd, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(xd, x, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_debug_gelu<<<(n / 2 + 256) / 256, 256>>>(xd, n, variant, yd);
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
    return (eb & ERR_TIMEOUT) ? BATS_ERR_TIMEOUT : BATS_ERR_INVALID_ARG;
  }
  return BATS_OK;
}

int bats_mlp_forward_bf16(bats_mlp_t* m, const uint32_t* Xb, int64_t n, float* Y) {
  if (!m || !Xb || !Y || n <= 0) return BATS_ERR_INVALID_ARG;
  if (!dev_ptr(Xb) || !dev_ptr(Y)) return BATS_ERR_INVALID_ARG;
  return launch_mlp_infer(Xb, Y, n, m->w, m->nsm, m->errw, m->stream) == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

int bats_mlp_sync(bats_mlp_t* m) {
  if (!m) return BATS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return BATS_ERR_CUDA;
  return mlp_check_err(m);
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
  if ((rc = mlp_check_err(m))) return rc;
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
    if ((rc = mlp_check_err(m))) return rc;
    *loss = ls / (8.0 * static_cast<double>(n));
  }
  return BATS_OK;
}

int bats_mlp_train_epoch(bats_mlp_t* m, const float* X, const float* T, int64_t n, const int64_t* perm,
                         int64_t n_perm, int64_t batch, float lr, double* mean_loss) {
  if (!m || !X || !T || !perm || n <= 0 || batch < 1 || n_perm < batch || !(lr >= 0.f)) return BATS_ERR_INVALID_ARG;
  if (!dev_ptr(X) || !dev_ptr(T) || !dev_ptr(perm)) return BATS_ERR_INVALID_ARG;
  const int64_t steps = n_perm / batch;
  if (steps > m->step_cap) {
    cudaFree(m->step_loss);
    m->step_loss = nullptr;
    m->step_cap = 0;
    if (cudaMalloc(&m->step_loss, sizeof(double) * steps) != cudaSuccess) {
      cudaGetLastError();
      return BATS_ERR_OUT_OF_MEMORY;
    }
    m->step_cap = steps;
  }
  for (int64_t s = 0; s < steps; s++) {
    if (launch_mlp_train(X, T, perm + s * batch, n, batch, m->w, m->G, m->step_loss + s, m->partial,
                         m->partial_loss, m->errw, m->nsm, m->stream) != cudaSuccess)
      return BATS_ERR_CUDA;
    m->step++;
    if (launch_mlp_adam(m->P, m->G, m->M1, m->M2, lr, m->step, m->stream) != cudaSuccess ||
        launch_mlp_pack(m->P, m->w, m->stream) != cudaSuccess)
      return BATS_ERR_CUDA;
  }
  std::vector<double> ls(static_cast<size_t>(steps));
  if (cudaMemcpyAsync(ls.data(), m->step_loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, m->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return BATS_ERR_CUDA;
  int rc = mlp_check_err(m);
  if (rc) return rc;
  if (mean_loss) {
    double acc = 0.0;
    for (double v : ls) acc += v / (8.0 * static_cast<double>(batch));
    *mean_loss = acc / static_cast<double>(steps);
  }
  return BATS_OK;
}

}  // extern "C"
