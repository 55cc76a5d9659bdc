// bats_stage.cu -- sm_103a kernels of one explicit stage of the ideal-MHD
// finite-volume update on a 2:1 block-adaptive grid (arXiv 2501.06717,
// Algorithms 1-2; Eqs. 1-5), fused: ghost fill + primitive recovery + limited
// reconstruction + Rusanov flux + Powell/B0 sources + conservative update (+
// CFL bound of the new state), one 8^3 block per CTA iteration.
//
// Shared-memory tile per block: [8 variables][1280 cells] = the 512 interior
// cells (staged by 1-D TMA bulk copies, one per variable, completing on an
// mbarrier) followed by the six 2-layer face slabs (768 ghost cells) that the
// dimension-by-dimension stencil reads; edge and corner ghosts are never read
// by the stencil and are not filled.
#include <cstdint>
#include <cuda_runtime.h>
#include <algorithm>
#include <type_traits>

#include "bats_internal.h"

namespace batsk {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + 1-D bulk copy (TMA), bounded waits.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for an mbarrier phase; gives up after ~1 s of wall time, records
// ERR_TIMEOUT and returns false (the caller then waits once more, bounded,
// so that no bulk copy is left in flight into this CTA's shared memory).
__device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > 1000000000ull) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
}

// ---------------------------------------------------------------------------
// Conversions without the FP64 pipe.  On GB300 the F2F instructions share the
// FP64 unit (about 1/64 of the FP32 rate); these use integer ops only.

// Float -> double, exact for normal floats and zero; float denormals -> 0.
__device__ __forceinline__ double f2d_int(float f) {
  uint32_t u = __float_as_uint(f);
  uint32_t s = u & 0x80000000u, a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + (896u << 20);
  uint32_t lo = a << 29;
  bool tiny = a < 0x00800000u;
  hi = tiny ? 0u : hi;
  lo = tiny ? 0u : lo;
  hi = (a >= 0x7f800000u) ? (0x7ff00000u | ((a >> 3) & 0x000fffffu)) : hi;
  return __hiloint2double(static_cast<int>(hi | s), static_cast<int>(lo));
}
// Double -> float, rounding half away from zero on the magnitude; values
// below the float normal range -> signed 0, above it -> inf.
__device__ __forceinline__ float d2f_int(double d) {
  uint32_t hi = static_cast<uint32_t>(__double2hiint(d)), lo = static_cast<uint32_t>(__double2loint(d));
  uint32_t s = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  uint32_t f = __funnelshift_l(lo, ahi, 3) - (896u << 23);
  f += (lo >> 28) & 1u;
  f = (ahi < 0x38100000u) ? 0u : f;
  f = (ahi >= 0x47f00000u) ? 0x7f800000u : f;
  return __uint_as_float(f | s);
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// Precision-generic scalar ops.

template <class R> struct Ops;
template <> struct Ops<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
};
template <> struct Ops<float> {
  static __device__ __forceinline__ float sqrt_(float x) { return sqrt_approx(x); }
  static __device__ __forceinline__ float div_(float a, float b) { return a * rcp_approx(b); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
};

template <class R>
__device__ __forceinline__ R minmod_(R a, R b) {
  R r = R(0);
  r = (a > R(0) && b > R(0)) ? (a < b ? a : b) : r;
  r = (a < R(0) && b < R(0)) ? (a > b ? a : b) : r;
  return r;
}
// MC limiter (beta = 2): sign(a) min(2|a|, 2|b|, |a+b|/2), 0 when signs differ.
template <class R>
__device__ __forceinline__ R mc_(R a, R b) {
  R c = R(0.5) * (a + b);
  R r = R(0);
  if (a > R(0) && b > R(0)) {
    R m = R(2) * a < R(2) * b ? R(2) * a : R(2) * b;
    r = m < c ? m : c;
  } else if (a < R(0) && b < R(0)) {
    R m = R(2) * a > R(2) * b ? R(2) * a : R(2) * b;
    r = m > c ? m : c;
  }
  return r;
}
template <class R>
__device__ __forceinline__ R limit_(int kind, R a, R b) {
  return kind == 1 ? mc_(a, b) : minmod_(a, b);
}

// Background field B0 at point x (split field B = B0 + B1).
template <class R>
__device__ __forceinline__ void b0_at(const PhysDev& ph, const R x[3], R B0[3]) {
  const double* q = ph.b0p;
  if (ph.b0 == B0_UNIFORM) {
    B0[0] = R(q[0]); B0[1] = R(q[1]); B0[2] = R(q[2]);
  } else if (ph.b0 == B0_DIPOLE) {
    R r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    R r = Ops<R>::sqrt_(r2);
    R inv_r5 = Ops<R>::div_(R(1), r2 * r2 * r);
    R mr = R(q[0]) * x[0] + R(q[1]) * x[1] + R(q[2]) * x[2];
#pragma unroll
    for (int c = 0; c < 3; c++) B0[c] = (R(3) * mr * x[c] - R(q[c]) * r2) * inv_r5;
  } else if (ph.b0 == B0_LINEAR) {
#pragma unroll
    for (int c = 0; c < 3; c++)
      B0[c] = R(q[c]) + R(q[3 + 3 * c]) * x[0] + R(q[4 + 3 * c]) * x[1] + R(q[5 + 3 * c]) * x[2];
  } else {
    B0[0] = B0[1] = B0[2] = R(0);
  }
}

// Primitive recovery in FP64 (Eq. 5): u = m/rho, p = (gamma-1)(e1 - m.u/2 - B1.B1/2).
__device__ __forceinline__ void prim64(const double U[8], double gm1, double W[8]) {
  double rho = U[0];
  double ux = U[1] / rho, uy = U[2] / rho, uz = U[3] / rho;
  double ke = 0.5 * (U[1] * ux + U[2] * uy + U[3] * uz);
  double me = 0.5 * (U[4] * U[4] + U[5] * U[5] + U[6] * U[6]);
  W[0] = rho; W[1] = ux; W[2] = uy; W[3] = uz;
  W[4] = U[4]; W[5] = U[5]; W[6] = U[6];
  W[7] = gm1 * ((U[7] - ke) - me);
}

// Mixed form: FP32 primitives of an FP64 state, with the pressure recovered in
// FP64 (the cancellation e1 - rho u^2/2 - B1^2/2 is done in FP64; 1/rho by an
// FP32 estimate plus one FP64 Newton-Raphson step).
__device__ __forceinline__ void prim_mixed(const double U[8], float gm1f, float W[8], double* p64 = nullptr) {
  float rho32 = d2f_int(U[0]);
  float rinv32 = rcp_approx(rho32);
  double r0 = f2d_int(rinv32);
  double e = fma(-U[0], r0, 1.0);
  double rinv = fma(r0, e, r0);
  double mm = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  double bb = U[4] * U[4] + U[5] * U[5] + U[6] * U[6];
  double x = fma(-0.5, bb, U[7]);
  x = fma(-0.5 * mm, rinv, x);
  float rf = d2f_int(rinv);
  W[0] = rho32;
  W[1] = d2f_int(U[1]) * rf;
  W[2] = d2f_int(U[2]) * rf;
  W[3] = d2f_int(U[3]) * rf;
  W[4] = d2f_int(U[4]);
  W[5] = d2f_int(U[5]);
  W[6] = d2f_int(U[6]);
  W[7] = d2f_int(x) * gm1f;
  if (p64) *p64 = x;
}

template <class R>
__device__ __forceinline__ void cons_from_prim(const R W[8], R inv_gm1, R U[8]) {
  R rho = W[0];
  R usq = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  R bsq = W[4] * W[4] + W[5] * W[5] + W[6] * W[6];
  U[0] = rho;
  U[1] = rho * W[1];
  U[2] = rho * W[2];
  U[3] = rho * W[3];
  U[4] = W[4];
  U[5] = W[5];
  U[6] = W[6];
  U[7] = W[7] * inv_gm1 + R(0.5) * rho * usq + R(0.5) * bsq;
}

// Fast magnetosonic speed along the frame's normal (component 0) with total B.
template <class R>
__device__ __forceinline__ R fast_speed_n(R gamma, R rho, R p, R bx, R by, R bz) {
  R rinv = Ops<R>::div_(R(1), rho);
  R a2 = Ops<R>::div_(gamma * p, rho);
  R b2 = (bx * bx + by * by + bz * bz) * rinv;
  R bn2 = bx * bx * rinv;
  R s = a2 + b2;
  R disc = s * s - R(4) * a2 * bn2;
  disc = disc < R(0) ? R(0) : disc;
  return Ops<R>::sqrt_(R(0.5) * (s + Ops<R>::sqrt_(disc)));
}
__device__ __forceinline__ double fast_speed_exact(double gamma, double rho, double p, double bx, double by,
                                                   double bz) {
  // FP64 path: the same divisions as the oracle, (gamma p)/rho and B^2/rho.
  double a2 = gamma * p / rho;
  double b2 = (bx * bx + by * by + bz * bz) / rho;
  double bn2 = bx * bx / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn2;
  disc = disc < 0.0 ? 0.0 : disc;
  return sqrt(0.5 * (s + sqrt(disc)));
}

// Split-field physical flux along the frame normal (component 0 of the
// rotated vectors): F_rho = rho un, F_m = rho u un + pt n - (B1 Bn + B0 B1n),
// F_B1 = un B - Bn u (normal component 0), F_e1 = un (e1 + pt) - (u.B1) Bn,
// pt = p + B1^2/2 + B0.B1.  Also U(W), un and the fast speed.
template <class R>
__device__ __forceinline__ void phys_flux(const R W[8], const R B0[3], R gamma, R inv_gm1, R F[8], R U[8],
                                          R& un, R& cf) {
  R rho = W[0];
  R u0 = W[1], u1 = W[2], u2 = W[3];
  R b10 = W[4], b11 = W[5], b12 = W[6], p = W[7];
  R B_0 = B0[0] + b10, B_1 = B0[1] + b11, B_2 = B0[2] + b12;
  R b1sq = b10 * b10 + b11 * b11 + b12 * b12;
  R b0b1 = B0[0] * b10 + B0[1] * b11 + B0[2] * b12;
  R usq = u0 * u0 + u1 * u1 + u2 * u2;
  R pt = p + R(0.5) * b1sq + b0b1;
  R e1 = p * inv_gm1 + R(0.5) * rho * usq + R(0.5) * b1sq;
  R ub1 = u0 * b10 + u1 * b11 + u2 * b12;
  un = u0;
  F[0] = rho * u0;
  F[1] = (rho * u0 * u0 + pt) - (b10 * B_0 + B0[0] * b10);
  F[2] = rho * u1 * u0 - (b11 * B_0 + B0[1] * b10);
  F[3] = rho * u2 * u0 - (b12 * B_0 + B0[2] * b10);
  F[4] = R(0);
  F[5] = u0 * B_1 - B_0 * u1;
  F[6] = u0 * B_2 - B_0 * u2;
  F[7] = u0 * (e1 + pt) - ub1 * B_0;
  U[0] = rho;
  U[1] = rho * u0;
  U[2] = rho * u1;
  U[3] = rho * u2;
  U[4] = b10;
  U[5] = b11;
  U[6] = b12;
  U[7] = e1;
  if constexpr (std::is_same<R, double>::value)
    cf = fast_speed_exact(gamma, rho, p, B_0, B_1, B_2);
  else
    cf = fast_speed_n<R>(gamma, rho, p, B_0, B_1, B_2);
}

// ---------------------------------------------------------------------------
// Ghost fill by point location (copy / restriction / prolongation / boundary).

struct GhostCtx {
  const GridDev* G;
  const BlockDev* blocks;
  const int32_t* levmap;
  const double* U;
  int32_t* err;
};

__device__ __forceinline__ int32_t map_lookup(const GridDev& G, const int32_t* levmap, int l, int bi, int bj,
                                              int bk) {
  int64_t nbi = static_cast<int64_t>(G.root[0]) << l, nbj = static_cast<int64_t>(G.root[1]) << l;
  return levmap[G.map_off[l] + (static_cast<int64_t>(bk) * nbj + bj) * nbi + bi];
}
// Leaf containing cell g of level lev (g inside the domain): same level or
// one coarser; -1 with ll = lev + 1 when the region is refined (2:1 balance).
__device__ __forceinline__ int locate(const GridDev& G, const int32_t* levmap, int lev, const int g[3], int& ll) {
  if (lev <= G.maxlev) {
    int id = map_lookup(G, levmap, lev, g[0] >> 3, g[1] >> 3, g[2] >> 3);
    if (id >= 0) { ll = lev; return id; }
  }
  if (lev >= 1) {
    int id = map_lookup(G, levmap, lev - 1, g[0] >> 4, g[1] >> 4, g[2] >> 4);
    if (id >= 0) { ll = lev - 1; return id; }
  }
  ll = lev + 1;
  return -1;
}
// Boundary mapping x, then y, then z: periodic wrap, outflow clamp (zero
// gradient); returns true when the fixed inflow state applies.
__device__ __forceinline__ bool bc_map(const GridDev& G, int lev, int g[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    int n = (G.root[a] << lev) * NC;
    if (g[a] >= 0 && g[a] < n) continue;
    int side = g[a] < 0 ? 0 : 1;
    int bc = G.bc[2 * a + side];
    if (bc == 0) g[a] = g[a] < 0 ? g[a] + n : g[a] - n;
    else if (bc == 1) g[a] = side ? n - 1 : 0;
    else return true;
  }
  return false;
}
__device__ __forceinline__ void load_cell(const GhostCtx& cx, int leaf, const int g[3], double out[8]) {
  const BlockDev& B = cx.blocks[leaf];
  int li = g[0] - B.bi * NC, lj = g[1] - B.bj * NC, lk = g[2] - B.bk * NC;
  const double* p = cx.U + static_cast<int64_t>(leaf) * (NV * NCELL) + (lk * NC + lj) * NC + li;
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = p[v * NCELL];
}
// Mean of the 8 children (level lev+1) of cell g, summed pairwise.
__device__ __noinline__ void restrict_cell(const GhostCtx& cx, int lev, const int g[3], double out[8]) {
  int f[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
  int ll;
  int leaf = locate(*cx.G, cx.levmap, lev + 1, f, ll);
  if (leaf < 0 || ll != lev + 1) {
    atomicOr(cx.err, ERR_BOUNDS);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = 0.0;
    return;
  }
  const BlockDev& B = cx.blocks[leaf];
  int li = f[0] - B.bi * NC, lj = f[1] - B.bj * NC, lk = f[2] - B.bk * NC;
  const double* p = cx.U + static_cast<int64_t>(leaf) * (NV * NCELL) + (lk * NC + lj) * NC + li;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const double* q = p + v * NCELL;
    double c0 = q[0], c1 = q[1], c2 = q[NC], c3 = q[NC + 1];
    double c4 = q[NC * NC], c5 = q[NC * NC + 1], c6 = q[NC * NC + NC], c7 = q[NC * NC + NC + 1];
    double s = __dadd_rn(__dadd_rn(__dadd_rn(c0, c1), __dadd_rn(c2, c3)),
                         __dadd_rn(__dadd_rn(c4, c5), __dadd_rn(c6, c7)));
    out[v] = 0.125 * s;
  }
}
// Copy or restriction at level lc (used for coarse samples of prolongation).
__device__ __noinline__ void coarse_value(const GhostCtx& cx, int lc, int gc[3], double out[8]) {
  const GridDev& G = *cx.G;
  if (bc_map(G, lc, gc)) {
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = G.Uinflow[v];
    return;
  }
  int ll;
  int leaf = locate(G, cx.levmap, lc, gc, ll);
  if (leaf >= 0 && ll == lc) load_cell(cx, leaf, gc, out);
  else if (leaf < 0) restrict_cell(cx, lc, gc, out);
  else {
    atomicOr(cx.err, ERR_BOUNDS);  // two levels coarser: excluded by 2:1 balance
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = 0.0;
  }
}
// Conservative state of ghost cell g (level lev): boundary mapping, then copy
// (same level), restriction (finer) or prolongation (coarser: coarse value plus
// (+-1/4) x minmod of the undivided coarse differences, axis by axis).
__device__ __noinline__ void ghost_value(const GhostCtx& cx, int lev, int g[3], double out[8]) {
  const GridDev& G = *cx.G;
  if (bc_map(G, lev, g)) {
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = G.Uinflow[v];
    return;
  }
  int ll;
  int leaf = locate(G, cx.levmap, lev, g, ll);
  if (leaf >= 0 && ll == lev) { load_cell(cx, leaf, g, out); return; }
  if (leaf < 0) { restrict_cell(cx, lev, g, out); return; }
  int gc[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
  double Vc[8];
  {
    int t[3] = {gc[0], gc[1], gc[2]};
    coarse_value(cx, lev - 1, t, Vc);
  }
  double acc[8];
#pragma unroll
  for (int v = 0; v < NV; v++) acc[v] = Vc[v];
#pragma unroll 1
  for (int a = 0; a < 3; a++) {
    double Vm[8], Vp[8];
    int tm[3] = {gc[0], gc[1], gc[2]}, tp[3] = {gc[0], gc[1], gc[2]};
    tm[a] -= 1;
    tp[a] += 1;
    coarse_value(cx, lev - 1, tm, Vm);
    coarse_value(cx, lev - 1, tp, Vp);
    double sgn = (g[a] & 1) ? 0.25 : -0.25;
#pragma unroll
    for (int v = 0; v < NV; v++) {
      double s = minmod_(__dsub_rn(Vc[v], Vm[v]), __dsub_rn(Vp[v], Vc[v]));
      acc[v] = __dadd_rn(acc[v], sgn * s);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = acc[v];
}

// Tile index of cell c (-2..9) along direction d at transverse (a, b).
__device__ __forceinline__ int tile_index(int d, int c, int a, int b) {
  int gi = 2 * d + (c >= NC ? 1 : 0);
  int ghost = NCELL + gi * 128 + (c < 0 ? c + 2 : c - NC) + 2 * (a + NC * b);
  int i = d == 0 ? c : a, j = d == 1 ? c : (d == 0 ? a : b), k = d == 2 ? c : b;
  int inner = (k * NC + j) * NC + i;
  return (c < 0 || c >= NC) ? ghost : inner;
}

// Fill face-slab ghost q (0..767) of block blk into the tile.
template <bool MIXED, class R>
__device__ __forceinline__ void fill_ghost(const StageArgs& a, const GhostCtx& cx, const BlockDev& B, int blk, int q,
                                           R* sT) {
  int s = q >> 7, loc = q & 127;
  int d = s >> 1, side = s & 1;
  int layer = loc & 1, ta = (loc >> 1) & 7, tb = loc >> 4;
  int c = side ? NC + layer : layer - 2;
  int ft = B.ftype[s];
  R w[8];
  if (ft == FACE_SAME || ft == FACE_OUTFLOW) {
    int src = ft == FACE_SAME ? B.fnb[s] : blk;
    int cn = ft == FACE_SAME ? (side ? c - NC : c + NC) : (side ? NC - 1 : 0);
    int i = d == 0 ? cn : ta, j = d == 1 ? cn : (d == 0 ? ta : tb), k = d == 2 ? cn : tb;
    int cell = (k * NC + j) * NC + i;
    if constexpr (MIXED) {
      const float* p = a.Win + static_cast<int64_t>(src) * (NV * NCELL) + cell;
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = p[v * NCELL];
    } else {
      const double* p = a.Uin + static_cast<int64_t>(src) * (NV * NCELL) + cell;
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = p[v * NCELL];
    }
  } else if (ft == FACE_INFLOW) {
    if constexpr (MIXED) {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = cx.G->Winflow32[v];
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = cx.G->Uinflow[v];
    }
  } else {
    int g[3];
    int i = d == 0 ? c : ta, j = d == 1 ? c : (d == 0 ? ta : tb), k = d == 2 ? c : tb;
    g[0] = B.bi * NC + i;
    g[1] = B.bj * NC + j;
    g[2] = B.bk * NC + k;
    double u[8];
    ghost_value(cx, B.level, g, u);
    if constexpr (MIXED) {
      prim_mixed(u, a.ph.gm1f, w);
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = u[v];
    }
  }
  int t = NCELL + q;
#pragma unroll
  for (int v = 0; v < NV; v++) sT[v * NTILE + t] = w[v];
}

// ---------------------------------------------------------------------------
// The fused stage kernel.

template <bool MIXED>
struct StageCfg {
  using R = typename std::conditional<MIXED, float, double>::type;
  static constexpr int NFCOMP = 12;  // 8 fluxes, face-averaged B1n, B0 (3)
  static constexpr size_t SMEM = sizeof(R) * (NV * NTILE + NFCOMP * NFACE);
};

template <bool MIXED>
__global__ void __launch_bounds__(STAGE_THREADS, MIXED ? 2 : 1) k_stage(const StageArgs a) {
  using R = typename StageCfg<MIXED>::R;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* sT = reinterpret_cast<R*>(smem_raw);       // [8][1280] tile
  R* sF = sT + NV * NTILE;                       // [12][576] face values
  __shared__ uint64_t bar;
  __shared__ R sred[STAGE_THREADS / 32];

  const int tid = threadIdx.x;
  const PhysDev& ph = a.ph;
  R gamma, inv_gm1;
  if constexpr (MIXED) { gamma = ph.gammaf; inv_gm1 = ph.inv_gm1f; }
  else { gamma = ph.gamma; inv_gm1 = ph.inv_gm1; }
  const bool has_b0 = ph.b0 != B0_NONE;

  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t parity = 0;

  const int nitems = (a.nblocks + a.blocks_per_item - 1) / a.blocks_per_item;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int b_end = min(a.nblocks, (item + 1) * a.blocks_per_item);
    for (int blk = item * a.blocks_per_item; blk < b_end; blk++) {
      const BlockDev& B = a.blocks[blk];
      const GridDev& G = a.grids[B.grid];
      GhostCtx cx{&G, a.blocks, a.levmap, a.Uin, a.err};

      // 1. interior by TMA bulk copies (one per variable), ghosts by threads
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bar, NV * NCELL * sizeof(R));
        const R* src = MIXED ? reinterpret_cast<const R*>(a.Win) : reinterpret_cast<const R*>(a.Uin);
        src += static_cast<int64_t>(blk) * (NV * NCELL);
#pragma unroll
        for (int v = 0; v < NV; v++) bulk_g2s(sT + v * NTILE, src + v * NCELL, NCELL * sizeof(R), &bar);
      }
      for (int q = tid; q < NGHOST; q += STAGE_THREADS) fill_ghost<MIXED, R>(a, cx, B, blk, q, sT);
      if (!mbar_wait_bounded(&bar, parity, a.err)) mbar_wait_bounded(&bar, parity, a.err);
      parity ^= 1u;
      __syncthreads();

      // 2. FP64 path: primitives in place over the whole tile
      if constexpr (!MIXED) {
        for (int c = tid; c < NTILE; c += STAGE_THREADS) {
          double U[8], W[8];
#pragma unroll
          for (int v = 0; v < NV; v++) U[v] = sT[v * NTILE + c];
          prim64(U, ph.gm1, W);
#pragma unroll
          for (int v = 0; v < NV; v++) sT[v * NTILE + c] = W[v];
        }
        __syncthreads();
      }

      // block geometry (per-level spacing precomputed on the host); positions
      // in the compute precision: FP64 for the FP64 form, FP32 for the mixed
      const int lev = B.level;
      R idx0, idx1, idx2, dxr0, dxr1, dxr2, lor0, lor1, lor2;
      if constexpr (MIXED) {
        idx0 = G.idxf[lev][0]; idx1 = G.idxf[lev][1]; idx2 = G.idxf[lev][2];
        dxr0 = G.dxf[lev][0]; dxr1 = G.dxf[lev][1]; dxr2 = G.dxf[lev][2];
        lor0 = G.lof[0]; lor1 = G.lof[1]; lor2 = G.lof[2];
      } else {
        idx0 = G.idx[lev][0]; idx1 = G.idx[lev][1]; idx2 = G.idx[lev][2];
        dxr0 = G.dx[lev][0]; dxr1 = G.dx[lev][1]; dxr2 = G.dx[lev][2];
        lor0 = G.lo[0]; lor1 = G.lo[1]; lor2 = G.lo[2];
      }
      const int gb0 = B.bi * NC, gb1 = B.bj * NC, gb2 = B.bk * NC;

      // per-cell accumulators (threads < 512 own cell tid)
      const int ci = tid & 7, cj = (tid >> 3) & 7, ck = tid >> 6;
      R res[8];
      R divb = R(0), divb0 = R(0), curl0 = R(0), curl1 = R(0), curl2 = R(0);
#pragma unroll
      for (int v = 0; v < NV; v++) res[v] = R(0);

#pragma unroll 1
      for (int d = 0; d < 3; d++) {
        // 3. faces of direction d: reconstruction + Rusanov flux in the frame
        //    (normal, t1, t2) = (d, d+1, d+2 mod 3)
        {
          const int t = tid;
          int f, ta, tb;
          if (d == 0) { f = t % 9; ta = (t / 9) & 7; tb = t / 72; }
          else if (d == 1) { ta = t & 7; f = (t >> 3) % 9; tb = t / 72; }
          else { ta = t & 7; tb = (t >> 3) & 7; f = t >> 6; }
          const int d1 = d == 2 ? 0 : d + 1, d2 = d == 0 ? 2 : d - 1;
          const int i0 = tile_index(d, f - 2, ta, tb), i1 = tile_index(d, f - 1, ta, tb);
          const int i2 = tile_index(d, f, ta, tb), i3 = tile_index(d, f + 1, ta, tb);
          // source variable of rotated component v
          R WL[8], WR[8];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            int sv = v;
            if (v >= 1 && v <= 3) sv = 1 + (v == 1 ? d : v == 2 ? d1 : d2);
            if (v >= 4 && v <= 6) sv = 4 + (v == 4 ? d : v == 5 ? d1 : d2);
            const R* col = sT + sv * NTILE;
            R w0 = col[i0], w1 = col[i1], w2 = col[i2], w3 = col[i3];
            R sl = limit_<R>(ph.limiter, w1 - w0, w2 - w1);
            R sr = limit_<R>(ph.limiter, w2 - w1, w3 - w2);
            WL[v] = w1 + R(0.5) * sl;
            WR[v] = w2 - R(0.5) * sr;
          }
          R B0f[3] = {R(0), R(0), R(0)}, B0r[3];
          if (has_b0) {
            // face centre: index f along d, (ta, tb) on the other two axes in
            // increasing order
            const int cc0 = d == 0 ? f : ta, cc1 = d == 1 ? f : (d == 0 ? ta : tb), cc2 = d == 2 ? f : tb;
            R xf[3];
            xf[0] = lor0 + (R(gb0 + cc0) + (d == 0 ? R(0) : R(0.5))) * dxr0;
            xf[1] = lor1 + (R(gb1 + cc1) + (d == 1 ? R(0) : R(0.5))) * dxr1;
            xf[2] = lor2 + (R(gb2 + cc2) + (d == 2 ? R(0) : R(0.5))) * dxr2;
            b0_at<R>(ph, xf, B0f);
          }
          B0r[0] = d == 0 ? B0f[0] : (d == 1 ? B0f[1] : B0f[2]);
          B0r[1] = d1 == 0 ? B0f[0] : (d1 == 1 ? B0f[1] : B0f[2]);
          B0r[2] = d2 == 0 ? B0f[0] : (d2 == 1 ? B0f[1] : B0f[2]);
          R FL[8], UL[8], FR[8], UR[8], unL, unR, cfL, cfR;
          phys_flux<R>(WL, B0r, gamma, inv_gm1, FL, UL, unL, cfL);
          phys_flux<R>(WR, B0r, gamma, inv_gm1, FR, UR, unR, cfR);
          R aL = Ops<R>::abs_(unL) + cfL, aR = Ops<R>::abs_(unR) + cfR;
          R cmax = aL > aR ? aL : aR;
          R Fr[8];
#pragma unroll
          for (int v = 0; v < NV; v++) Fr[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * cmax * (UR[v] - UL[v]);
          // store un-rotated
          sF[0 * NFACE + t] = Fr[0];
          sF[(1 + d) * NFACE + t] = Fr[1];
          sF[(1 + d1) * NFACE + t] = Fr[2];
          sF[(1 + d2) * NFACE + t] = Fr[3];
          sF[(4 + d) * NFACE + t] = Fr[4];
          sF[(4 + d1) * NFACE + t] = Fr[5];
          sF[(4 + d2) * NFACE + t] = Fr[6];
          sF[7 * NFACE + t] = Fr[7];
          sF[8 * NFACE + t] = R(0.5) * (WL[4] + WR[4]);
          if (has_b0) {
            sF[9 * NFACE + t] = B0f[0];
            sF[10 * NFACE + t] = B0f[1];
            sF[11 * NFACE + t] = B0f[2];
          }
        }
        __syncthreads();
        // 4. flux differences into the cells
        if (tid < NCELL) {
          int tl, th;
          if (d == 0) { tl = (ck * 8 + cj) * 9 + ci; th = tl + 1; }
          else if (d == 1) { tl = (ck * 9 + cj) * 8 + ci; th = tl + 8; }
          else { tl = (ck * 8 + cj) * 8 + ci; th = tl + 64; }
          const R id = d == 0 ? idx0 : (d == 1 ? idx1 : idx2);
#pragma unroll
          for (int v = 0; v < NV; v++) {
            R df = (sF[v * NFACE + th] - sF[v * NFACE + tl]) * id;
            res[v] = d == 0 ? -df : res[v] - df;
          }
          divb = divb + (sF[8 * NFACE + th] - sF[8 * NFACE + tl]) * id;
          if (has_b0) {
            R dbx = (sF[9 * NFACE + th] - sF[9 * NFACE + tl]) * id;
            R dby = (sF[10 * NFACE + th] - sF[10 * NFACE + tl]) * id;
            R dbz = (sF[11 * NFACE + th] - sF[11 * NFACE + tl]) * id;
            if (d == 0) { divb0 = dbx; curl2 = dby; curl1 = -dbz; }
            else if (d == 1) { divb0 = divb0 + dby; curl0 = dbz; curl2 = curl2 - dbx; }
            else { divb0 = divb0 + dbz; curl1 = curl1 + dbx; curl0 = curl0 - dby; }
          }
        }
        __syncthreads();
      }

      // 5. sources and update of the owned cell
      R smax_loc = R(0);
      if (tid < NCELL) {
        const int c = tid;
        bool in_body = false;
        if (B.body) {  // FP64, the same centre formula as the host and the oracle
          double x = G.lo[0] + ((static_cast<double>(gb0) + ci) + 0.5) * G.dx[lev][0];
          double y = G.lo[1] + ((static_cast<double>(gb1) + cj) + 0.5) * G.dx[lev][1];
          double z = G.lo[2] + ((static_cast<double>(gb2) + ck) + 0.5) * G.dx[lev][2];
          in_body = (x * x + y * y + z * z) < G.body_r * G.body_r;
        }
        R Wc[8];
#pragma unroll
        for (int v = 0; v < NV; v++) Wc[v] = sT[v * NTILE + c];
        R B0c[3] = {R(0), R(0), R(0)};
        if (has_b0) {
          R xr[3] = {lor0 + (R(gb0 + ci) + R(0.5)) * dxr0, lor1 + (R(gb1 + cj) + R(0.5)) * dxr1,
                     lor2 + (R(gb2 + ck) + R(0.5)) * dxr2};
          b0_at<R>(ph, xr, B0c);
        }
        R S[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        if (ph.powell) {
          R ub1 = Wc[1] * Wc[4] + Wc[2] * Wc[5] + Wc[3] * Wc[6];
#pragma unroll
          for (int e = 0; e < 3; e++) {
            S[1 + e] = -divb * (B0c[e] + Wc[4 + e]);
            S[4 + e] = -divb * Wc[1 + e];
          }
          S[7] = -divb * ub1;
        }
        if (has_b0) {
          R b1x = Wc[4], b1y = Wc[5], b1z = Wc[6];
          S[1] = (S[1] - b1x * divb0) + (b1y * curl2 - b1z * curl1);
          S[2] = (S[2] - b1y * divb0) + (b1z * curl0 - b1x * curl2);
          S[3] = (S[3] - b1z * divb0) + (b1x * curl1 - b1y * curl0);
        }
        const double cdt = a.beta * a.dt[B.grid];
        const int64_t base = static_cast<int64_t>(blk) * (NV * NCELL) + c;
        double Uo[8];
        bool bad = false;
#pragma unroll
        for (int v = 0; v < NV; v++) {
          R r = res[v] + S[v];
          double rd;
          if constexpr (MIXED) rd = f2d_int(r);
          else rd = r;
          double ub = a.Ubase[base + v * NCELL];
          double o;
          if (a.kind == 0) o = fma(cdt, rd, ub);
          else o = 0.5 * ub + 0.5 * fma(cdt, rd, a.Uin[base + v * NCELL]);
          if (a.kind == 2) o = rd;  // residual only (debug view)
          o = in_body ? (a.kind == 2 ? 0.0 : G.Ubody[v]) : o;
          Uo[v] = o;
          bad |= !(o == o) || isinf(o);
        }
        if (a.kind != 2) bad |= !(Uo[0] > 0.0);
        R Wn[8];
        bool need_w = MIXED || a.last;
        if (need_w && a.kind != 2) {
          if constexpr (MIXED) {
            double p64;
            prim_mixed(Uo, ph.gm1f, Wn, &p64);
            bad |= !(p64 > 0.0);
          } else {
            prim64(Uo, ph.gm1, Wn);
            bad |= !(Wn[7] > 0.0);
          }
        }
        if (bad && !in_body && a.kind != 2) {
          atomicOr(&a.err[0], ERR_NONPHYSICAL);
          atomicMin(&a.err[1], blk);
        }
        // outputs
        const bool write_u = !MIXED || a.last || a.write_u_all || B.need_u;
        if (write_u || a.kind == 2) {
#pragma unroll
          for (int v = 0; v < NV; v++) a.Uout[base + v * NCELL] = Uo[v];
        }
        if constexpr (MIXED) {
          if (a.kind != 2) {
#pragma unroll
            for (int v = 0; v < NV; v++) a.Wout[base + v * NCELL] = Wn[v];
          }
        }
        // CFL bound of the new state: sum_d (|u_d| + c_f,d) / dx_d
        if (a.last && !in_body && a.kind != 2) {
          R Bt[3] = {B0c[0] + Wn[4], B0c[1] + Wn[5], B0c[2] + Wn[6]};
          R s = R(0);
#pragma unroll
          for (int e = 0; e < 3; e++) {
            R bn = Bt[e], bt1 = Bt[(e + 1) % 3], bt2 = Bt[(e + 2) % 3];
            R cf;
            if constexpr (MIXED) {
              cf = fast_speed_n<R>(gamma, Wn[0], Wn[7], bn, bt1, bt2);
              s = s + (Ops<R>::abs_(Wn[1 + e]) + cf) * (e == 0 ? idx0 : (e == 1 ? idx1 : idx2));
            } else {
              cf = fast_speed_exact(ph.gamma, Wn[0], Wn[7], bn, bt1, bt2);
              s = s + (Ops<R>::abs_(Wn[1 + e]) + cf) / (e == 0 ? dxr0 : (e == 1 ? dxr1 : dxr2));
            }
          }
          smax_loc = s;
        }
      }
      if (a.last && a.kind != 2) {
        R m = smax_loc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          R q = __shfl_xor_sync(0xffffffffu, m, o);
          m = q > m ? q : m;
        }
        if ((tid & 31) == 0) sred[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
          R mm = R(0);
          for (int w = 0; w < STAGE_THREADS / 32; w++) mm = sred[w] > mm ? sred[w] : mm;
          double md;
          if constexpr (MIXED) md = f2d_int(mm);
          else md = mm;
          if (md > 0.0) atomicMax(&a.smax_next[B.grid], static_cast<unsigned long long>(__double_as_longlong(md)));
        }
      }
      __syncthreads();
    }
  }
}


// ---------------------------------------------------------------------------
// Small kernels.

// [8][nb][512] (external) <-> [nb][8][512] (internal) for blocks block0..block0+nb
__global__ void k_to_internal(const double* __restrict__ ext, double* __restrict__ in, int block0, int nb) {
  int64_t n = static_cast<int64_t>(nb) * NV * NCELL;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int c = static_cast<int>(e % NCELL);
    int64_t r = e / NCELL;
    int b = static_cast<int>(r % nb);
    int v = static_cast<int>(r / nb);
    in[(static_cast<int64_t>(block0 + b) * NV + v) * NCELL + c] = ext[e];
  }
}
__global__ void k_to_external(const double* __restrict__ in, double* __restrict__ ext, int block0, int nb) {
  int64_t n = static_cast<int64_t>(nb) * NV * NCELL;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int c = static_cast<int>(e % NCELL);
    int64_t r = e / NCELL;
    int b = static_cast<int>(r % nb);
    int v = static_cast<int>(r / nb);
    ext[e] = in[(static_cast<int64_t>(block0 + b) * NV + v) * NCELL + c];
  }
}

// Conservative inflow/body states (and the mixed-form primitives of the inflow).
__global__ void k_init_grid_states(GridDev* grids, int ngrids, double inv_gm1, double gm1) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrids) return;
  GridDev& G = grids[g];
  cons_from_prim<double>(G.Winflow, inv_gm1, G.Uinflow);
  cons_from_prim<double>(G.Wbody, inv_gm1, G.Ubody);
  float w[8];
  prim_mixed(G.Uinflow, static_cast<float>(gm1), w);
  for (int v = 0; v < NV; v++) G.Winflow32[v] = w[v];
}

// Mixed form: W = FP32 primitives of U for blocks [b0, b0+nb).
__global__ void k_prim_mixed(const double* __restrict__ U, float* __restrict__ Wt, int b0, int nb, float gm1f) {
  int64_t n = static_cast<int64_t>(nb) * NCELL;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int blk = b0 + static_cast<int>(e / NCELL), c = static_cast<int>(e % NCELL);
    int64_t base = static_cast<int64_t>(blk) * NV * NCELL + c;
    double u[8];
    float w[8];
    for (int v = 0; v < NV; v++) u[v] = U[base + v * NCELL];
    prim_mixed(u, gm1f, w);
    for (int v = 0; v < NV; v++) Wt[base + v * NCELL] = w[v];
  }
}

// CFL bound of the current state for blocks [b0, b0+nb): one CTA per block.
template <bool MIXED>
__global__ void k_cfl(const double* __restrict__ U, const float* __restrict__ Wt, const GridDev* grids,
                      const BlockDev* blocks, PhysDev ph, int b0, unsigned long long* smax) {
  __shared__ double sred[NCELL / 32];
  int blk = b0 + blockIdx.x, c = threadIdx.x;
  const BlockDev B = blocks[blk];
  const GridDev& G = grids[B.grid];
  int ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;
  double dxd[3], xc[3];
  for (int d = 0; d < 3; d++) dxd[d] = (G.hi[d] - G.lo[d]) / static_cast<double>((static_cast<int64_t>(G.root[d]) << B.level) * NC);
  xc[0] = G.lo[0] + ((static_cast<double>(B.bi * NC) + ci) + 0.5) * dxd[0];
  xc[1] = G.lo[1] + ((static_cast<double>(B.bj * NC) + cj) + 0.5) * dxd[1];
  xc[2] = G.lo[2] + ((static_cast<double>(B.bk * NC) + ck) + 0.5) * dxd[2];
  bool in_body = G.body_r > 0.0 && (xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]) < G.body_r * G.body_r;
  int64_t base = static_cast<int64_t>(blk) * NV * NCELL + c;
  double s = 0.0;
  if (!in_body) {
    if constexpr (MIXED) {
      float W[8], B0c[3] = {0.f, 0.f, 0.f};
      for (int v = 0; v < NV; v++) W[v] = Wt[base + v * NCELL];
      float xr[3] = {float(xc[0]), float(xc[1]), float(xc[2])};
      if (ph.b0 != B0_NONE) b0_at<float>(ph, xr, B0c);
      float Bt[3] = {B0c[0] + W[4], B0c[1] + W[5], B0c[2] + W[6]};
      float sf = 0.f;
      for (int e = 0; e < 3; e++) {
        float cf = fast_speed_n<float>(float(ph.gamma), W[0], W[7], Bt[e], Bt[(e + 1) % 3], Bt[(e + 2) % 3]);
        sf = sf + (fabsf(W[1 + e]) + cf) * rcp_approx(float(dxd[e]));
      }
      s = sf;
    } else {
      double u[8], W[8], B0c[3] = {0, 0, 0};
      for (int v = 0; v < NV; v++) u[v] = U[base + v * NCELL];
      prim64(u, ph.gm1, W);
      if (ph.b0 != B0_NONE) b0_at<double>(ph, xc, B0c);
      double Bt[3] = {B0c[0] + W[4], B0c[1] + W[5], B0c[2] + W[6]};
      for (int e = 0; e < 3; e++) {
        double cf = fast_speed_exact(ph.gamma, W[0], W[7], Bt[e], Bt[(e + 1) % 3], Bt[(e + 2) % 3]);
        s = s + (fabs(W[1 + e]) + cf) / dxd[e];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((c & 31) == 0) sred[c >> 5] = s;
  __syncthreads();
  if (c == 0) {
    double m = 0.0;
    for (int w = 0; w < NCELL / 32; w++) m = fmax(m, sred[w]);
    if (m > 0.0) atomicMax(&smax[B.grid], static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// Per-grid time-step bookkeeping.
//  mode 0 (before a step): dt = cfl > 0 ? cfl / smax : fixed_dt; smax_next = 0
//  mode 1 (after a step):  t += dt; smax = smax_next
__global__ void k_dt(int ngrids, int mode, double cfl, double fixed_dt, double* dt, double* t,
                     unsigned long long* smax, unsigned long long* smax_next) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrids) return;
  if (mode == 0) {
    double s = __longlong_as_double(static_cast<long long>(smax[g]));
    dt[g] = cfl > 0.0 ? cfl / s : fixed_dt;
    smax_next[g] = 0ull;
  } else {
    t[g] += dt[g];
    smax[g] = smax_next[g];
  }
}

// Debug view of the ghost fill: padded tiles [8][nb][12][12][12] (external
// layout) of blocks [b0, b0+nb): the interior and the face slabs, filled by
// the same code as the stage kernel (FP64 form); edge/corner cells are 0.
__global__ void k_debug_fill(const StageArgs a, int b0, int nb, double* T) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* sT = reinterpret_cast<double*>(smem_raw);
  const int blk = b0 + blockIdx.x;
  const BlockDev& B = a.blocks[blk];
  GhostCtx cx{&a.grids[B.grid], a.blocks, a.levmap, a.Uin, a.err};
  for (int e = threadIdx.x; e < NV * NCELL; e += blockDim.x)
    sT[(e / NCELL) * NTILE + (e % NCELL)] = a.Uin[static_cast<int64_t>(blk) * NV * NCELL + e];
  for (int q = threadIdx.x; q < NGHOST; q += blockDim.x) fill_ghost<false, double>(a, cx, B, blk, q, sT);
  __syncthreads();
  const int tile = 12 * 12 * 12;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    int i = e % 12 - 2, j = (e / 12) % 12 - 2, k = e / 144 - 2;
    int oi = (i < 0 || i >= NC), oj = (j < 0 || j >= NC), ok = (k < 0 || k >= NC);
    int t = -1;
    if (oi + oj + ok == 0) t = (k * NC + j) * NC + i;
    else if (oi + oj + ok == 1) {
      int d = oi ? 0 : (oj ? 1 : 2);
      int c = d == 0 ? i : (d == 1 ? j : k);
      int ta = d == 0 ? j : i, tb = d == 2 ? j : k;
      t = tile_index(d, c, ta, tb);
    }
    for (int v = 0; v < NV; v++)
      T[(static_cast<int64_t>(v) * nb + blockIdx.x) * tile + e] = t >= 0 ? sT[v * NTILE + t] : 0.0;
  }
}

// Conversion self-check against CUDA's own conversions: n float/double pairs.
__global__ void k_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  f2d_out[i] = f2d_int(f[i]);
  d2f_out[i] = d2f_int(d[i]);
}

// ---------------------------------------------------------------------------
// Host-side launchers (kernel stubs stay in this translation unit).

size_t stage_smem_bytes(bool mixed) {
  return mixed ? StageCfg<true>::SMEM : StageCfg<false>::SMEM;
}

cudaError_t stage_setup(int occ[2]) {
  cudaError_t e = cudaFuncSetAttribute(k_stage<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(StageCfg<false>::SMEM));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_stage<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(StageCfg<true>::SMEM));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_debug_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(double) * NV * NTILE));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_stage<false>, STAGE_THREADS, StageCfg<false>::SMEM);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_stage<true>, STAGE_THREADS, StageCfg<true>::SMEM);
  return e;
}

cudaError_t launch_stage_kernel(bool mixed, int grid, cudaStream_t st, const StageArgs& a) {
  if (mixed) k_stage<true><<<grid, STAGE_THREADS, StageCfg<true>::SMEM, st>>>(a);
  else k_stage<false><<<grid, STAGE_THREADS, StageCfg<false>::SMEM, st>>>(a);
  return cudaGetLastError();
}

static int grid_for(int64_t n) { return static_cast<int>(std::min<int64_t>((n + 255) / 256, 4096)); }

cudaError_t launch_to_internal(const double* ext, double* in, int block0, int nb, cudaStream_t st) {
  k_to_internal<<<grid_for(static_cast<int64_t>(nb) * NV * NCELL), 256, 0, st>>>(ext, in, block0, nb);
  return cudaGetLastError();
}
cudaError_t launch_to_external(const double* in, double* ext, int block0, int nb, cudaStream_t st) {
  k_to_external<<<grid_for(static_cast<int64_t>(nb) * NV * NCELL), 256, 0, st>>>(in, ext, block0, nb);
  return cudaGetLastError();
}
cudaError_t launch_init_grid_states(GridDev* grids, int ngrids, double inv_gm1, double gm1, cudaStream_t st) {
  k_init_grid_states<<<(ngrids + 63) / 64, 64, 0, st>>>(grids, ngrids, inv_gm1, gm1);
  return cudaGetLastError();
}
cudaError_t launch_prim_mixed(const double* U, float* Wt, int b0, int nb, float gm1f, cudaStream_t st) {
  k_prim_mixed<<<grid_for(static_cast<int64_t>(nb) * NCELL), 256, 0, st>>>(U, Wt, b0, nb, gm1f);
  return cudaGetLastError();
}
cudaError_t launch_cfl(bool mixed, const double* U, const float* Wt, const GridDev* grids, const BlockDev* blocks,
                       const PhysDev& ph, int b0, int nb, unsigned long long* smax, cudaStream_t st) {
  if (mixed) k_cfl<true><<<nb, NCELL, 0, st>>>(U, Wt, grids, blocks, ph, b0, smax);
  else k_cfl<false><<<nb, NCELL, 0, st>>>(U, Wt, grids, blocks, ph, b0, smax);
  return cudaGetLastError();
}
cudaError_t launch_dt(int ngrids, int mode, double cfl, double fixed_dt, double* dt, double* t,
                      unsigned long long* smax, unsigned long long* smax_next, cudaStream_t st) {
  k_dt<<<(ngrids + 127) / 128, 128, 0, st>>>(ngrids, mode, cfl, fixed_dt, dt, t, smax, smax_next);
  return cudaGetLastError();
}
cudaError_t launch_debug_fill(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st) {
  k_debug_fill<<<nb, 256, sizeof(double) * NV * NTILE, st>>>(a, b0, nb, T);
  return cudaGetLastError();
}
cudaError_t launch_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out) {
  k_check_conversions<<<(n + 255) / 256, 256>>>(f, d, n, f2d_out, d2f_out);
  return cudaGetLastError();
}

}  // namespace batsk
