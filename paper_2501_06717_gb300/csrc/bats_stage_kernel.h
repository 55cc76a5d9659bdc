// bats_stage_kernel.h -- the stage kernel template of the ideal-MHD
// finite-volume update on a 2:1 block-adaptive grid (arXiv 2501.06717,
// Algorithms 1-2; Eqs. 1-5) and every device helper it uses: ghost fill +
// primitive recovery + limited reconstruction + numerical flux (Rusanov, HLL,
// Linde) + Powell/B0 sources + conservative update (+ CFL bound of the new
// state), one 8^3 block per CTA iteration.  Included by bats_stage.cu (the
// Rusanov and learned instantiations, the small kernels, the launchers) and
// bats_stage_flux.cu (the HLL and Linde instantiations), which nvcc compiles
// in parallel.  Only templates and device functions live here; each
// translation unit's device code is a module of its own.
//
// FP64 form: shared-memory tile per block [8 variables][1280 cells] = the 512
// interior cells (1-D bulk copies, one per variable, completing on an
// mbarrier) followed by the six 2-layer face slabs (768 ghost cells) that the
// dimension-by-dimension stencil reads; edge and corner ghosts are never read
// by the stencil and are not filled.  Mixed form: the tile of FP32 primitives
// staged by tensor copies (see mx_issue_copies).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <algorithm>
#include <cuda_bf16.h>
#include <type_traits>

#include "bats_internal.h"
#include "bats_tc.h"

namespace batsk {

// ---------------------------------------------------------------------------
// Checked build (-DBATS_CHECKED, a separate library used by the tests in
// place of a memory checker): every index into the shared tile and face
// arrays, the state arrays, the block maps and the slot buffers is tested
// against its range before use; a failing index sets g_index_err and is
// replaced by the range's first value, so the access stays in bounds and the
// kernel runs to its end.  The normal build compiles the checks away.
#ifdef BATS_CHECKED
static __device__ int32_t g_index_err;  // one per translation unit
__device__ __forceinline__ int64_t chk(int64_t i, int64_t lo, int64_t hi) {
  if (i < lo || i >= hi) {
    atomicOr(&g_index_err, 1);
    return lo;
  }
  return i;
}
#else
__device__ __forceinline__ int64_t chk(int64_t i, int64_t, int64_t) { return i; }
#endif
__device__ __forceinline__ int chki(int i, int lo, int hi) { return static_cast<int>(chk(i, lo, hi)); }

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
// Hint that [p, p + bytes) will be read soon: bring it into L2 (p 16-byte
// aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
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
static __device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int32_t* err) {
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
// FP32: the smaller magnitude with a's sign when the signs agree, else 0 (a
// zero argument gives a signed zero, which adds like 0), in five operations.
template <>
__device__ __forceinline__ float minmod_<float>(float a, float b) {
  const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
  const float m = fminf(fabsf(a), fabsf(b));
  const float r = __uint_as_float((__float_as_uint(m) & 0x7fffffffu) | (ua & 0x80000000u));
  return static_cast<int32_t>(ua ^ ub) < 0 ? 0.f : r;
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
// kind 0 minmod, 1 MC, 2 none (first order: piecewise-constant faces)
// FP32: the same selection by the sign bits (2|a|, 2|b| and |a+b|/2 when the
// signs agree, else 0).
template <>
__device__ __forceinline__ float mc_<float>(float a, float b) {
  const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
  const float m = fminf(fminf(2.f * fabsf(a), 2.f * fabsf(b)), fabsf(0.5f * (a + b)));
  const float r = __uint_as_float((__float_as_uint(m) & 0x7fffffffu) | (ua & 0x80000000u));
  return static_cast<int32_t>(ua ^ ub) < 0 ? 0.f : r;
}
template <class R>
__device__ __forceinline__ R limit_(int kind, R a, R b) {
  return kind == 2 ? R(0) : (kind == 1 ? mc_(a, b) : minmod_(a, b));
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

// Mixed form: FP32 primitives of an FP64 state.  The pressure comes from the
// difference p/(gamma-1) = e1 - S, S = m.m/(2 rho) + B1.B1/2.  Where S <= e1/2
// the difference is at least half of e1 and FP32 operands give p to about
// 2e-7; where S > e1/2 (low beta, high Mach: the subtraction cancels) it is
// recomputed in FP64, 1/rho by an FP32 estimate plus one FP64 Newton-Raphson
// step.  *p64 (optional) receives e1 - S as a double (sign and finiteness
// checks).
__device__ __forceinline__ void prim_mixed(const double U[8], float gm1f, float W[8], double* p64 = nullptr) {
  const float rho32 = d2f_int(U[0]);
  const float rinv32 = rcp_approx(rho32);
  const float m0 = d2f_int(U[1]), m1 = d2f_int(U[2]), m2 = d2f_int(U[3]);
  const float b0 = d2f_int(U[4]), b1 = d2f_int(U[5]), b2 = d2f_int(U[6]);
  const float e32 = d2f_int(U[7]);
  const float ke = 0.5f * (m0 * m0 + m1 * m1 + m2 * m2) * rinv32;
  const float me = 0.5f * (b0 * b0 + b1 * b1 + b2 * b2);
  const float sum = ke + me;
  float x32 = e32 - sum;
  double x;
  if (sum > 0.5f * e32) {
    double r0 = f2d_int(rinv32);
    double e = fma(-U[0], r0, 1.0);
    double rinv = fma(r0, e, r0);
    double mm = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    double bb = U[4] * U[4] + U[5] * U[5] + U[6] * U[6];
    x = fma(-0.5, bb, U[7]);
    x = fma(-0.5 * mm, rinv, x);
    x32 = d2f_int(x);
  } else {
    x = f2d_int(x32);
  }
  W[0] = rho32;
  W[1] = m0 * rinv32;
  W[2] = m1 * rinv32;
  W[3] = m2 * rinv32;
  W[4] = b0;
  W[5] = b1;
  W[6] = b2;
  W[7] = x32 * gm1f;
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

// minmod of two doubles by integer tests on the bit patterns: 0 unless both
// are nonzero with the same sign, else the one of smaller magnitude (the
// second on a tie).  The same selection as the floating-point definition,
// without the FP64 comparison unit.
__device__ __forceinline__ double minmod_d(double a, double b) {
  long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  unsigned long long ma = static_cast<unsigned long long>(ia) & 0x7fffffffffffffffull;
  unsigned long long mb = static_cast<unsigned long long>(ib) & 0x7fffffffffffffffull;
  bool same = ((ia ^ ib) >= 0) && ma != 0 && mb != 0;
  long long r = ma < mb ? ia : ib;
  return same ? __longlong_as_double(r) : 0.0;
}
// The FP64 limiter's minmod by the same integer operations: the same value as
// the comparison form for every finite argument, issued on the integer pipe
// instead of the FP64 pipe (which bounds the FP64 form).
template <>
__device__ __forceinline__ double minmod_<double>(double a, double b) {
  return minmod_d(a, b);
}
// Validity tests on bit patterns: finite, and finite and > 0.
__device__ __forceinline__ bool finite_d(double x) {
  return (static_cast<unsigned>(__double2hiint(x)) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool positive_d(double x) { return __double_as_longlong(x) > 0 && finite_d(x); }
__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

// Primitives of U + dU from the primitives W of U (FP32 throughout).  The
// increments of the kinetic and magnetic energies are formed from dU itself,
// so the pressure carries no cancellation however small it is against the
// energy:  rho' = rho + drho,  u' = u + (dm - u drho) / rho',  B' = B + dB,
//   p' = p + (gamma - 1) [de - dK - (B.dB + |dB|^2 / 2)],
//   dK = (2 rho u.dm - rho drho |u|^2 + |dm|^2) / (2 rho')
// (dK is the change of |m|^2 / (2 rho) for m = rho u).
__device__ __forceinline__ void prim_increment(const float W[8], const float dU[8], float gm1f, float Wn[8]) {
  const float rc = W[0], u0 = W[1], u1 = W[2], u2 = W[3];
  const float rf = rc + dU[0];
  const float irf = rcp_approx(rf);
  const float udm = u0 * dU[1] + u1 * dU[2] + u2 * dU[3];
  const float usq = u0 * u0 + u1 * u1 + u2 * u2;
  const float dmsq = dU[1] * dU[1] + dU[2] * dU[2] + dU[3] * dU[3];
  const float dK = 0.5f * ((2.f * rc * udm - rc * dU[0] * usq) + dmsq) * irf;
  const float dM = (W[4] * dU[4] + W[5] * dU[5] + W[6] * dU[6]) + 0.5f * (dU[4] * dU[4] + dU[5] * dU[5] + dU[6] * dU[6]);
  Wn[0] = rf;
  Wn[1] = u0 + (dU[1] - u0 * dU[0]) * irf;
  Wn[2] = u1 + (dU[2] - u1 * dU[0]) * irf;
  Wn[3] = u2 + (dU[3] - u2 * dU[0]) * irf;
  Wn[4] = W[4] + dU[4];
  Wn[5] = W[5] + dU[5];
  Wn[6] = W[6] + dU[6];
  Wn[7] = W[7] + gm1f * ((dU[7] - dK) - dM);
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
  l = chki(l, 0, G.maxlev + 1);
  int64_t nbi = static_cast<int64_t>(G.root[0]) << l, nbj = static_cast<int64_t>(G.root[1]) << l;
  bi = static_cast<int>(chk(bi, 0, nbi));
  bj = static_cast<int>(chk(bj, 0, nbj));
  bk = static_cast<int>(chk(bk, 0, static_cast<int64_t>(G.root[2]) << l));
  return levmap[G.map_off[l] + (static_cast<int64_t>(bk) * nbj + bj) * nbi + bi];
}
// Leaf containing cell g of level lev (g inside the domain): same level or
// one coarser; -1 with ll = lev + 1 when the region is refined (2:1 balance).
__device__ __forceinline__ int locate(const GridDev& G, const int32_t* levmap, int lev, const int g[3], int& ll) {
  if (lev <= G.maxlev) {
    int id = map_lookup(G, levmap, lev, g[0] >> 3, g[1] >> 3, g[2] >> 3);
    if (id >= 0) { ll = lev; return chki(id, G.block0, G.block0 + G.nb); }
  }
  if (lev >= 1) {
    int id = map_lookup(G, levmap, lev - 1, g[0] >> 4, g[1] >> 4, g[2] >> 4);
    if (id >= 0) { ll = lev - 1; return chki(id, G.block0, G.block0 + G.nb); }
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
  int li = chki(g[0] - B.bi * NC, 0, NC), lj = chki(g[1] - B.bj * NC, 0, NC), lk = chki(g[2] - B.bk * NC, 0, NC);
  const double* p = cx.U + static_cast<int64_t>(leaf) * (NV * NCELL) + (lk * NC + lj) * NC + li;
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = p[v * NCELL];
}
// Mean of the 8 children (level lev+1) of cell g, summed pairwise.
static __device__ __noinline__ void restrict_cell(const GhostCtx& cx, int lev, const int g[3], double out[8]) {
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
  int li = chki(f[0] - B.bi * NC, 0, NC - 1), lj = chki(f[1] - B.bj * NC, 0, NC - 1),
      lk = chki(f[2] - B.bk * NC, 0, NC - 1);
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
static __device__ __noinline__ void coarse_value(const GhostCtx& cx, int lc, int gc[3], double out[8]) {
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
static __device__ __noinline__ void ghost_value(const GhostCtx& cx, int lev, int g[3], double out[8]) {
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
      double s = minmod_d(__dsub_rn(Vc[v], Vm[v]), __dsub_rn(Vp[v], Vc[v]));
      acc[v] = __dadd_rn(acc[v], sgn * s);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; v++) out[v] = acc[v];
}

// One variable of the mean of the 8 children (level lev+1) of cell g.
__device__ __forceinline__ double restrict_v(const GhostCtx& cx, int lev, const int g[3], int v) {
  int f[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
  int ll;
  int leaf = locate(*cx.G, cx.levmap, lev + 1, f, ll);
  if (leaf < 0 || ll != lev + 1) {
    atomicOr(cx.err, ERR_BOUNDS);
    return 0.0;
  }
  const BlockDev& B = cx.blocks[leaf];
  int li = f[0] - B.bi * NC, lj = f[1] - B.bj * NC, lk = f[2] - B.bk * NC;
  const double* q = cx.U + static_cast<int64_t>(leaf) * (NV * NCELL) + v * NCELL + (lk * NC + lj) * NC + li;
  double c0 = q[0], c1 = q[1], c2 = q[NC], c3 = q[NC + 1];
  double c4 = q[NC * NC], c5 = q[NC * NC + 1], c6 = q[NC * NC + NC], c7 = q[NC * NC + NC + 1];
  double sum = __dadd_rn(__dadd_rn(__dadd_rn(c0, c1), __dadd_rn(c2, c3)),
                         __dadd_rn(__dadd_rn(c4, c5), __dadd_rn(c6, c7)));
  return 0.125 * sum;
}
// One variable of the copy or restriction at level lc (coarse sample).
__device__ __forceinline__ double coarse_value_v(const GhostCtx& cx, int lc, int g0, int g1, int g2, int v) {
  const GridDev& G = *cx.G;
  int gc[3] = {g0, g1, g2};
  if (bc_map(G, lc, gc)) return G.Uinflow[v];
  int ll;
  int leaf = locate(G, cx.levmap, lc, gc, ll);
  if (leaf >= 0 && ll == lc) {
    const BlockDev& B = cx.blocks[leaf];
    int li = gc[0] - B.bi * NC, lj = gc[1] - B.bj * NC, lk = gc[2] - B.bk * NC;
    return cx.U[static_cast<int64_t>(leaf) * (NV * NCELL) + v * NCELL + (lk * NC + lj) * NC + li];
  }
  if (leaf < 0) return restrict_v(cx, lc, gc, v);
  atomicOr(cx.err, ERR_BOUNDS);  // two levels coarser: excluded by 2:1 balance
  return 0.0;
}

// Prolongation of one variable v for the 2x2x2 fine ghost cells of a face
// slab of face s that share coarse cell cc (0..15 over the face): the seven
// coarse samples and three minmod slopes are computed once, and the eight
// children are Vc + (+-1/4) sx + (+-1/4) sy + (+-1/4) sz summed x, then y,
// then z (the partial sums are shared between children).  Results go to
// scr[(local fine index in the slab) * 8 + v].
static __device__ __noinline__ void prolong_item(const GhostCtx& cx, const BlockDev& B, int s, int cc, int v, double* scr) {
  const int d = s >> 1, side = s & 1;
  const int ca = cc & 3, cb = cc >> 2;
  const int lev = B.level;
  // fine base cell (even coordinates) of the 2x2x2 group, global at level lev
  const int n0 = side ? NC : -2;
  int b0 = B.bi * NC + (d == 0 ? n0 : 2 * ca);
  int b1 = B.bj * NC + (d == 1 ? n0 : (d == 0 ? 2 * ca : 2 * cb));
  int b2 = B.bk * NC + (d == 2 ? n0 : 2 * cb);
  const int c0 = b0 >> 1, c1 = b1 >> 1, c2 = b2 >> 1;
  const double Vc = coarse_value_v(cx, lev - 1, c0, c1, c2, v);
  double qx, qy, qz;
  {
    double m = coarse_value_v(cx, lev - 1, c0 - 1, c1, c2, v), p = coarse_value_v(cx, lev - 1, c0 + 1, c1, c2, v);
    qx = 0.25 * minmod_d(__dsub_rn(Vc, m), __dsub_rn(p, Vc));
  }
  {
    double m = coarse_value_v(cx, lev - 1, c0, c1 - 1, c2, v), p = coarse_value_v(cx, lev - 1, c0, c1 + 1, c2, v);
    qy = 0.25 * minmod_d(__dsub_rn(Vc, m), __dsub_rn(p, Vc));
  }
  {
    double m = coarse_value_v(cx, lev - 1, c0, c1, c2 - 1, v), p = coarse_value_v(cx, lev - 1, c0, c1, c2 + 1, v);
    qz = 0.25 * minmod_d(__dsub_rn(Vc, m), __dsub_rn(p, Vc));
  }
  // even fine index -> -1/4, odd -> +1/4 along each axis
  const double tx0 = __dsub_rn(Vc, qx), tx1 = __dadd_rn(Vc, qx);
  const double t00 = __dsub_rn(tx0, qy), t01 = __dadd_rn(tx0, qy), t10 = __dsub_rn(tx1, qy), t11 = __dadd_rn(tx1, qy);
#pragma unroll
  for (int o = 0; o < 8; o++) {
    const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
    const double txy = ox ? (oy ? t11 : t10) : (oy ? t01 : t00);
    const double val = oz ? __dadd_rn(txy, qz) : __dsub_rn(txy, qz);
    // local index in the face slab: layer (normal), then the two transverse axes
    const int on = d == 0 ? ox : (d == 1 ? oy : oz);
    const int oa = d == 0 ? oy : ox;
    const int ob = d == 2 ? oy : oz;
    const int local = on + 2 * ((2 * ca + oa) + NC * (2 * cb + ob));
    scr[local * NV + v] = val;
  }
}

// ---------------------------------------------------------------------------
// Mixed form: ghost cells at resolution changes from the FP32 primitive
// copies W alone; the FP64 state is never read by a ghost fill.  Every value
// is the same quantity the FP64 path computes from the conservative state
// (the conservative mean of the children; the coarse value plus limited
// slopes of the conservative variables), rearranged so that the pressure is
// never the small difference of two large numbers: the stored p of each cell
// is FP64-accurate, and only differences and variances are formed in FP32.

// Primitives of cell g (global, level of `leaf`) from W.
__device__ __forceinline__ void load_w(const float* Wt, const BlockDev* blocks, int leaf, const int g[3], float w[8]) {
  const BlockDev& B = blocks[leaf];
  const int li = chki(g[0] - B.bi * NC, 0, NC), lj = chki(g[1] - B.bj * NC, 0, NC), lk = chki(g[2] - B.bk * NC, 0, NC);
  const float* p = Wt + static_cast<int64_t>(leaf) * (NV * NCELL) + (lk * NC + lj) * NC + li;
#pragma unroll
  for (int v = 0; v < NV; v++) w[v] = p[v * NCELL];
}

__device__ __forceinline__ float sum8(const float c[8]) {
  return ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}

// Restriction in primitive form: the conservative mean of the 8 children
// (level lev + 1) of cell g (level lev), as primitives.  With rho~ = mean rho_i,
// u~ = sum rho_i u_i / sum rho_i and B~ = mean B_i, the pressure of the mean
// state is p~ = mean p_i + (gamma - 1) [mean(rho_i |u_i - u~|^2) + mean(|B_i - B~|^2)] / 2
// (the kinetic and magnetic energies of the mean fall short of the mean
// energies by those two variances), a sum of non-negative terms.
// The restriction of the 8 fine cells whose corner cell (lowest i, j, k) is
// at p (a leaf's FP32 primitives, variable stride NCELL) to one coarse cell,
// as primitives: density and field the means, velocity the mass-weighted
// mean, pressure the mean plus the velocity and field variances.
static __device__ __noinline__ void restrict_at(const float* p, float gm1f, float w[8]) {
  const int off[8] = {0, 1, NC, NC + 1, NC * NC, NC * NC + 1, NC * NC + NC, NC * NC + NC + 1};
  float rho[8], c[8];
#pragma unroll
  for (int o = 0; o < 8; o++) rho[o] = p[off[o]];
  const float srho = sum8(rho);
  const float irs = rcp_approx(srho);
  float ut[3], var = 0.f;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    float u[8];
#pragma unroll
    for (int o = 0; o < 8; o++) u[o] = p[(1 + e) * NCELL + off[o]];
    const float ub = 0.125f * sum8(u);
#pragma unroll
    for (int o = 0; o < 8; o++) c[o] = rho[o] * (u[o] - ub);
    ut[e] = ub + sum8(c) * irs;
#pragma unroll
    for (int o = 0; o < 8; o++) {
      const float du = u[o] - ut[e];
      c[o] = rho[o] * du * du;
    }
    var += sum8(c);
  }
  float bt[3];
#pragma unroll
  for (int e = 0; e < 3; e++) {
    float b[8];
#pragma unroll
    for (int o = 0; o < 8; o++) b[o] = p[(4 + e) * NCELL + off[o]];
    bt[e] = 0.125f * sum8(b);
#pragma unroll
    for (int o = 0; o < 8; o++) {
      const float db = b[o] - bt[e];
      c[o] = db * db;
    }
    var += sum8(c);
  }
#pragma unroll
  for (int o = 0; o < 8; o++) c[o] = p[7 * NCELL + off[o]];
  w[0] = 0.125f * srho;
  w[1] = ut[0];
  w[2] = ut[1];
  w[3] = ut[2];
  w[4] = bt[0];
  w[5] = bt[1];
  w[6] = bt[2];
  w[7] = 0.125f * sum8(c) + gm1f * (0.0625f * var);
}

static __device__ __noinline__ void restrict_w(const float* Wt, const GridDev& G, const BlockDev* blocks,
                                        const int32_t* levmap, int lev, const int g[3], float gm1f, float w[8],
                                        int32_t* err) {
  const int f[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
  int ll;
  const int leaf = locate(G, levmap, lev + 1, f, ll);
  if (leaf < 0 || ll != lev + 1) {
    atomicOr(err, ERR_BOUNDS);
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = 0.f;
    return;
  }
  const BlockDev& B = blocks[leaf];
  const int li = chki(f[0] - B.bi * NC, 0, NC - 1), lj = chki(f[1] - B.bj * NC, 0, NC - 1),
            lk = chki(f[2] - B.bk * NC, 0, NC - 1);
  const float* p = Wt + static_cast<int64_t>(leaf) * (NV * NCELL) + (lk * NC + lj) * NC + li;
  restrict_at(p, gm1f, w);
}

// Primitives of the cell g (global, level lev): boundary mapping, then copy
// (leaf at lev) or restriction (finer region); a coarser leaf is excluded by
// the 2:1 balance and flagged.
static __device__ __noinline__ void sample_w(const float* Wt, const GridDev& G, const BlockDev* blocks,
                                      const int32_t* levmap, int lev, int g[3], float gm1f, float w[8],
                                      int32_t* err) {
  if (bc_map(G, lev, g)) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = G.Winflow32[v];
    return;
  }
  int ll;
  const int leaf = locate(G, levmap, lev, g, ll);
  if (leaf >= 0 && ll == lev) {
    load_w(Wt, blocks, leaf, g, w);
  } else if (leaf < 0) {
    restrict_w(Wt, G, blocks, levmap, lev, g, gm1f, w, err);
  } else {
    atomicOr(err, ERR_BOUNDS);
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = 0.f;
  }
}

// Coarse samples of the prolongation of one COARSER face: the 6 x 6 box of
// the coarse layer that holds the face's ghost cells (its 4 corners are not
// used), the 4 x 4 cells one coarse layer inwards (inside this block) and
// one outwards.  Per sample the table holds the conservative state (FP32),
// p and u.
constexpr int PSLOTS = 68;
constexpr int PSTRIDE = 12;

__device__ __forceinline__ bool psample(const BlockDev& B, int s, int k, int gc[3]) {
  const int d = s >> 1, side = s & 1;
  const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
  const int co[3] = {B.bi * (NC / 2), B.bj * (NC / 2), B.bk * (NC / 2)};
  int t1, t2, n;
  if (k < 36) {
    t1 = k % 6;
    t2 = k / 6;
    if ((t1 == 0 || t1 == 5) && (t2 == 0 || t2 == 5)) return false;
    n = side ? co[d] + 4 : co[d] - 1;
  } else {
    const int j = k < 52 ? k - 36 : k - 52;
    t1 = 1 + (j & 3);
    t2 = 1 + (j >> 2);
    n = k < 52 ? (side ? co[d] + 3 : co[d]) : (side ? co[d] + 5 : co[d] - 2);
  }
  gc[d] = n;
  gc[ta] = co[ta] - 1 + t1;
  gc[tb] = co[tb] - 1 + t2;
  return true;
}

// Fine ghost cell `local` (0..127, as in the face slab) of COARSER face s
// from the sample table: the coarse value plus (+-1/4) x minmod of the
// undivided coarse differences of the conservative variables (x, then y,
// then z), turned into primitives from the coarse cell's own primitives and
// the increment (prim_increment).
__device__ __forceinline__ void prolong_child_w(const float* tab, int s, int local, float gm1f, float w[8]) {
  const int d = s >> 1, side = s & 1;
  const int ta = d == 0 ? 1 : 0;
  const int on = local & 1, taf = (local >> 1) & 7, tbf = local >> 4;
  const int ca = taf >> 1, oa = taf & 1, cb = tbf >> 1, ob = tbf & 1;
  const int kc = (cb + 1) * 6 + (ca + 1);
  const int kin = 36 + ca + 4 * cb, kfar = 52 + ca + 4 * cb;
  const float* Uc = tab + kc * PSTRIDE;
  float dl[8];
#pragma unroll
  for (int v = 0; v < NV; v++) dl[v] = 0.f;
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
    int km, kp, odd;
    if (ax == d) {
      km = side ? kin : kfar;
      kp = side ? kfar : kin;
      odd = on;
    } else if (ax == ta) {
      km = kc - 1;
      kp = kc + 1;
      odd = oa;
    } else {
      km = kc - 6;
      kp = kc + 6;
      odd = ob;
    }
    const float* Um = tab + km * PSTRIDE;
    const float* Up = tab + kp * PSTRIDE;
    const float sg = odd ? 0.25f : -0.25f;
#pragma unroll
    for (int v = 0; v < NV; v++) dl[v] = dl[v] + sg * minmod_<float>(Uc[v] - Um[v], Up[v] - Uc[v]);
  }
  const float Wc[8] = {Uc[0], Uc[9], Uc[10], Uc[11], Uc[4], Uc[5], Uc[6], Uc[8]};
  prim_increment(Wc, dl, gm1f, w);
}

// Tile index of cell c (-2..9) along direction d at transverse (a, b).
__device__ __forceinline__ int tile_index(int d, int c, int a, int b) {
  int gi = 2 * d + (c >= NC ? 1 : 0);
  int ghost = NCELL + gi * 128 + (c < 0 ? c + 2 : c - NC) + 2 * (a + NC * b);
  int i = d == 0 ? c : a, j = d == 1 ? c : (d == 0 ? a : b), k = d == 2 ? c : b;
  int inner = (k * NC + j) * NC + i;
  return (c < 0 || c >= NC) ? ghost : inner;
}

// Staged tile of the mixed plain kernel (layouts: MX_* in bats_internal.h).
// Interior cell (i, j, k) of one variable in the swizzled tile.
__device__ __forceinline__ int mx_int(int i, int j, int k) { return 64 * k + 8 * j + (i ^ (4 * ((j >> 2) & 1))); }
// Start of face s's slab, the variable stride in it, and the element of
// ghost cell c (-2, -1 or 8, 9 along the face's axis) at transverse
// coordinates (ta, tb) (increasing axis order).
__device__ __forceinline__ int mx_slab_base(int s) {
  return s == 0 ? MX_GX0 : s == 1 ? MX_GX1 : s == 2 ? MX_GY0 : s == 3 ? MX_GY1 : s == 4 ? MX_GZ0 : MX_GZ1;
}
__device__ __forceinline__ int mx_slab_vstride(int d) { return d == 0 ? 256 : 128; }
__device__ __forceinline__ int mx_slab_elem(int d, int side, int c, int ta, int tb) {
  const int p = side ? c - NC : (d == 0 ? c + 4 : c + 2);
  return d == 0 ? (tb * NC + ta) * 4 + p : (d == 1 ? (tb * 2 + p) * NC + ta : (p * NC + tb) * NC + ta);
}
__device__ __forceinline__ uint32_t mx_slab_bytes(int d) { return d == 0 ? NV * 256 * 4 : NV * 128 * 4; }

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
    int src = chki(ft == FACE_SAME ? B.fnb[s] : blk, 0, a.nblocks);
    int cn = ft == FACE_SAME ? (side ? c - NC : c + NC) : (side ? NC - 1 : 0);
    int i = d == 0 ? cn : ta, j = d == 1 ? cn : (d == 0 ? ta : tb), k = d == 2 ? cn : tb;
    int cell = chki((k * NC + j) * NC + i, 0, NCELL);
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
    if constexpr (MIXED) {
      float wf[8];
      sample_w(a.Win, *cx.G, cx.blocks, cx.levmap, B.level, g, a.ph.gm1f, wf, cx.err);
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = wf[v];
    } else {
      double u[8];
      ghost_value(cx, B.level, g, u);
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = u[v];
    }
  }
  int t = chki(NCELL + q, NCELL, NTILE);
#pragma unroll
  for (int v = 0; v < NV; v++) sT[v * NTILE + t] = w[v];
}

// All face-slab ghosts of block blk.  Faces whose neighbour is coarser are
// filled by prolongation work items (one per coarse cell and variable, up to
// three such faces per block) through the FP64 scratch `scr` (3 x 128 x 8
// doubles); every other ghost cell is filled directly.  Ends with the tile
// complete for the calling CTA after a __syncthreads (the caller's, for
// blocks without coarser faces).
template <bool MIXED, class R>
__device__ __forceinline__ void fill_ghosts_block(const StageArgs& a, const GhostCtx& cx, const BlockDev& B, int blk,
                                                  R* sT, double* scr, int tid, int nthr) {
  unsigned cmask = 0;
#pragma unroll
  for (int f = 0; f < 6; f++) cmask |= (B.ftype[f] == FACE_COARSER ? 1u : 0u) << f;
  const int ncoarse = __popc(cmask);
  const int nheavy = ncoarse * 128;
  for (int q = tid; q < nheavy + NGHOST; q += nthr) {
    if (q < nheavy) {
      const int slot = q >> 7, rem = q & 127;
      unsigned m = cmask;
      for (int k = 0; k < slot; k++) m &= m - 1;
      const int sface = __ffs(m) - 1;
      prolong_item(cx, B, sface, rem >> 3, rem & 7, scr + slot * 128 * NV);
    } else {
      const int g = q - nheavy;
      if (!((cmask >> (g >> 7)) & 1u)) fill_ghost<MIXED, R>(a, cx, B, blk, g, sT);
    }
  }
  if (ncoarse) {
    __syncthreads();
    for (int q = tid; q < nheavy; q += nthr) {
      const int slot = q >> 7, local = q & 127;
      unsigned m = cmask;
      for (int k = 0; k < slot; k++) m &= m - 1;
      const int sface = __ffs(m) - 1;
      const double* u = scr + (slot * 128 + local) * NV;
      double uu[8];
#pragma unroll
      for (int v = 0; v < NV; v++) uu[v] = u[v];
      R w[8];
      if constexpr (MIXED) {
        prim_mixed(uu, a.ph.gm1f, w);
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) w[v] = uu[v];
      }
      const int t = NCELL + sface * 128 + local;
#pragma unroll
      for (int v = 0; v < NV; v++) sT[v * NTILE + t] = w[v];
    }
  }
}

// Mixed form: the face-slab ghosts of block blk from W.  Faces at a
// resolution change come precomputed from the ghost-slab buffer (k_amr_ghosts,
// launched before the stage): the stage kernel copies those slabs with bulk
// copies; with copy_amr the threads copy them here (debug view).
__device__ __forceinline__ void fill_ghosts_block_mixed(const StageArgs& a, const GhostCtx& cx, const BlockDev& B,
                                                        int blk, float* sT, int tid, int nthr, bool copy_amr) {
  unsigned amask = 0;
#pragma unroll
  for (int f = 0; f < 6; f++) amask |= (B.ftype[f] == FACE_COARSER || B.ftype[f] == FACE_FINER ? 1u : 0u) << f;
  for (int q = tid; q < NGHOST; q += nthr) {
    if (!((amask >> (q >> 7)) & 1u)) fill_ghost<true, float>(a, cx, B, blk, q, sT);
    else if (copy_amr) {
      const int s = q >> 7, local = q & 127;
      const float* src = a.gbuf + chk(B.rslot[s], 0, a.nslots) * GSLOT + local;
#pragma unroll
      for (int v = 0; v < NV; v++) sT[v * NTILE + NCELL + q] = src[v * 128];
    }
  }
}

template <bool MIXED>
struct StageCfg {
  using R = typename std::conditional<MIXED, float, double>::type;
  static constexpr int THREADS = MIXED ? STAGE_THREADS_MIXED : STAGE_THREADS_FP64;
  static constexpr int NFC = 9;  // per face: 8 fluxes and the face-averaged normal B1
  static constexpr size_t SMEM = sizeof(R) * (NV * NTILE + 3 * NFC * NFACE);
  // the mixed plain kernel's staged tile (MX_TILE floats, 1024-byte aligned
  // for the swizzled tensor copy) and its face values
  static constexpr size_t SMEM_MX = sizeof(float) * (MX_TILE + 3 * NFC * NFACE) + 1024;
};

// Load the 8 primitives of tile cell `idx` in the face frame (normal, t1, t2):
// offsets o[v] already select the rotated component's column.
template <class R>
__device__ __forceinline__ void load_rot(const R* sT, const int o[8], int idx, R w[8]) {
  idx = chki(idx, 0, NTILE);
#pragma unroll
  for (int v = 0; v < NV; v++) w[v] = sT[o[v] + idx];
}

// B0 at the centre of the face on the low side of cell (i, j, k) (block-local)
// normal to axis d, or at the cell centre when d < 0.
template <class R>
__device__ __forceinline__ void b0_face(const PhysDev& ph, int d, int i, int j, int k, int gb0, int gb1, int gb2,
                                        R lo0, R lo1, R lo2, R dx0, R dx1, R dx2, R B0[3]) {
  R x[3];
  x[0] = lo0 + (R(gb0 + i) + (d == 0 ? R(0) : R(0.5))) * dx0;
  x[1] = lo1 + (R(gb1 + j) + (d == 1 ? R(0) : R(0.5))) * dx1;
  x[2] = lo2 + (R(gb2 + k) + (d == 2 ? R(0) : R(0.5))) * dx2;
  b0_at<R>(ph, x, B0);
}

// ---------------------------------------------------------------------------
// Mixed form, plain faces (no learned correction): packed FP32.  GB300 issues
// FADD2 / FMUL2 / FFMA2 on float2 pairs (two FP32 lanes per instruction);
// every quantity of a face's two sides -- its left and right reconstructed
// states -- is such a pair, so the physical fluxes, the fast speeds and the
// flux combination of both sides take one instruction each.  One direction D
// per thread group (warp-uniform), a runtime value: the three groups run one
// copy of the code, which keeps the instruction working set small (a copy per
// direction measured 2.6 % slower).  The face values are stored doubled (2 F,
// and the sum of the two sides' normal B1);
// the cell phase scales its flux differences by 1/2.

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float p_sum(float2 a) { return a.x + a.y; }

// minmod as the median of (0, a, b): the smaller magnitude when a and b share
// a sign, else 0 (four min/max operations)
__device__ __forceinline__ float minmod_med(float a, float b) {
  return fminf(fmaxf(a, b), fmaxf(fminf(a, b), 0.f));
}
template <int LIM>
__device__ __forceinline__ float limit_f(float a, float b) {
  if constexpr (LIM == 2) return 0.f;
  else if constexpr (LIM == 1) return mc_<float>(a, b);
  else return minmod_med(a, b);
}

// Twice the numerical flux (Rusanov, HLL or Linde) of one face in the face frame from
// the pairs W2[v] = (left, right) of reconstructed primitives and the face's
// B0 (components in the frame).  The same physics as phys_flux + the flux
// combination of the generic path: split-field flux, fast speed with the
// total field, F = (F_L + F_R)/2 - cmax (U_R - U_L)/2 with cmax the larger
// |u_n| + c_f (Rusanov), the two-state HLL flux, or HLL with the contact wave
// restored (Linde).
// dsgn = 1: W2 = (left, right); dsgn = -1: W2 = (right, left).
template <bool HAS_B0, int FLX>
__device__ __forceinline__ void face_flux2(const float2 W2[8], const float B0r[3], float gamma, float inv_gm1,
                                           float dsgn, float Fr2[8]) {
  const float2 rho = W2[0], u0 = W2[1], u1 = W2[2], u2 = W2[3];
  const float2 b0 = W2[4], b1 = W2[5], b2 = W2[6], p = W2[7];
  float2 Bt0 = b0, Bt1 = b1, Bt2 = b2;
  if constexpr (HAS_B0) {
    Bt0 = p_add(b0, p_bc(B0r[0]));
    Bt1 = p_add(b1, p_bc(B0r[1]));
    Bt2 = p_add(b2, p_bc(B0r[2]));
  }
  // fast speeds of both sides (total field, along the normal)
  const float2 rinv = make_float2(rcp_approx(rho.x), rcp_approx(rho.y));
  const float2 b1sq = p_fma(b2, b2, p_fma(b1, b1, p_mul(b0, b0)));
  const float2 bsq = HAS_B0 ? p_fma(Bt2, Bt2, p_fma(Bt1, Bt1, p_mul(Bt0, Bt0))) : b1sq;
  const float2 a2 = p_mul(p_mul(p_bc(gamma), p), rinv);
  const float2 bb = p_mul(bsq, rinv);
  const float2 bn2 = p_mul(p_mul(Bt0, Bt0), rinv);
  const float2 s = p_add(a2, bb);
  const float2 disc = p_fma(p_mul(a2, bn2), p_bc(-4.f), p_mul(s, s));
  const float2 sq = make_float2(sqrt_approx(fmaxf(disc.x, 0.f)), sqrt_approx(fmaxf(disc.y, 0.f)));
  const float2 t = p_mul(p_add(s, sq), p_bc(0.5f));
  const float2 cf = make_float2(sqrt_approx(t.x), sqrt_approx(t.y));
  // coefficients of the combination 2F = sum over the two sides of (cF F + cU U)
  float2 cF = p_bc(1.f), cU;
  float lq = 0.f;  // Linde: twice the restored contact part's weight, delta alpha S_L S_R / (S_R - S_L)
  if constexpr (FLX == FLUX_HLL || FLX == FLUX_LINDE) {
    // S_L = min(unL - cfL, unR - cfR, 0), S_R = max(unL + cfL, unR + cfR, 0),
    // F = F_L - k ((F_R - F_L) - S_R (U_R - U_L)), k = S_L / (S_R - S_L)
    const float2 lo = p_fma(cf, p_bc(-1.f), u0), hi = p_add(u0, cf);
    const float sl = fminf(fminf(lo.x, lo.y), 0.f), sr = fmaxf(fmaxf(hi.x, hi.y), 0.f);
    const float den = sr - sl;
    const float k2 = den > 0.f ? 2.f * (sl * rcp_approx(den)) : 0.f;
    cF = dsgn > 0.f ? make_float2(2.f + k2, -k2) : make_float2(-k2, 2.f + k2);
    const float ks = dsgn * (k2 * sr);
    cU = make_float2(-ks, ks);
    if constexpr (FLX == FLUX_LINDE) {
      // the contact wave restored: alpha = minmod((rho_R - rho_L) - (p_R - p_L)
      // / c^2, rho_R - rho_L), delta = c / (c + |u_n|), with the means of the
      // two sides and c^2 = gamma p / rho (W2's order is (left, right) when
      // dsgn = 1)
      const float rm = 0.5f * p_sum(rho), pm = 0.5f * p_sum(p);
      const float c2 = gamma * pm * rcp_approx(rm), cs = sqrt_approx(c2);
      const float drho = dsgn * (rho.y - rho.x);
      const float alpha = minmod_med(drho - dsgn * (p.y - p.x) * rcp_approx(c2), drho);
      const float delta = cs * rcp_approx(cs + fabsf(0.5f * p_sum(u0)));
      lq = den > 0.f ? 2.f * delta * alpha * (sl * sr) * rcp_approx(den) : 0.f;
    }
  } else {
    const float cmax = dsgn * fmaxf(fabsf(u0.x) + cf.x, fabsf(u0.y) + cf.y);
    cU = make_float2(cmax, -cmax);
  }
  auto comb = [&](float2 F, float2 U) -> float {
    if constexpr (FLX == FLUX_HLL || FLX == FLUX_LINDE) return p_sum(p_fma(F, cF, p_mul(U, cU)));
    else return p_sum(p_fma(U, cU, F));
  };
  // split-field physical fluxes of both sides
  const float2 usq = p_fma(u2, u2, p_fma(u1, u1, p_mul(u0, u0)));
  float2 pt = p_fma(b1sq, p_bc(0.5f), p);
  if constexpr (HAS_B0)
    pt = p_add(pt, p_fma(p_bc(B0r[2]), b2, p_fma(p_bc(B0r[1]), b1, p_mul(p_bc(B0r[0]), b0))));
  const float2 e1 = p_fma(p, p_bc(inv_gm1), p_mul(p_bc(0.5f), p_fma(rho, usq, b1sq)));
  const float2 ub1 = p_fma(u2, b2, p_fma(u1, b1, p_mul(u0, b0)));
  const float2 m0 = p_mul(rho, u0), m1 = p_mul(rho, u1), m2 = p_mul(rho, u2);
  const float2 nB0 = p_mul(Bt0, p_bc(-1.f));
  float2 F1 = p_fma(b0, nB0, p_fma(m0, u0, pt));
  float2 F2 = p_fma(b1, nB0, p_mul(m1, u0));
  float2 F3 = p_fma(b2, nB0, p_mul(m2, u0));
  if constexpr (HAS_B0) {
    F1 = p_fma(b0, p_bc(-B0r[0]), F1);
    F2 = p_fma(b0, p_bc(-B0r[1]), F2);
    F3 = p_fma(b0, p_bc(-B0r[2]), F3);
  }
  const float2 F5 = p_fma(nB0, u1, p_mul(u0, Bt1));
  const float2 F6 = p_fma(nB0, u2, p_mul(u0, Bt2));
  const float2 F7 = p_fma(nB0, ub1, p_mul(u0, p_add(e1, pt)));
  Fr2[0] = comb(m0, rho);
  Fr2[1] = comb(F1, m0);
  Fr2[2] = comb(F2, m1);
  Fr2[3] = comb(F3, m2);
  Fr2[4] = p_sum(p_mul(b0, cU));
  Fr2[5] = comb(F5, b1);
  Fr2[6] = comb(F6, b2);
  Fr2[7] = comb(F7, e1);
  if constexpr (FLX == FLUX_LINDE) {
    const float um0 = 0.5f * p_sum(u0), um1 = 0.5f * p_sum(u1), um2 = 0.5f * p_sum(u2);
    Fr2[0] -= lq;
    Fr2[1] -= lq * um0;
    Fr2[2] -= lq * um1;
    Fr2[3] -= lq * um2;
    Fr2[7] -= lq * 0.5f * (um0 * um0 + um1 * um1 + um2 * um2);
  }
}

// ---------------------------------------------------------------------------
// Mixed form, plain stage kernel: tile staging.  Per block one thread issues
// the copies that complete on the block's mbarrier: the interior by one
// tensor copy (box 8 x 8 x 8 cells x 8 variables, 32-byte swizzle), each
// same-level face slab by one tensor copy of the neighbour's cells nearest
// the face (stage_tma = 1), and each precomputed slab of a face at a
// resolution change by a bulk copy from the ghost-slab buffer.  The threads
// fill the rest: outflow and inflow faces, and the same-level slabs when
// stage_tma = 0.  Layouts: see MX_* in bats_internal.h.

// 4-D tensor copy global -> shared (coordinates innermost first), completing
// on bar with the copied bytes.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}


// Primitives of face-slab ghost (s, layer, ta, tb) of block blk for a
// same-level, outflow or inflow face: the neighbour's (or, outflow, the
// block's own boundary) cell from Win, or the inflow state.
__device__ __forceinline__ void mx_ghost_value(const StageArgs& a, const GridDev& G, const BlockDev& B, int blk,
                                               int s, int layer, int ta, int tb, float w[8]) {
  const int d = s >> 1, side = s & 1;
  const int ft = B.ftype[s];
  if (ft == FACE_INFLOW) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = G.Winflow32[v];
    return;
  }
  const int c = side ? NC + layer : layer - 2;
  const int src = chki(ft == FACE_SAME ? B.fnb[s] : blk, 0, a.nblocks);
  const int cn = ft == FACE_SAME ? (side ? c - NC : c + NC) : (side ? NC - 1 : 0);
  const int i = d == 0 ? cn : ta, j = d == 1 ? cn : (d == 0 ? ta : tb), k = d == 2 ? cn : tb;
  const float* p = a.Win + static_cast<int64_t>(src) * (NV * NCELL) + chki((k * NC + j) * NC + i, 0, NCELL);
#pragma unroll
  for (int v = 0; v < NV; v++) w[v] = p[v * NCELL];
}

// Faces of block B whose slabs come by copies: tensor copies (same level,
// stage_tma = 1) and bulk copies from the ghost-slab buffer (resolution
// changes).
__device__ __forceinline__ void mx_copy_masks(const StageArgs& a, const BlockDev& B, unsigned& tmask,
                                              unsigned& amask) {
  tmask = 0;
  amask = 0;
#pragma unroll
  for (int f = 0; f < 6; f++) {
    const int ft = B.ftype[f];
    tmask |= (ft == FACE_SAME && a.stage_tma ? 1u : 0u) << f;
    amask |= (ft == FACE_COARSER || ft == FACE_FINER ? 1u : 0u) << f;
  }
}

// Issue (one thread) the copies of block blk's tile on bar: the interior,
// the copied face slabs.  Any generic-proxy access to sT that they overwrite
// must be ordered before (the caller's barrier); this fences the proxies.
__device__ __forceinline__ void mx_issue_copies(const StageArgs& a, const BlockDev& B, int blk, float* sT,
                                                uint64_t* bar) {
  unsigned tmask, amask;
  mx_copy_masks(a, B, tmask, amask);
  {
    fence_proxy_async();
    uint32_t bytes = NV * NCELL * 4;
#pragma unroll
    for (int f = 0; f < 6; f++)
      if (((tmask | amask) >> f) & 1u) bytes += mx_slab_bytes(f >> 1);
    mbar_expect_tx(bar, bytes);
    tma_load_4d(sT, &a.tm[0], 0, 0, 0, blk * NV, bar);
#pragma unroll
    for (int f = 0; f < 6; f++) {
      if ((tmask >> f) & 1u) {
        const int nb = chki(B.fnb[f], 0, a.nblocks), d = f >> 1, side = f & 1;
        // the neighbour's cells nearest the face: 4-7 / 0-3 along x, 6-7 / 0-1 along y and z
        const int o = side ? 0 : (d == 0 ? 4 : 6);
        tma_load_4d(sT + mx_slab_base(f), &a.tm[1 + d], d == 0 ? o : 0, d == 1 ? o : 0, d == 2 ? o : 0, nb * NV,
                    bar);
      } else if ((amask >> f) & 1u) {
        const float* g = a.gbuf + chk(B.rslot[f], 0, a.nslots) * GSLOT;
        bulk_g2s(sT + mx_slab_base(f), g, mx_slab_bytes(f >> 1), bar);
      }
    }
  }
}

// The calling threads fill the face slabs of block blk that no copy brings:
// outflow and inflow faces, and same-level faces when stage_tma = 0.
__device__ __forceinline__ void mx_fill_slabs(const StageArgs& a, const BlockDev& B, int blk, float* sT, int tid,
                                              int nthr) {
  unsigned tmask, amask;
  mx_copy_masks(a, B, tmask, amask);
  const unsigned fill = 0x3fu & ~(tmask | amask);
  const int nfill = __popc(fill) * 128;
  for (int q = tid; q < nfill; q += nthr) {
    const int slot = q >> 7, loc = q & 127;
    unsigned m = fill;
    for (int k = 0; k < slot; k++) m &= m - 1;
    const int s = __ffs(m) - 1, d = s >> 1, side = s & 1;
    const int layer = loc & 1, ta = (loc >> 1) & 7, tb = loc >> 4;
    float w[8];
    mx_ghost_value(a, a.grids[B.grid], B, blk, s, layer, ta, tb, w);
    const int c = side ? NC + layer : layer - 2;
    float* o = sT + mx_slab_base(s) + chki(mx_slab_elem(d, side, c, ta, tb), 0, mx_slab_vstride(d));
    const int vs = mx_slab_vstride(d);
#pragma unroll
    for (int v = 0; v < NV; v++) o[v * vs] = w[v];
  }
}

// Stage block blk into the tile sT: copies issued by thread 0 on bar, the
// remaining slabs filled by the calling threads.  Returns after the fill;
// the caller waits on bar and synchronises.
__device__ __forceinline__ void mx_stage_tile(const StageArgs& a, const BlockDev& B, int blk, float* sT,
                                              uint64_t* bar, int tid, int nthr) {
  if (tid == 0) mx_issue_copies(a, B, blk, sT, bar);
  mx_fill_slabs(a, B, blk, sT, tid, nthr);
}

// The faces of one direction D on this thread's grid line for the staged
// tile: lane half 0 walks up from cell -2 (faces 0-4), half 1 walks down from
// cell 9 (faces 8-5; its fifth step is face 4, computed by half 0, and not
// stored), so that at every step both halves read the same kind of cell (two
// ghost cells, then interior cells) with the same variable stride.  Walking
// down, a face's two sides come as (right, left): the dissipation's sign
// flips with the lane's direction.  Writes twice the fluxes (un-rotated
// components) and the sum of the two sides' normal B1 into sF[D][9][576].
// The mixed plain kernel keeps each direction's face values in the face frame
// (normal component first, then the next two axes cyclically), so that its
// one runtime copy of the face code stores at fixed offsets: the slot of
// variable v (x, y, z order) among the values of direction d.
__host__ __device__ constexpr int frot(int v, int d) {
  return (v >= 1 && v <= 6) ? ((v - 1) / 3) * 3 + 1 + (((v - 1) % 3 - d + 3) % 3) : v;
}
static_assert(frot(1, 0) == 1 && frot(2, 1) == 1 && frot(3, 2) == 1 && frot(1, 1) == 3 && frot(1, 2) == 2 &&
                  frot(4, 1) == 6 && frot(6, 2) == 4 && frot(7, 1) == 7 && frot(8, 2) == 8,
              "face-frame slots");

template <int LIM, bool HAS_B0, int FLX>
__device__ __forceinline__ void faces_mx(const int D, const StageArgs& a, const BlockDev& B, const float* sT, float* sF,
                                         int fline, int fhalf, float gamma, float inv_gm1, int gb0, int gb1, int gb2,
                                         float lor0, float lor1, float lor2, float dxr0, float dxr1, float dxr2) {
  const int D1 = D == 2 ? 0 : D + 1, D2 = D == 0 ? 2 : D - 1;
  constexpr int VI = NCELL;                 // variable stride, interior
  const int VG = D == 0 ? 256 : 128;    // variable stride, this direction's slabs
  const int fta = fline & 7, ftb = fline >> 3;
  const bool h1 = fhalf != 0;
  // interior index of cell c along the line
  auto cint = [&](int c) -> int {
    if (D == 0) return mx_int(c, fta, ftb);
    if (D == 1) return mx_int(fta, c, ftb);
    return mx_int(fta, ftb, c);
  };
  // window step j: half 0 cell j - 2, half 1 cell 9 - j
  auto cell_of = [&](int j) -> int { return h1 ? 9 - j : j - 2; };
  const int gbase = (h1 ? (D == 0 ? MX_GX1 : D == 1 ? MX_GY1 : MX_GZ1) : (D == 0 ? MX_GX0 : D == 1 ? MX_GY0 : MX_GZ0));
  auto load_g = [&](int j, float w[8]) {  // j = 0, 1: ghost cells
    const float* q = sT + gbase + chki(mx_slab_elem(D, h1 ? 1 : 0, cell_of(j), fta, ftb), 0, VG);
    w[0] = q[0]; w[1] = q[(1 + D) * VG]; w[2] = q[(1 + D1) * VG]; w[3] = q[(1 + D2) * VG];
    w[4] = q[(4 + D) * VG]; w[5] = q[(4 + D1) * VG]; w[6] = q[(4 + D2) * VG]; w[7] = q[7 * VG];
  };
  auto load_i = [&](int j, float w[8]) {  // j >= 2: interior cells
    const float* q = sT + chki(cint(cell_of(j)), 0, NCELL);
    w[0] = q[0]; w[1] = q[(1 + D) * VI]; w[2] = q[(1 + D1) * VI]; w[3] = q[(1 + D2) * VI];
    w[4] = q[(4 + D) * VI]; w[5] = q[(4 + D1) * VI]; w[6] = q[(4 + D2) * VI]; w[7] = q[7 * VI];
  };
  float W0[8], d[8], WL[8];
  {
    float Wm2[8], Wm1[8];
    load_g(0, Wm2);
    load_g(1, Wm1);
    load_i(2, W0);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      d[v] = W0[v] - Wm1[v];
      WL[v] = fmaf(0.5f, limit_f<LIM>(Wm1[v] - Wm2[v], d[v]), Wm1[v]);
    }
  }
  // face of step k: half 0 face k, half 1 face 8 - k
  const int fstep = h1 ? -1 : 1;
  float* const fo = sF + D * (9 * NFACE) + chki(fline * 9 + (h1 ? 8 : 0), 0, NFACE);
  const float dsgn = h1 ? -1.f : 1.f;
#pragma unroll
  for (int k = 0; k < 5; k++) {
    float Wp[8];
    load_i(k + 3, Wp);
    float2 W2[8];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const float dn = Wp[v] - W0[v];
      const float s0 = limit_f<LIM>(d[v], dn);
      W2[v] = make_float2(WL[v], fmaf(-0.5f, s0, W0[v]));
      WL[v] = fmaf(0.5f, s0, W0[v]);
      W0[v] = Wp[v];
      d[v] = dn;
    }
    float B0r[3] = {0.f, 0.f, 0.f};
    if constexpr (HAS_B0) {
      const int f = h1 ? 8 - k : k;
      const int ci_ = D == 0 ? f : fta, cj_ = D == 1 ? f : (D == 0 ? fta : ftb), ck_ = D == 2 ? f : ftb;
      float B0f[3];
      b0_face<float>(a.ph, D, ci_, cj_, ck_, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, B0f);
      B0r[0] = B0f[D];
      B0r[1] = B0f[D1];
      B0r[2] = B0f[D2];
    }
    float Fr2[8];
    face_flux2<HAS_B0, FLX>(W2, B0r, gamma, inv_gm1, dsgn, Fr2);
    const float bn2 = W2[4].x + W2[4].y;
    if (k == 4 && h1) continue;  // face 4 is half 0's
    float* const o = fo + k * fstep;  // in the face frame (frot)
#pragma unroll
    for (int v = 0; v < NV; v++) o[v * NFACE] = Fr2[v];
    o[8 * NFACE] = bn2;
    // refluxing: the block-face fluxes (face 0: half 0 step 0; face 8: half 1 step 0)
    if (k == 0 && a.freg) {
      const int sl = chki(B.rslot[2 * D + (h1 ? 1 : 0)], -1, a.nslots);
      if (sl >= 0) {
        double* r = a.freg + (static_cast<int64_t>(sl) * 64 + fta * NC + ftb) * NV;
        r[0] = f2d_int(0.5f * Fr2[0]);
        r[1 + D] = f2d_int(0.5f * Fr2[1]);
        r[1 + D1] = f2d_int(0.5f * Fr2[2]);
        r[1 + D2] = f2d_int(0.5f * Fr2[3]);
        r[4 + D] = f2d_int(0.5f * Fr2[4]);
        r[4 + D1] = f2d_int(0.5f * Fr2[5]);
        r[4 + D2] = f2d_int(0.5f * Fr2[6]);
        r[7] = f2d_int(0.5f * Fr2[7]);
      }
    }
  }
}

// Mixed plain kernel, common case (first or second midpoint stage with the
// global dt, no body cell in the block, no B0): the cell phase on the first
// 256 threads, two cells each -- cell c and cell c + 256 (the same (i, j),
// four layers apart in k) -- with the FP32 work packed over the pair and the
// FP64 accumulation per cell.  The same arithmetic, value for value, as the
// general cell phase (which runs the other cases, one cell per thread).
// Returns this thread's largest CFL bound (last stage), 0 otherwise.
// The pair's primitives Wc (the stage input) come from the tile, read by the
// caller before the next block's copies overwrite it (first stage only: the
// last stage reads them, for the Powell term, from memory).
__device__ __forceinline__ void cells_mx_pair_w(const float* sT, int tid, float2 Wc[8]) {
  if (tid >= NCELL / 2) return;
  const int cs = tid ^ (((tid >> 5) & 1) << 2);  // the interior's swizzle (the pair shares it)
#pragma unroll
  for (int v = 0; v < NV; v++) Wc[v] = make_float2(sT[v * NCELL + cs], sT[v * NCELL + cs + NCELL / 2]);
}
__device__ __forceinline__ float cells_mx_pair(const StageArgs& a, const GridDev& G, const BlockDev& B, int blk,
                                               const float2 Wc[8], const float* sF, int tid, float fx, float fy,
                                               float fz, float idx0, float idx1, float idx2, float gamma) {
  if (tid >= NCELL / 2) return 0.f;
  const PhysDev& ph = a.ph;
  const int c = tid, ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;  // ck 0..3; the pair's second cell: ck + 4
  const int tx = (ck * NC + cj) * 9 + ci, ty = (ck * NC + ci) * 9 + cj, tz = (cj * NC + ci) * 9 + ck;
  constexpr int DX = 4 * NC * 9, DZ = 4;   // face-index offsets of the second cell (x, y: +288; z: +4)
  const float* Fx = sF;
  const float* Fy = sF + 9 * NFACE;
  const float* Fz = sF + 2 * 9 * NFACE;
  const bool light = !a.last && !a.write_u_all;
  const int64_t base = static_cast<int64_t>(blk) * (NV * NCELL) + c;
  constexpr int H = NCELL / 2;  // the pair's second cell
  const float2 fx2 = p_bc(fx), fy2 = p_bc(fy), fz2 = p_bc(fz);
  // t[v] = sum_d (F_d,i+1/2 - F_d,i-1/2) / dx_d (v = 8: the face-averaged
  // normal B1, i.e. div B); the residual is -t + S
  float2 t[9];
#pragma unroll
  for (int v = 0; v < 9; v++) {
    const float* px = Fx + frot(v, 0) * NFACE + tx;  // face-frame slots (the x frame is the identity)
    const float* py = Fy + frot(v, 1) * NFACE + ty;
    const float* pz = Fz + frot(v, 2) * NFACE + tz;
    const float2 x0 = make_float2(px[0], px[DX]), x1 = make_float2(px[1], px[DX + 1]);
    const float2 y0 = make_float2(py[0], py[DX]), y1 = make_float2(py[1], py[DX + 1]);
    const float2 z0 = make_float2(pz[0], pz[DZ]), z1 = make_float2(pz[1], pz[DZ + 1]);
    float2 r = p_mul(p_fma(x0, p_bc(-1.f), x1), fx2);
    r = p_fma(p_fma(y0, p_bc(-1.f), y1), fy2, r);
    r = p_fma(p_fma(z0, p_bc(-1.f), z1), fz2, r);
    t[v] = r;
  }
  // residual R = -t + S (Powell: S = -div B (0, B, u, u.B1))
  float2 R[8];
#pragma unroll
  for (int v = 0; v < NV; v++) R[v] = p_mul(t[v], p_bc(-1.f));
  if (ph.powell) {
    // the stage input: in registers in the first stage; later stages read it
    // from memory here (the tile already receives the next block)
    float2 Wi[8];
    if (light) {
#pragma unroll
      for (int v = 0; v < NV; v++) Wi[v] = Wc[v];
    } else {
      const float* wi = a.Win + static_cast<int64_t>(blk) * (NV * NCELL) + c;
#pragma unroll
      for (int v = 0; v < NV; v++) Wi[v] = make_float2(wi[v * NCELL], wi[v * NCELL + NCELL / 2]);
    }
    const float2 nd = p_mul(t[8], p_bc(-1.f));
    const float2 ub1 = p_fma(Wi[3], Wi[6], p_fma(Wi[2], Wi[5], p_mul(Wi[1], Wi[4])));
#pragma unroll
    for (int e = 0; e < 3; e++) {
      R[1 + e] = p_fma(nd, Wi[4 + e], R[1 + e]);
      R[4 + e] = p_fma(nd, Wi[1 + e], R[4 + e]);
    }
    R[7] = p_fma(nd, ub1, R[7]);
  }
  const double cdt = a.beta * a.dt[B.grid];
  if (light) {
    // first midpoint stage: W* = W^n + the increment, in FP32
    const float c32 = d2f_int(cdt);
    float2 dU[8];
#pragma unroll
    for (int v = 0; v < NV; v++) dU[v] = p_mul(p_bc(c32), R[v]);
    const float gm1f = ph.gm1f;
    const float2 rf = p_add(Wc[0], dU[0]);
    const float2 irf = make_float2(rcp_approx(rf.x), rcp_approx(rf.y));
    const float2 udm = p_fma(Wc[3], dU[3], p_fma(Wc[2], dU[2], p_mul(Wc[1], dU[1])));
    const float2 usq = p_fma(Wc[3], Wc[3], p_fma(Wc[2], Wc[2], p_mul(Wc[1], Wc[1])));
    const float2 dmsq = p_fma(dU[3], dU[3], p_fma(dU[2], dU[2], p_mul(dU[1], dU[1])));
    // dK = ((2 rho u.dm - rho drho |u|^2) + |dm|^2) / (2 rho')
    const float2 k1 = p_mul(p_mul(p_bc(2.f), Wc[0]), udm);
    const float2 k2 = p_mul(p_mul(Wc[0], dU[0]), usq);
    const float2 dK = p_mul(p_mul(p_bc(0.5f), p_add(p_fma(k2, p_bc(-1.f), k1), dmsq)), irf);
    const float2 bdb = p_fma(Wc[6], dU[6], p_fma(Wc[5], dU[5], p_mul(Wc[4], dU[4])));
    const float2 db2 = p_fma(dU[6], dU[6], p_fma(dU[5], dU[5], p_mul(dU[4], dU[4])));
    const float2 dM = p_fma(p_bc(0.5f), db2, bdb);
    float2 Wl[8];
    Wl[0] = rf;
#pragma unroll
    for (int e = 1; e < 4; e++) Wl[e] = p_fma(p_fma(Wc[e], p_mul(dU[0], p_bc(-1.f)), dU[e]), irf, Wc[e]);
#pragma unroll
    for (int e = 4; e < 7; e++) Wl[e] = p_add(Wc[e], dU[e]);
    Wl[7] = p_fma(p_bc(gm1f), p_add(p_fma(dK, p_bc(-1.f), dU[7]), p_mul(dM, p_bc(-1.f))), Wc[7]);
    bool badA = !(Wl[0].x > 0.f) || !(Wl[7].x > 0.f), badB = !(Wl[0].y > 0.f) || !(Wl[7].y > 0.f);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      badA |= !finite_f(Wl[v].x);
      badB |= !finite_f(Wl[v].y);
    }
    if (badA || badB) {
      atomicOr(&a.err[0], ERR_NONPHYSICAL);
      atomicMin(&a.err[1], blk);
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      a.Wout[base + v * NCELL] = Wl[v].x;
      a.Wout[base + v * NCELL + H] = Wl[v].y;
    }
    return 0.f;
  }
  // last stage (or the FP64 state kept): U^{n+1} = U^n + c R in FP64, then
  // the FP32 primitives (FP64 pressure where it cancels) and the CFL bound.
  // Both cells' new states before any store (Uout may alias Ubase, so the
  // base-state loads of the pair precede every store)
  double U2[2][8];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    U2[0][v] = fma(cdt, f2d_int(R[v].x), a.Ubase[base + v * NCELL]);
    U2[1][v] = fma(cdt, f2d_int(R[v].y), a.Ubase[base + H + v * NCELL]);
  }
  float2 Wn[8];
  bool bad = false;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int64_t b = base + h * H;
    double* const Uo = U2[h];
#pragma unroll
    for (int v = 0; v < NV; v++) bad |= !finite_d(Uo[v]);
    bad |= !positive_d(Uo[0]);
    float w[8];
    double p64;
    prim_mixed(Uo, ph.gm1f, w, &p64);
    bad |= !positive_d(p64);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      a.Uout[b + v * NCELL] = Uo[v];
      a.Wout[b + v * NCELL] = w[v];
      if (h) Wn[v].y = w[v];
      else Wn[v].x = w[v];
    }
  }
  if (bad) {
    atomicOr(&a.err[0], ERR_NONPHYSICAL);
    atomicMin(&a.err[1], blk);
  }
  if (!a.last) return 0.f;
  // CFL bound sum_d (|u_d| + c_f,d) / dx_d of both cells (fast speeds with
  // the total field B1, no B0 here); cells that refluxing corrects afterwards
  // are bounded by the correction kernel
  const float2 rinv = make_float2(rcp_approx(Wn[0].x), rcp_approx(Wn[0].y));
  const float2 a2 = p_mul(p_mul(p_bc(gamma), Wn[7]), rinv);
  const float2 bsq = p_fma(Wn[6], Wn[6], p_fma(Wn[5], Wn[5], p_mul(Wn[4], Wn[4])));
  const float2 b2 = p_mul(bsq, rinv);
  const float2 s = p_add(a2, b2);
  const float2 ss = p_mul(s, s);
  float2 sacc = p_bc(0.f);
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const float2 bn2 = p_mul(p_mul(Wn[4 + e], Wn[4 + e]), rinv);
    const float2 disc = p_fma(p_mul(a2, bn2), p_bc(-4.f), ss);
    const float2 sq = make_float2(sqrt_approx(fmaxf(disc.x, 0.f)), sqrt_approx(fmaxf(disc.y, 0.f)));
    const float2 q = p_mul(p_add(s, sq), p_bc(0.5f));
    const float2 cf = make_float2(sqrt_approx(q.x), sqrt_approx(q.y));
    const float2 au = make_float2(fabsf(Wn[1 + e].x), fabsf(Wn[1 + e].y));
    sacc = p_fma(p_add(au, cf), p_bc(e == 0 ? idx0 : (e == 1 ? idx1 : idx2)), sacc);
  }
  float m = 0.f;
  if (a.freg) {
    // reflux-corrected cells (next to a refined face) are left out here
    const bool rA = (ci == 0 && B.ftype[0] == FACE_FINER) || (ci == NC - 1 && B.ftype[1] == FACE_FINER) ||
                    (cj == 0 && B.ftype[2] == FACE_FINER) || (cj == NC - 1 && B.ftype[3] == FACE_FINER) ||
                    (ck == 0 && B.ftype[4] == FACE_FINER);
    const bool rB = (ci == 0 && B.ftype[0] == FACE_FINER) || (ci == NC - 1 && B.ftype[1] == FACE_FINER) ||
                    (cj == 0 && B.ftype[2] == FACE_FINER) || (cj == NC - 1 && B.ftype[3] == FACE_FINER) ||
                    (ck + 4 == NC - 1 && B.ftype[5] == FACE_FINER);
    m = fmaxf(rA ? 0.f : sacc.x, rB ? 0.f : sacc.y);
  } else {
    m = fmaxf(sacc.x, sacc.y);
  }
  return m;
}

constexpr int TC_TILE_F = 128;  // rows per tensor-core tile (MMA M = tensor-memory lanes)
// ---------------------------------------------------------------------------
// Learned correction fused into the mixed form's stage kernel.  At every face
// step of the face phase the CTA's 384 threads hold 384 faces (one each):
// thread t's face is row t % 128 of tile t / 128, the tensor-memory lane its
// warp may read.  The three layers run on the tensor cores (tcgen05.mma,
// M = 128, K = 16 per instruction, BF16 operands from shared memory in the
// no-swizzle K-major canonical layout, FP32 accumulators in tensor memory,
// 64 columns per tile), each thread turning its own row's accumulator into
// the next layer's BF16 operand and, after the last layer, into its own
// face's correction.  As in the inference kernel the biases ride in the
// products (ones in the inputs' and activations' bias columns, the bias
// pairs in the weights) and the hidden activations are twice the GELU (the
// next layer's weights halved).

struct LrnSmem {
  alignas(128) uint8_t x[3][TC_TILE_F * 96];   // inputs, K = 48 (40 features, the bias columns, zeros)
  alignas(128) uint8_t h[3][TC_TILE_F * 160];  // hidden activations, K = 80 (64, the bias columns, zeros)
  alignas(128) uint8_t w1[64 * 96];             // B of layer 1: N = 64, K = 48
  alignas(128) uint8_t w2[64 * 160];            // B of layer 2: N = 64, K = 80 (weights halved)
  alignas(128) uint8_t w3[16 * 160];            // B of layer 3: N = 16 (8 outputs, 8 zero rows), K = 80 (halved)
  uint64_t bar[3];                              // MMA completion, per tile (warp group)
  uint32_t tmem;
};
constexpr int LRN_TMEM_COLS = 256;  // 3 tiles x 64 columns, rounded up to a power of two
// the mixed learned kernel: the generic tile and face values, then the
// fused network's operands and weights (128-byte aligned)
constexpr size_t kSmemLx = (sizeof(float) * (NV * NTILE + 3 * 9 * NFACE) + 127) / 128 * 128 + sizeof(LrnSmem) + 128;

// Weights into shared memory and the constant columns of the activation
// tiles (all threads), tensor memory and the MMA barrier (warp 0, thread 0).
__device__ __forceinline__ void lrn_setup(LrnSmem& s, const MlpDev& m, int tid, int nthr) {
  for (int e = tid; e < 64 * 6; e += nthr) {
    const int r = e / 6, kc = e % 6;
    *reinterpret_cast<uint4*>(s.w1 + cm_off(r, kc, SBO_K48)) = *reinterpret_cast<const uint4*>(m.w1b + r * 24 + kc * 4);
  }
  for (int e = tid; e < 64 * 10; e += nthr) {
    const int r = e / 10, kc = e % 10;
    *reinterpret_cast<uint4*>(s.w2 + cm_off(r, kc, SBO_K80)) = *reinterpret_cast<const uint4*>(m.w2b + r * 40 + kc * 4);
  }
  for (int e = tid; e < 16 * 10; e += nthr) {
    const int r = e / 10, kc = e % 10;
    *reinterpret_cast<uint4*>(s.w3 + cm_off(r, kc, SBO_K80)) = *reinterpret_cast<const uint4*>(m.w3b + r * 40 + kc * 4);
  }
  const uint4 ones = make_uint4(pack_bf16(1.f, 1.f), 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
  for (int e = tid; e < 3 * TC_TILE_F; e += nthr) {
    uint8_t* h = s.h[e / TC_TILE_F];
    *reinterpret_cast<uint4*>(h + cm_off(e % TC_TILE_F, 8, SBO_K80)) = ones;
    *reinterpret_cast<uint4*>(h + cm_off(e % TC_TILE_F, 9, SBO_K80)) = zero;
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&s.tmem)),
                 "r"(LRN_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init_tc(&s.bar[0]);
    mbar_init_tc(&s.bar[1]);
    mbar_init_tc(&s.bar[2]);
  }
}
// pending: this thread's last wait on its group's barrier ran out (the group's
// MMAs may still run): its group leader waits for them once more.
__device__ __forceinline__ void lrn_teardown(LrnSmem& s, int tid, bool pending, uint32_t phase, int32_t* err) {
  if (pending && (tid & 127) == 0) mbar_wait_bounded_tc(&s.bar[tid >> 7], phase, err);
  tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(LRN_TMEM_COLS)
                 : "memory");
  }
}

// A barrier of the 128 threads of warp group g (named barrier 1 + g) that
// returns whether any of them passed `bad`.
__device__ __forceinline__ bool group_sync_or(int g, bool bad) {
  uint32_t any;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(any)
      : "r"(bad ? 1u : 0u), "r"(1 + g)
      : "memory");
  return any != 0;
}

// Layer `layer` (0, 1, 2) of this warp group's tile (the groups run apart:
// each hands its tile to the tensor cores and waits for its own products
// while the others compute): after a barrier of the group, one elected
// thread of its first warp issues the MMAs (descriptors built
// warp-uniformly; K slice k: 256 bytes further, 16 in the descriptor's
// address field) and commits them to the group's barrier; every thread of
// the group waits (bounded).  false for the whole group when some wait ran
// out (pending then marks the threads whose own wait did).
__device__ __forceinline__ bool lrn_layer(LrnSmem& s, int layer, int tid, uint32_t& phase, bool& pending,
                                          int32_t* err) {
  const int g = tid >> 7;
  proxy_fence_smem();
  tc_fence_before();
  group_sync_or(g, false);
  if ((tid & 127) < 32) {
    constexpr uint32_t ID64 = umma_idesc_bf16(TC_TILE_F, 64), ID16 = umma_idesc_bf16(TC_TILE_F, 16);
    const uint64_t bw = layer == 0 ? umma_sdesc(tc_saddr(s.w1), 128, SBO_K48)
                                   : umma_sdesc(tc_saddr(layer == 1 ? s.w2 : s.w3), 128, SBO_K80);
    const uint64_t ba = layer == 0 ? umma_sdesc(tc_saddr(s.x[g]), 128, SBO_K48)
                                   : umma_sdesc(tc_saddr(s.h[g]), 128, SBO_K80);
    if (elect_one()) {
      tc_fence_after();
      const uint32_t d = s.tmem + 64 * g;
      if (layer == 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) umma_bf16(d, ba + 16 * k, bw + 16 * k, ID64, k);
      } else {
#pragma unroll
        for (int k = 0; k < 5; k++) umma_bf16(d, ba + 16 * k, bw + 16 * k, layer == 1 ? ID64 : ID16, k);
      }
      umma_commit(&s.bar[g]);
    }
    __syncwarp();
  }
  const bool got = mbar_wait_bounded_tc(&s.bar[g], phase, err);
  if (!got) pending = true;
  if (group_sync_or(g, !got)) return false;  // phase kept: the teardown waits on it once more
  phase ^= 1u;
  tc_fence_after();
  return true;
}

// The network for this thread's face (row tid % 128 of tile tid / 128):
// xrow its 48 BF16 inputs (6 chunks of 8; the last chunk is replaced by the
// bias columns), y its 8 outputs.  false (for every thread of the warp group)
// when a wait ran out.
__device__ __forceinline__ bool lrn_network(LrnSmem& s, const uint4 xrow[6], float y[8], int tid, uint32_t& phase,
                                            bool& pending, int32_t* err) {
  const int tile = tid >> 7, row = tid & 127;
  const uint32_t tl = s.tmem + (static_cast<uint32_t>(32 * ((tid >> 5) & 3)) << 16) + 64 * tile;
#pragma unroll
  for (int kc = 0; kc < 5; kc++) *reinterpret_cast<uint4*>(s.x[tile] + cm_off(row, kc, SBO_K48)) = xrow[kc];
  *reinterpret_cast<uint4*>(s.x[tile] + cm_off(row, 5, SBO_K48)) = make_uint4(pack_bf16(1.f, 1.f), 0u, 0u, 0u);
#pragma unroll 1
  for (int layer = 0; layer < 2; layer++) {
    if (!lrn_layer(s, layer, tid, phase, pending, err)) return false;
#pragma unroll
    for (int q = 0; q < 2; q++) {
      float z[32];
      tmem_ld32(tl + 32 * q, z);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const float* v = z + 8 * c;
        *reinterpret_cast<uint4*>(s.h[tile] + cm_off(row, 4 * q + c, SBO_K80)) =
            make_uint4(gelu2x_pack(v[0], v[1]), gelu2x_pack(v[2], v[3]), gelu2x_pack(v[4], v[5]),
                       gelu2x_pack(v[6], v[7]));
      }
    }
  }
  if (!lrn_layer(s, 2, tid, phase, pending, err)) return false;
  float v[16];
  tmem_ld16(tl, v);
#pragma unroll
  for (int k = 0; k < 8; k++) y[k] = v[k];
  return true;
}

// The fused stage (StageCfg::THREADS threads).  Per block: (1) interior by TMA, face-slab
// ghosts by threads; (2) FP64 form: primitives in place; (3) faces of all
// three directions at once on the first FACE_THREADS threads, two per grid
// line (faces 0-4 and 5-8), each sliding a window along its line so that
// every cell is loaded and every limited slope computed once; (4) per cell:
// flux differences x, y, z, the sources, the update and (last stage) the CFL
// bound.
template <bool MIXED, int LIM, bool HAS_B0, bool LRN, int FLX>
__global__ void __launch_bounds__(StageCfg<MIXED>::THREADS, (MIXED && !LRN) ? 2 : 1)
    k_stage(const __grid_constant__ StageArgs a) {
  using R = typename StageCfg<MIXED>::R;
  constexpr int STAGE_THREADS = StageCfg<MIXED>::THREADS;
  constexpr int NFC = StageCfg<MIXED>::NFC;
  // mixed form without the learned correction: the staged tile (tensor copies)
  constexpr bool MX = MIXED && !LRN;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* sT;                                         // tile: [8][1280] (generic) or the staged layout (MX)
  if constexpr (MX) {
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    sT = reinterpret_cast<R*>(smem_raw + pad);
  } else {
    sT = reinterpret_cast<R*>(smem_raw);
  }
  R* sF = sT + (MX ? MX_TILE : NV * NTILE);      // [3][9][576] face values
  // mixed learned kernel: the network runs fused, on the tensor cores
  constexpr bool LX = MIXED && LRN;
  LrnSmem* ls = nullptr;
  if constexpr (LX) {
    const uintptr_t e = reinterpret_cast<uintptr_t>(sF + 3 * StageCfg<MIXED>::NFC * NFACE);
    ls = reinterpret_cast<LrnSmem*>((e + 127) & ~uintptr_t(127));
  }
  const bool fused = LX && a.learned && a.kind < 3;
  uint32_t mphase = 0;
  bool mfail = false;  // a tensor-core wait ran out (uniform over the warp group, then the CTA)
  bool mpending = false;  // this thread's own wait ran out
  __shared__ uint64_t bar;
  __shared__ R sred[STAGE_THREADS / 32];

  const int tid = threadIdx.x;
  const PhysDev& ph = a.ph;
  R gamma, inv_gm1;
  if constexpr (MIXED) { gamma = ph.gammaf; inv_gm1 = ph.inv_gm1f; }
  else { gamma = ph.gamma; inv_gm1 = ph.inv_gm1; }
  constexpr bool has_b0 = HAS_B0;

  // this thread's line in the face phase
  const int fd = tid >> 7;                      // direction 0..2
  const int fline = (tid & 127) >> 1, fhalf = tid & 1;
  const int fta = fline & 7, ftb = fline >> 3;  // transverse coordinates (increasing axis order)
  const int fd1 = fd == 2 ? 0 : fd + 1, fd2 = fd == 0 ? 2 : fd - 1;
  const int fstride = fd == 0 ? 1 : (fd == 1 ? NC : NC * NC);
  const int fibase = fd == 0 ? (ftb * NC + fta) * NC : (fd == 1 ? ftb * NC * NC + fta : ftb * NC + fta);
  const int flo = NCELL + 2 * fd * 128 + 2 * (fta + NC * ftb), fhi = flo + 128;
  int rot[8];
  rot[0] = 0;
  rot[1] = (1 + fd) * NTILE;
  rot[2] = (1 + fd1) * NTILE;
  rot[3] = (1 + fd2) * NTILE;
  rot[4] = (4 + fd) * NTILE;
  rot[5] = (4 + fd1) * NTILE;
  rot[6] = (4 + fd2) * NTILE;
  rot[7] = 7 * NTILE;
  // flux store columns (un-rotated)
  R* const fcol = sF + fd * NFC * NFACE;

  if (tid == 0) mbar_init(&bar, 1);
  if constexpr (LX) {
    if (fused) {
      lrn_setup(*ls, a.mlp, tid, STAGE_THREADS);
      proxy_fence_smem();
      tc_fence_before();
    }
  }
  __syncthreads();
  if constexpr (LX) {
    if (fused) tc_fence_after();
  }
  uint32_t parity = 0;

  const int nitems = (a.nblocks + a.blocks_per_item - 1) / a.blocks_per_item;
  if constexpr (MX) {
    // the staged tile's copies run one block ahead: those of each block are
    // issued while the block before it is in its cell phase (which reads the
    // face values and global memory only); the first block's here
    const int b0 = blockIdx.x * a.blocks_per_item;
    if (tid == 0 && b0 < a.nblocks) mx_issue_copies(a, a.blocks[b0], b0, reinterpret_cast<float*>(sT), &bar);
  }
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int b_end = min(a.nblocks, (item + 1) * a.blocks_per_item);
    for (int blk = item * a.blocks_per_item; blk < b_end; blk++) {
      const BlockDev& B = a.blocks[blk];
      const GridDev& G = a.grids[B.grid];
      GhostCtx cx{&G, a.blocks, a.levmap, a.Uin, a.err};

      // 1. interior by TMA bulk copies (one per variable), ghosts by threads;
      //    the mixed plain kernel: the staged tile (tensor copies)
      if constexpr (MX) mx_fill_slabs(a, B, blk, reinterpret_cast<float*>(sT), tid, STAGE_THREADS);
      if (tid == 0 && !MX) {
        fence_proxy_async();
        // mixed form: the ghost slabs of faces at resolution changes come
        // precomputed, by bulk copies on the same barrier
        unsigned amask = 0;
        if constexpr (MIXED) {
          if (a.gbuf) {
#pragma unroll
            for (int f = 0; f < 6; f++)
              amask |= (B.ftype[f] == FACE_COARSER || B.ftype[f] == FACE_FINER ? 1u : 0u) << f;
          }
        }
        mbar_expect_tx(&bar, NV * NCELL * sizeof(R) + __popc(amask) * (NV * 128 * sizeof(float)));
        const R* src = MIXED ? reinterpret_cast<const R*>(a.Win) : reinterpret_cast<const R*>(a.Uin);
        src += static_cast<int64_t>(blk) * (NV * NCELL);
#pragma unroll
        for (int v = 0; v < NV; v++) bulk_g2s(sT + v * NTILE, src + v * NCELL, NCELL * sizeof(R), &bar);
        if constexpr (MIXED) {
          for (int f = 0; f < 6; f++) {
            if (!((amask >> f) & 1u)) continue;
            const float* g = a.gbuf + chk(B.rslot[f], 0, a.nslots) * GSLOT;
#pragma unroll
            for (int v = 0; v < NV; v++) bulk_g2s(sT + v * NTILE + NCELL + f * 128, g + v * 128, 128 * sizeof(float), &bar);
          }
        }
      }
      if (tid == 0) {
        // this CTA's next block: its interior on its way to L2 while this
        // block is computed, so that its bulk copies read L2, not HBM
        const int nblk = blk + 1 < b_end ? blk + 1 : (item + static_cast<int>(gridDim.x)) * a.blocks_per_item;
        if (nblk < a.nblocks) {
          const R* nsrc = MIXED ? reinterpret_cast<const R*>(a.Win) : reinterpret_cast<const R*>(a.Uin);
          prefetch_l2(nsrc + static_cast<int64_t>(nblk) * (NV * NCELL), NV * NCELL * sizeof(R));
        }
        // the FP64 states the cell phase reads, on their way to L2 meanwhile
        const int64_t boff = static_cast<int64_t>(blk) * (NV * NCELL);
        const bool reads_ubase = a.kind < 3 && !(MIXED && a.kind == 0 && !a.last && !a.write_u_all);
        if (reads_ubase) prefetch_l2(a.Ubase + boff, NV * NCELL * sizeof(double));
        if (MIXED && a.kind == 1) prefetch_l2(a.Uin + boff, NV * NCELL * sizeof(double));
      }
      if constexpr (MX) {
      } else if constexpr (MIXED) {
        fill_ghosts_block_mixed(a, cx, B, blk, sT, tid, STAGE_THREADS, false);
      } else {
        fill_ghosts_block<false, double>(a, cx, B, blk, sT, sF, tid, STAGE_THREADS);
      }
      if (!mbar_wait_bounded(&bar, parity, a.err)) mbar_wait_bounded(&bar, parity, a.err);
      parity ^= 1u;
      __syncthreads();

      // 2. FP64 form: primitives in place over the whole tile
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

      // 3. faces: reconstruction + Rusanov flux in the frame (d, d+1, d+2);
      //    corr = add the network's correction (learned form)
      auto faces = [&](const bool corr) {
          auto cidx = [&](int c) { return c < 0 ? flo + (c + 2) : (c >= NC ? fhi + (c - NC) : fibase + c * fstride); };
          const int f0 = fhalf ? 5 : 0, nf = fhalf ? 4 : 5;
          // window along the line.  Plain: the cell W0, the difference d = W0 - W-1
          // and the left state WL of the next face, W-1 + s-1 / 2 (each difference
          // and slope formed once).  Learned: the cells f-2..f, kept for the
          // network's inputs.
          R Wm1[8], W0[8], sm1[8];
          R Wm2[8];
          load_rot<R>(sT, rot, cidx(f0 - 2), Wm2);
          load_rot<R>(sT, rot, cidx(f0 - 1), Wm1);
          load_rot<R>(sT, rot, cidx(f0), W0);
          R d[8], WL[8];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            const R dm = Wm1[v] - Wm2[v];
            d[v] = W0[v] - Wm1[v];
            sm1[v] = limit_<R>(LIM, dm, d[v]);
            WL[v] = Wm1[v] + R(0.5) * sm1[v];
          }
          // fused network: every thread takes five steps (the CTA's 384 faces
          // of a step go through the network together); a lane of the upper
          // half has four faces and computes a throw-away fifth
          const int nsteps = (LX && fused && corr) ? 5 : nf;
#pragma unroll 1
          for (int k = 0; k < nsteps; k++) {
            const bool valid = k < nf;
            const int f = f0 + k;
            R Wp[8], WR[8], s0[8], dn[8];
            load_rot<R>(sT, rot, cidx(valid ? f + 1 : f), Wp);
#pragma unroll
            for (int v = 0; v < NV; v++) {
              dn[v] = Wp[v] - W0[v];
              s0[v] = limit_<R>(LIM, d[v], dn[v]);
              WR[v] = W0[v] - R(0.5) * s0[v];
            }
            R B0f[3] = {R(0), R(0), R(0)}, B0r[3];
            if constexpr (HAS_B0) {
              const int ci_ = fd == 0 ? f : fta, cj_ = fd == 1 ? f : (fd == 0 ? fta : ftb), ck_ = fd == 2 ? f : ftb;
              b0_face<R>(ph, fd, ci_, cj_, ck_, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, B0f);
            }
            B0r[0] = fd == 0 ? B0f[0] : (fd == 1 ? B0f[1] : B0f[2]);
            B0r[1] = fd1 == 0 ? B0f[0] : (fd1 == 1 ? B0f[1] : B0f[2]);
            B0r[2] = fd2 == 0 ? B0f[0] : (fd2 == 1 ? B0f[1] : B0f[2]);
            R FL[8], UL[8], FR[8], UR[8], unL, unR, cfL, cfR;
            phys_flux<R>(WL, B0r, gamma, inv_gm1, FL, UL, unL, cfL);
            phys_flux<R>(WR, B0r, gamma, inv_gm1, FR, UR, unR, cfR);
            R aL = Ops<R>::abs_(unL) + cfL, aR = Ops<R>::abs_(unR) + cfR;
            R cmax = aL > aR ? aL : aR;
            const int fi = chki(fline * 9 + (f < 9 ? f : 8), 0, NFACE);  // (f = 9: the throw-away step)
            R Fr[8];
            if constexpr (FLX == FLUX_HLL || FLX == FLUX_LINDE) {
              // HLL with S_L = min(unL - cfL, unR - cfR, 0), S_R = max(unL + cfL,
              // unR + cfR, 0):  F = F_L - S_L/(S_R - S_L) ((F_R - F_L) - S_R (U_R - U_L)),
              // which is F_L when every wave moves right (S_L = 0), F_R when every
              // wave moves left (S_R = 0), else the two-state HLL flux
              const R zero = R(0);
              R sl = unL - cfL < unR - cfR ? unL - cfL : unR - cfR;
              R sr = unL + cfL > unR + cfR ? unL + cfL : unR + cfR;
              sl = sl < zero ? sl : zero;
              sr = sr > zero ? sr : zero;
              const R den = sr - sl;
              const R kk = den > zero ? Ops<R>::div_(sl, den) : zero;
#pragma unroll
              for (int v = 0; v < NV; v++) Fr[v] = FL[v] - kk * ((FR[v] - FL[v]) - sr * (UR[v] - UL[v]));
              if constexpr (FLX == FLUX_LINDE) {
                // Linde: the contact wave restored, F -= delta alpha S_L S_R / (S_R - S_L) r,
                // alpha = minmod((rho_R - rho_L) - (p_R - p_L) / c^2, rho_R - rho_L),
                // delta = c / (c + |u_n|), r = (1, u, 0, |u|^2 / 2), means of the two
                // face states, c^2 = gamma p / rho
                const R rm = R(0.5) * (WL[0] + WR[0]), pm = R(0.5) * (WL[7] + WR[7]);
                const R um0 = R(0.5) * (WL[1] + WR[1]), um1 = R(0.5) * (WL[2] + WR[2]),
                        um2 = R(0.5) * (WL[3] + WR[3]);
                const R c2 = Ops<R>::div_(gamma * pm, rm), cs = Ops<R>::sqrt_(c2);
                const R alpha = minmod_<R>((WR[0] - WL[0]) - Ops<R>::div_(WR[7] - WL[7], c2), WR[0] - WL[0]);
                const R delta = Ops<R>::div_(cs, cs + Ops<R>::abs_(um0));
                const R q = den > zero ? Ops<R>::div_(delta * alpha * (sl * sr), den) : zero;
                Fr[0] -= q;
                Fr[1] -= q * um0;
                Fr[2] -= q * um1;
                Fr[3] -= q * um2;
                Fr[7] -= q * (R(0.5) * ((um0 * um0 + um1 * um1) + um2 * um2));
              }
            } else {
#pragma unroll
              for (int v = 0; v < NV; v++) Fr[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * cmax * (UR[v] - UL[v]);
            }
            if constexpr (LRN) {
              // network inputs: the 4 stencil cells f-2..f+1 and (WL + WR)/2 in
              // the face frame, scaled by rho_ref = mean stencil density and
              // c_ref = cmax (u / c_ref, B / (sqrt(rho_ref) c_ref), p / (rho_ref c_ref^2))
              const int64_t gface = (static_cast<int64_t>(blk) * 3 + fd) * NFACE + fi;
              const R rho_ref = R(0.25) * (((Wm2[0] + Wm1[0]) + W0[0]) + Wp[0]);
              const R c_ref = cmax;
              const R sq = Ops<R>::sqrt_(rho_ref);
              if (a.kind >= 3) {
                const R ir = Ops<R>::div_(R(1), rho_ref), ic = Ops<R>::div_(R(1), c_ref);
                const R ib = Ops<R>::div_(R(1), sq * c_ref), ip = Ops<R>::div_(R(1), rho_ref * c_ref * c_ref);
                float xin[40];
#pragma unroll
                for (int sidx = 0; sidx < 5; sidx++) {
                  const R* Wsrc = sidx == 0 ? Wm2 : (sidx == 1 ? Wm1 : (sidx == 2 ? W0 : Wp));
                  R wv[8];
#pragma unroll
                  for (int v = 0; v < NV; v++) wv[v] = sidx < 4 ? Wsrc[v] : R(0.5) * (WL[v] + WR[v]);
                  xin[8 * sidx + 0] = static_cast<float>(wv[0] * ir);
#pragma unroll
                  for (int c = 1; c < 4; c++) xin[8 * sidx + c] = static_cast<float>(wv[c] * ic);
#pragma unroll
                  for (int c = 4; c < 7; c++) xin[8 * sidx + c] = static_cast<float>(wv[c] * ib);
                  xin[8 * sidx + 7] = static_cast<float>(wv[7] * ip);
                }
                if (a.kind == 3) {
                  uint32_t* dst = a.Xb + gface * 24;
#pragma unroll
                  for (int q = 0; q < 20; q++) {
                    __nv_bfloat162 v2 = __floats2bfloat162_rn(xin[2 * q], xin[2 * q + 1]);
                    dst[q] = *reinterpret_cast<uint32_t*>(&v2);
                  }
#pragma unroll
                  for (int q = 20; q < 24; q++) dst[q] = 0u;
                } else {
                  if (a.Xf) {
                    float* dst = a.Xf + gface * 40;
#pragma unroll
                    for (int q = 0; q < 40; q++) dst[q] = xin[q];
                  }
                  double* fo = a.Fd + gface * 10;
                  fo[8] = rho_ref;
                  fo[9] = c_ref;
                  fo[0] = Fr[0];
                  fo[1 + fd] = Fr[1];
                  fo[1 + fd1] = Fr[2];
                  fo[1 + fd2] = Fr[3];
                  fo[4 + fd] = Fr[4];
                  fo[4 + fd1] = Fr[5];
                  fo[4 + fd2] = Fr[6];
                  fo[7] = Fr[7];
                }
              } else if (LX && a.learned && corr) {
                // the network on the tensor cores, with the CTA's other faces
                // of this step; inputs as for kind 3
                const R ir = Ops<R>::div_(R(1), rho_ref), ic = Ops<R>::div_(R(1), c_ref);
                const R ib = Ops<R>::div_(R(1), sq * c_ref), ip = Ops<R>::div_(R(1), rho_ref * c_ref * c_ref);
                float xin[40];
#pragma unroll
                for (int sidx = 0; sidx < 5; sidx++) {
                  const R* Wsrc = sidx == 0 ? Wm2 : (sidx == 1 ? Wm1 : (sidx == 2 ? W0 : Wp));
                  R wv[8];
#pragma unroll
                  for (int v = 0; v < NV; v++) wv[v] = sidx < 4 ? Wsrc[v] : R(0.5) * (WL[v] + WR[v]);
                  xin[8 * sidx + 0] = static_cast<float>(wv[0] * ir);
#pragma unroll
                  for (int c = 1; c < 4; c++) xin[8 * sidx + c] = static_cast<float>(wv[c] * ic);
#pragma unroll
                  for (int c = 4; c < 7; c++) xin[8 * sidx + c] = static_cast<float>(wv[c] * ib);
                  xin[8 * sidx + 7] = static_cast<float>(wv[7] * ip);
                }
                uint4 xrow[6];
#pragma unroll
                for (int q = 0; q < 5; q++)
                  xrow[q] = make_uint4(pack_bf16(xin[8 * q], xin[8 * q + 1]), pack_bf16(xin[8 * q + 2], xin[8 * q + 3]),
                                       pack_bf16(xin[8 * q + 4], xin[8 * q + 5]),
                                       pack_bf16(xin[8 * q + 6], xin[8 * q + 7]));
                xrow[5] = make_uint4(0u, 0u, 0u, 0u);
                float yv[8];
                if (!lrn_network(*ls, xrow, yv, tid, mphase, mpending, a.err)) {
                  mfail = true;
                  break;
                }
                const R sc0 = rho_ref * c_ref, sc1 = rho_ref * c_ref * c_ref, sc4 = sq * c_ref * c_ref;
                const R sc7 = rho_ref * c_ref * c_ref * c_ref;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                  const R sc = v == 0 ? sc0 : (v < 4 ? sc1 : (v < 7 ? sc4 : sc7));
                  R dF = R(yv[v]) * sc;
                  const R lim = Ops<R>::abs_(R(0.5) * cmax * (UR[v] - UL[v]));
                  dF = dF > lim ? lim : dF;
                  dF = dF < -lim ? -lim : dF;
                  Fr[v] = Fr[v] + dF;
                }
              } else if (a.learned && corr) {
                // correction back in flux units, clipped to the Rusanov dissipation
                const float* yv = a.Y + gface * 8;
                const R sc0 = rho_ref * c_ref, sc1 = rho_ref * c_ref * c_ref, sc4 = sq * c_ref * c_ref;
                const R sc7 = rho_ref * c_ref * c_ref * c_ref;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                  const R sc = v == 0 ? sc0 : (v < 4 ? sc1 : (v < 7 ? sc4 : sc7));
                  R dF = R(yv[v]) * sc;
                  const R lim = Ops<R>::abs_(R(0.5) * cmax * (UR[v] - UL[v]));
                  dF = dF > lim ? lim : dF;
                  dF = dF < -lim ? -lim : dF;
                  Fr[v] = Fr[v] + dF;
                }
              }
            }
            if (!valid) continue;  // the throw-away fifth step
            const R bnf = R(0.5) * (WL[4] + WR[4]);  // face-averaged normal B1 (Powell)
#pragma unroll
            for (int v = 0; v < NV; v++) {
              if constexpr (LRN) {
                Wm2[v] = Wm1[v];
                Wm1[v] = W0[v];
              }
              WL[v] = W0[v] + R(0.5) * s0[v];
              W0[v] = Wp[v];
              d[v] = dn[v];
            }
            if (a.kind >= 3) continue;
            fcol[0 * NFACE + fi] = Fr[0];
            fcol[(1 + fd) * NFACE + fi] = Fr[1];
            fcol[(1 + fd1) * NFACE + fi] = Fr[2];
            fcol[(1 + fd2) * NFACE + fi] = Fr[3];
            fcol[(4 + fd) * NFACE + fi] = Fr[4];
            fcol[(4 + fd1) * NFACE + fi] = Fr[5];
            fcol[(4 + fd2) * NFACE + fi] = Fr[6];
            fcol[7 * NFACE + fi] = Fr[7];
            fcol[8 * NFACE + fi] = bnf;
            // refluxing: the block-face fluxes of faces at resolution changes
            if (a.freg && (f == 0 || f == NC)) {
              const int sl = chki(B.rslot[2 * fd + (f == NC ? 1 : 0)], -1, a.nslots);
              if (sl >= 0) {
                double* o = a.freg + (static_cast<int64_t>(sl) * 64 + fta * NC + ftb) * NV;
                double Fd[8];
#pragma unroll
                for (int v = 0; v < NV; v++) {
                  if constexpr (MIXED) Fd[v] = f2d_int(Fr[v]);
                  else Fd[v] = Fr[v];
                }
                o[0] = Fd[0];
                o[1 + fd] = Fd[1];
                o[1 + fd1] = Fd[2];
                o[1 + fd2] = Fd[3];
                o[4 + fd] = Fd[4];
                o[4 + fd1] = Fd[5];
                o[4 + fd2] = Fd[6];
                o[7] = Fd[7];
              }
            }
          }
      };
      // 4. per cell: flux differences, sources, update, CFL bound.  commit =
      //    false only checks the update (learned form): returns whether this
      //    thread met a non-physical cell, writes nothing
      auto cells = [&](const bool commit, auto fast_c) -> bool {
        // FAST (compile time): kind 0, no local time steps, no body cell in the
        // block.  The general form keeps those paths, whose FP64 work the
        // compiler would otherwise issue predicated off for every cell (GB300
        // runs FP64 at 1/64 of the FP32 rate, so even dead FP64 instructions
        // cost).
        constexpr bool FAST = decltype(fast_c)::value;
        const int kind = FAST ? 0 : a.kind;
        double* const dtc = FAST ? nullptr : a.dtc;
        const bool blk_body = FAST ? false : B.body != 0;
        // the packed mixed face phase stores doubled face values
        constexpr R FS = (MIXED && !LRN) ? R(0.5) : R(1);
        const R fidx0 = FS * idx0, fidx1 = FS * idx1, fidx2 = FS * idx2;
        bool any_bad = false;
        R smax_loc = R(0);
        const double cdt_blk = a.beta * a.dt[B.grid];
        // mixed form, first stage of the midpoint scheme: U* only feeds the
        // second stage's FP32 primitives, so W* = W^n + the increment, in FP32
        // (the FP64 state is read and accumulated in the last stage only)
        const bool light = MIXED && kind == 0 && !a.last && !a.write_u_all;
        const float c32_blk = d2f_int(cdt_blk);
        for (int c = tid; c < NCELL; c += STAGE_THREADS) {
          // local time stepping: this cell's own dt
          const double cdt = dtc ? a.beta * dtc[static_cast<int64_t>(blk) * NCELL + c] : cdt_blk;
          const float c32 = dtc ? d2f_int(cdt) : c32_blk;
          const int ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;
          // face indices (line * 9 + position) of the low faces in x, y, z
          const int tx = chki((ck * NC + cj) * 9 + ci, 0, NFACE - 1);
          const int ty = chki((ck * NC + ci) * 9 + cj, 0, NFACE - 1);
          const int tz = chki((cj * NC + ci) * 9 + ck, 0, NFACE - 1);
          const R* Fx = sF;
          const R* Fy = sF + NFC * NFACE;
          const R* Fz = sF + 2 * NFC * NFACE;
          R res[8];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            // the mixed plain kernel's face values are in the face frame (frot)
            const int vx = MX ? frot(v, 0) : v, vy = MX ? frot(v, 1) : v, vz = MX ? frot(v, 2) : v;
            R r = -((Fx[vx * NFACE + tx + 1] - Fx[vx * NFACE + tx]) * fidx0);
            r = r - (Fy[vy * NFACE + ty + 1] - Fy[vy * NFACE + ty]) * fidx1;
            r = r - (Fz[vz * NFACE + tz + 1] - Fz[vz * NFACE + tz]) * fidx2;
            res[v] = r;
          }
          const R divb = ((Fx[8 * NFACE + tx + 1] - Fx[8 * NFACE + tx]) * fidx0 +
                          (Fy[8 * NFACE + ty + 1] - Fy[8 * NFACE + ty]) * fidx1) +
                         (Fz[8 * NFACE + tz + 1] - Fz[8 * NFACE + tz]) * fidx2;
          bool in_body = false;
          if (blk_body) {  // FP64, the same centre formula as the host and the oracle
            double x = G.lo[0] + ((static_cast<double>(gb0) + ci) + 0.5) * G.dx[lev][0];
            double y = G.lo[1] + ((static_cast<double>(gb1) + cj) + 0.5) * G.dx[lev][1];
            double z = G.lo[2] + ((static_cast<double>(gb2) + ck) + 0.5) * G.dx[lev][2];
            in_body = (x * x + y * y + z * z) < G.body_r * G.body_r;
          }
          R Wc[8];
          if constexpr (MX) {
            const int cs = c ^ (((c >> 5) & 1) << 2);  // the interior's swizzle (j >= 4: halves exchanged)
#pragma unroll
            for (int v = 0; v < NV; v++) Wc[v] = sT[v * NCELL + cs];
          } else {
#pragma unroll
            for (int v = 0; v < NV; v++) Wc[v] = sT[v * NTILE + c];
          }
          R B0c[3] = {R(0), R(0), R(0)};
          R S[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
          if constexpr (HAS_B0) b0_face<R>(ph, -1, ci, cj, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, B0c);
          if (ph.powell) {
            R ub1 = Wc[1] * Wc[4] + Wc[2] * Wc[5] + Wc[3] * Wc[6];
#pragma unroll
            for (int e = 0; e < 3; e++) {
              S[1 + e] = -divb * (B0c[e] + Wc[4 + e]);
              S[4 + e] = -divb * Wc[1 + e];
            }
            S[7] = -divb * ub1;
          }
          if constexpr (HAS_B0) {
            // split-field correction from the face-centre B0 of the six faces:
            // S_m += -B1 (div B0)_h + B1 x (curl B0)_h
            R xm[3], xp[3], ym[3], yp[3], zm[3], zp[3];
            b0_face<R>(ph, 0, ci, cj, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, xm);
            b0_face<R>(ph, 0, ci + 1, cj, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, xp);
            b0_face<R>(ph, 1, ci, cj, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, ym);
            b0_face<R>(ph, 1, ci, cj + 1, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, yp);
            b0_face<R>(ph, 2, ci, cj, ck, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, zm);
            b0_face<R>(ph, 2, ci, cj, ck + 1, gb0, gb1, gb2, lor0, lor1, lor2, dxr0, dxr1, dxr2, zp);
            R divb0 = ((xp[0] - xm[0]) * idx0 + (yp[1] - ym[1]) * idx1) + (zp[2] - zm[2]) * idx2;
            R cu0 = (yp[2] - ym[2]) * idx1 - (zp[1] - zm[1]) * idx2;
            R cu1 = (zp[0] - zm[0]) * idx2 - (xp[2] - xm[2]) * idx0;
            R cu2 = (xp[1] - xm[1]) * idx0 - (yp[0] - ym[0]) * idx1;
            R b1x = Wc[4], b1y = Wc[5], b1z = Wc[6];
            S[1] = (S[1] - b1x * divb0) + (b1y * cu2 - b1z * cu1);
            S[2] = (S[2] - b1y * divb0) + (b1z * cu0 - b1x * cu2);
            S[3] = (S[3] - b1z * divb0) + (b1x * cu1 - b1y * cu0);
          }
          const int64_t base = static_cast<int64_t>(blk) * (NV * NCELL) + c;
          if constexpr (MIXED) {
            if (light) {
              float dU[8], Wl[8];
#pragma unroll
              for (int v = 0; v < NV; v++) dU[v] = c32 * (res[v] + S[v]);
              prim_increment(Wc, dU, ph.gm1f, Wl);
              if (in_body) prim_mixed(G.Ubody, ph.gm1f, Wl);
              bool badl = !(Wl[0] > 0.f) || !(Wl[7] > 0.f);
#pragma unroll
              for (int v = 0; v < NV; v++) badl |= !finite_f(Wl[v]);
              if (badl && !in_body) {
                any_bad = true;
                if (commit) {
                  atomicOr(&a.err[0], ERR_NONPHYSICAL);
                  atomicMin(&a.err[1], blk);
                }
              }
              if (!commit) continue;
#pragma unroll
              for (int v = 0; v < NV; v++) a.Wout[base + v * NCELL] = Wl[v];
              continue;
            }
          }
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
            if (kind == 0) o = fma(cdt, rd, ub);
            else o = 0.5 * ub + 0.5 * fma(cdt, rd, a.Uin[base + v * NCELL]);
            if (kind == 2) o = rd;  // residual only (debug view)
            Uo[v] = o;
          }
          if (in_body) {  // a branch, not a select: no loads of the body state elsewhere
#pragma unroll
            for (int v = 0; v < NV; v++) Uo[v] = kind == 2 ? 0.0 : G.Ubody[v];
          }
#pragma unroll
          for (int v = 0; v < NV; v++) bad |= !finite_d(Uo[v]);
          if (kind != 2) bad |= !positive_d(Uo[0]);
          R Wn[8];
          const bool need_w = MIXED || a.last || !commit;
          if (need_w && kind != 2) {
            if constexpr (MIXED) {
              double p64;
              prim_mixed(Uo, ph.gm1f, Wn, &p64);
              bad |= !positive_d(p64);
            } else {
              prim64(Uo, ph.gm1, Wn);
              bad |= !positive_d(Wn[7]);
            }
          }
          if (bad && !in_body && kind != 2) {
            any_bad = true;
            if (commit) {
              atomicOr(&a.err[0], ERR_NONPHYSICAL);
              atomicMin(&a.err[1], blk);
            }
          }
          if (!commit) continue;
          const bool write_u = !MIXED || a.last || a.write_u_all;
          if (write_u || kind == 2) {
#pragma unroll
            for (int v = 0; v < NV; v++) a.Uout[base + v * NCELL] = Uo[v];
          }
          if constexpr (MIXED) {
            if (kind != 2) {
#pragma unroll
              for (int v = 0; v < NV; v++) a.Wout[base + v * NCELL] = Wn[v];
            }
          }
          // CFL bound of the new state: sum_d (|u_d| + c_f,d) / dx_d (cells that
          // refluxing corrects afterwards are bounded by the correction kernel)
          const bool refl = a.freg && ((ci == 0 && B.ftype[0] == FACE_FINER) || (ci == NC - 1 && B.ftype[1] == FACE_FINER) ||
                                       (cj == 0 && B.ftype[2] == FACE_FINER) || (cj == NC - 1 && B.ftype[3] == FACE_FINER) ||
                                       (ck == 0 && B.ftype[4] == FACE_FINER) || (ck == NC - 1 && B.ftype[5] == FACE_FINER));
          if (a.last && !in_body && kind != 2 && !refl) {
            R Bt[3] = {B0c[0] + Wn[4], B0c[1] + Wn[5], B0c[2] + Wn[6]};
            R sacc = R(0);
#pragma unroll
            for (int e = 0; e < 3; e++) {
              R bn = Bt[e], bt1 = Bt[(e + 1) % 3], bt2 = Bt[(e + 2) % 3];
              R cf;
              if constexpr (MIXED) {
                cf = fast_speed_n<R>(gamma, Wn[0], Wn[7], bn, bt1, bt2);
                sacc = sacc + (Ops<R>::abs_(Wn[1 + e]) + cf) * (e == 0 ? idx0 : (e == 1 ? idx1 : idx2));
              } else {
                cf = fast_speed_exact(ph.gamma, Wn[0], Wn[7], bn, bt1, bt2);
                sacc = sacc + (Ops<R>::abs_(Wn[1 + e]) + cf) / (e == 0 ? dxr0 : (e == 1 ? dxr1 : dxr2));
              }
            }
            smax_loc = sacc > smax_loc ? sacc : smax_loc;
            if (dtc) {
              double sd;
              if constexpr (MIXED) sd = f2d_int(sacc);
              else sd = sacc;
              dtc[static_cast<int64_t>(blk) * NCELL + c] = a.cfl / sd;
            }
          } else if (a.last && dtc && kind != 2 && in_body) {
            dtc[static_cast<int64_t>(blk) * NCELL + c] = 0.0;  // body cell
          }
        }
        if (commit && a.last && kind != 2) {
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
        return any_bad;
      };

      if constexpr (MX) {
        // one direction per warp group (fd is warp-uniform)
        if (tid < FACE_THREADS) {
          faces_mx<LIM, HAS_B0, FLX>(fd, a, B, sT, sF, fline, fhalf, gamma, inv_gm1, gb0, gb1, gb2, lor0, lor1, lor2,
                                     dxr0, dxr1, dxr2);
        }
      } else {
        if (tid < FACE_THREADS) faces(true);
      }
      // a tensor-core wait ran out in some warp group: the error is flagged, stop
      if (__syncthreads_or(mfail)) {
        mfail = true;
        break;
      }
      // the staged tile's next block (its copies go out once this block's
      // cell phase has read what it needs from the tile)
      const int nblk = blk + 1 < b_end ? blk + 1 : (item + static_cast<int>(gridDim.x)) * a.blocks_per_item;
      // issuer: a thread of a warp with no cell work in the packed cell phase
      // (threads 256-383), so that its wait for the next block's table entry
      // delays no cell's update
      auto issue_next = [&](int issuer) {
        if constexpr (MX) {
          if (tid == issuer && nblk < a.nblocks)
            mx_issue_copies(a, a.blocks[nblk], nblk, reinterpret_cast<float*>(sT), &bar);
        }
      };
      if (a.kind >= 3) continue;  // features / dumps only
      const bool fast = a.kind == 0 && !a.dtc && !B.body;
      if constexpr (MX && !HAS_B0) {
        if (fast) {
          // the common case: two cells per thread, packed; the pair's
          // primitives from the tile, then the tile is free for the next block
          float2 Wc[8];
          if (!a.last && !a.write_u_all) cells_mx_pair_w(reinterpret_cast<const float*>(sT), tid, Wc);
          __syncthreads();
          issue_next(NCELL / 2);
          const float m = cells_mx_pair(a, G, B, blk, Wc, sF, tid, 0.5f * idx0, 0.5f * idx1, 0.5f * idx2, idx0,
                                        idx1, idx2, gamma);
          if (a.last) {
            float mm = m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
            if ((tid & 31) == 0) sred[tid >> 5] = mm;
            __syncthreads();
            if (tid == 0) {
              float mx = 0.f;
              for (int w = 0; w < STAGE_THREADS / 32; w++) mx = fmaxf(mx, sred[w]);
              const double md = f2d_int(mx);
              if (md > 0.0) atomicMax(&a.smax_next[B.grid], static_cast<unsigned long long>(__double_as_longlong(md)));
            }
          }
          __syncthreads();
          continue;
        }
      }
      auto run_cells = [&](const bool commit) -> bool {
        return fast ? cells(commit, std::true_type{}) : cells(commit, std::false_type{});
      };
      if constexpr (LRN) {
        // fallback of the learned form: a block whose learned update leaves a
        // non-physical cell (rho <= 0, p <= 0 or not finite) is recomputed
        // with the plain Rusanov flux
        if (a.learned && a.kind < 2) {
          if (__syncthreads_or(run_cells(false))) {
            if (tid < FACE_THREADS) faces(false);
            __syncthreads();
            if (tid == 0) atomicAdd(&a.err[2], 1);
          }
        }
      }
      run_cells(true);
      __syncthreads();
      issue_next(0);
    }
    if (mfail) break;
  }
  if constexpr (LX) {
    if (fused) lrn_teardown(*ls, tid, mpending, mphase, a.err);
  }
}

}  // namespace batsk
