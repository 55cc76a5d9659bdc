/*
 * oracle.c -- plain, slow, FP64 CPU reference for one explicit stage of the
 * ideal-MHD finite-volume update on a 2:1 block-adaptive grid of 8^3-cell
 * blocks with 2 ghost layers (the single-GPU solver of the BATSRUS GPU paper,
 * arXiv 2501.06717, Section 3, Algorithms 1-2, Eqs. 1-5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes, step by step, in the order of Algorithm 1 (face values,
 * face fluxes, sources, update) followed by the ghost fill:
 *
 *  - State per cell U = (rho, rho u, B1, e1), B = B0 + B1 (split field),
 *    mu0 = 1 (Section 5.1), e1 = p/(gamma-1) + rho u^2/2 + B1^2/2 (Eq. 5 with
 *    B -> B1 when B0 is split off).
 *  - Ghost cells (Section 4.1; copy / restriction / prolongation, Section 4.2)
 *    are defined by point location: a ghost centre is mapped through the
 *    domain boundary conditions, the leaf containing it is found, and its
 *    value is a copy (same level), the mean of the 8 finer children
 *    (restriction) or the coarse value plus minmod-limited linear slopes of
 *    the conservative variables (prolongation).
 *  - Primitive recovery p = (gamma-1)(e1 - m.u/2 - B1.B1/2) (Eq. 5).
 *  - Limited linear reconstruction of primitives (minmod or MC).
 *  - Rusanov flux of the split-field ideal-MHD fluxes of Eqs. 1-4 (the HLL
 *    two-state flux as an option).
 *  - Powell 8-wave source terms (right-hand sides of Eqs. 2-4) and the
 *    split-field B0 correction.
 *  - Conservative update; two-stage second-order time stepping (Section 5.2
 *    names a "two-stage second-order" scheme; read here as the midpoint
 *    predictor-corrector, with SSP-RK2 as an option).
 *  - Global CFL time step per grid.
 *
 * Every point the paper leaves open is a stated reading; the list lives in
 * the design notes and in the comments next to each formula below.
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared oracle.c -lm
 * (no FMA contraction, so the arithmetic is the order written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 8          /* conserved variables */
#define NC 8          /* cells per block per axis */
#define NG 2          /* ghost layers */
#define NT 12         /* padded tile width NC + 2 NG */
#define NCELL 512     /* cells per block */
#define MAXLEV 14

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2 };
enum { LIM_MINMOD = 0, LIM_MC = 1, LIM_NONE = 2 };
enum { RK_MIDPOINT = 0, RK_SSP2 = 1, RK_EULER = 2 };
enum { B0_NONE = 0, B0_UNIFORM = 1, B0_DIPOLE = 2, B0_LINEAR = 3 };
enum { FLUX_RUSANOV = 0, FLUX_HLL = 1, FLUX_LINDE = 2 };
enum { OR_OK = 0, OR_EINVAL = -1, OR_EUNBALANCED = -2, OR_ENOMEM = -3 };
enum { GT_INTERIOR = 0, GT_COPY = 1, GT_RESTRICT = 2, GT_PROLONG = 3, GT_INFLOW = 4 };

/* Learned flux correction: a 40 -> 64 -> 64 -> 8 MLP with GELU. */
#define MLP_IN 40
#define MLP_H 64
#define MLP_OUT 8
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT)

typedef struct {
  double lo[3], hi[3];
  int32_t root[3];
  int32_t n_leaves;
  const int32_t* leaves; /* n_leaves x 4: level, i, j, k (block coords at that level) */
  int32_t bc[6];         /* -x, +x, -y, +y, -z, +z */
  double inflow[8];      /* primitive rho, u(3), B1(3), p */
  double body_r;         /* cells with centre radius < body_r are held fixed */
  double body[8];        /* primitive body state */
  double gamma;
  int32_t limiter, rk, b0, powell;
  double b0_param[12];   /* UNIFORM: B0; DIPOLE: moment m; LINEAR: B0c(3) + G(3x3 row-major) */
  int32_t learned;       /* 1 = add the MLP flux correction */
  int32_t no_fallback;   /* test switch: 1 keeps a learned block update even where it is non-physical */
  const double* mlp;     /* MLP_NPARAM weights (W1,b1,W2,b2,W3,b3), row-major [out][in] */
  int32_t local_dt;      /* 1 = local time stepping: each cell its own dt (steady-state runs) */
  int32_t reflux;        /* 1 = conservative flux correction at resolution changes */
  int32_t flux;          /* FLUX_RUSANOV, FLUX_HLL (two-state HLL, Davis wave-speed bounds) or
                            FLUX_LINDE (HLL with the contact wave restored) */
  int32_t learned_last_only; /* learned form: 1 = the correction in the last stage of a step only (the
                              * stage whose fluxes enter U^{n+1}, where the training target is defined) */
} or_desc;

typedef struct {
  const or_desc* d;
  int nb, maxlev;
  long ncell[MAXLEV + 1][3];  /* cells per axis at each level */
  long nblk[MAXLEV + 1][3];   /* block positions per axis at each level */
  int32_t* map[MAXLEV + 1];   /* block position -> leaf id, or -1 */
  double dx[MAXLEV + 1][3];
  double Uinflow[NV], Ubody[NV];
  const double* U;            /* state [NV][nb][NCELL] being read */
  long deep_prolong;          /* prolongations that needed a coarser-than-one-level source */
} grid_t;

/* ------------------------------------------------------------------------ */
/* State conversions (Eq. 5 with the split field).                           */

static void cons_from_prim(double gamma, const double W[NV], double U[NV]) {
  double rho = W[0];
  double usq = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  double bsq = W[4] * W[4] + W[5] * W[5] + W[6] * W[6];
  U[0] = rho;
  U[1] = rho * W[1];
  U[2] = rho * W[2];
  U[3] = rho * W[3];
  U[4] = W[4];
  U[5] = W[5];
  U[6] = W[6];
  U[7] = W[7] * (1.0 / (gamma - 1.0)) + 0.5 * rho * usq + 0.5 * bsq;
}

static void prim_from_cons(double gamma, const double U[NV], double W[NV]) {
  double rho = U[0];
  double ux = U[1] / rho, uy = U[2] / rho, uz = U[3] / rho;
  double ke = 0.5 * (U[1] * ux + U[2] * uy + U[3] * uz);
  double me = 0.5 * (U[4] * U[4] + U[5] * U[5] + U[6] * U[6]);
  W[0] = rho;
  W[1] = ux;
  W[2] = uy;
  W[3] = uz;
  W[4] = U[4];
  W[5] = U[5];
  W[6] = U[6];
  W[7] = (gamma - 1.0) * (U[7] - ke - me);
}

/* ------------------------------------------------------------------------ */
/* Background field B0 (split field B = B0 + B1), evaluated analytically.    */

static void b0_at(const or_desc* d, const double x[3], double B0[3]) {
  const double* q = d->b0_param;
  switch (d->b0) {
    case B0_UNIFORM:
      B0[0] = q[0]; B0[1] = q[1]; B0[2] = q[2];
      return;
    case B0_DIPOLE: {
      /* point dipole with moment m at the origin: (3 (m.r) r - m r^2) / r^5 */
      double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      double r = sqrt(r2);
      double inv_r5 = 1.0 / (r2 * r2 * r);
      double mr = q[0] * x[0] + q[1] * x[1] + q[2] * x[2];
      for (int c = 0; c < 3; c++) B0[c] = (3.0 * mr * x[c] - q[c] * r2) * inv_r5;
      return;
    }
    case B0_LINEAR:
      for (int c = 0; c < 3; c++)
        B0[c] = q[c] + q[3 + 3 * c] * x[0] + q[4 + 3 * c] * x[1] + q[5 + 3 * c] * x[2];
      return;
    default:
      B0[0] = B0[1] = B0[2] = 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Grid: level maps for point location, validation, 2:1 balance check.      */

static void grid_free(grid_t* G) {
  for (int l = 0; l <= MAXLEV; l++) { free(G->map[l]); G->map[l] = NULL; }
}

static long map_index(const grid_t* G, int lev, long bi, long bj, long bk) {
  return (bk * G->nblk[lev][1] + bj) * G->nblk[lev][0] + bi;
}

/* Find the leaf containing cell g of level lev (g inside the domain).
 * Returns the leaf id and sets *leaf_lev; returns -1 with *leaf_lev = lev+1
 * when the cell's region is covered by finer leaves. */
static int locate(const grid_t* G, int lev, const long g[3], int* leaf_lev) {
  int top = lev < G->maxlev ? lev : G->maxlev;
  for (int l = top; l >= 0; l--) {
    int sh = lev - l;
    long bi = (g[0] >> sh) / NC, bj = (g[1] >> sh) / NC, bk = (g[2] >> sh) / NC;
    int32_t id = G->map[l][map_index(G, l, bi, bj, bk)];
    if (id >= 0) { *leaf_lev = l; return id; }
  }
  *leaf_lev = lev + 1;
  return -1;
}

/* Map cell g of level lev through the boundary conditions, axis x then y then
 * z: periodic wraps, outflow clamps to the first interior cell (zero
 * gradient), inflow returns 1 (the fixed inflow state applies). */
static int apply_bc(const grid_t* G, int lev, long g[3]) {
  for (int a = 0; a < 3; a++) {
    long n = G->ncell[lev][a];
    if (g[a] >= 0 && g[a] < n) continue;
    int side = g[a] < 0 ? 0 : 1;
    int bc = G->d->bc[2 * a + side];
    if (bc == BC_PERIODIC) g[a] = ((g[a] % n) + n) % n;
    else if (bc == BC_OUTFLOW) g[a] = side ? n - 1 : 0;
    else return 1;
  }
  return 0;
}

static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

/* Value of the conservative state at cell g of level lev (point location).
 * Copy at the same level; restriction = mean of the 8 children summed
 * pairwise; prolongation = coarse value + 0.25 * (+-1) * minmod slope per
 * axis, the slopes being undivided differences of coarse-level values. */
static void value_at(grid_t* G, int lev, const long g0[3], double out[NV]) {
  long g[3] = {g0[0], g0[1], g0[2]};
  if (apply_bc(G, lev, g)) { memcpy(out, G->Uinflow, sizeof(double) * NV); return; }
  int ll;
  int id = locate(G, lev, g, &ll);
  if (id >= 0 && ll == lev) {
    const int32_t* L = G->d->leaves + 4 * id;
    long li = g[0] - (long)L[1] * NC, lj = g[1] - (long)L[2] * NC, lk = g[2] - (long)L[3] * NC;
    long c = (lk * NC + lj) * NC + li;
    for (int v = 0; v < NV; v++) out[v] = G->U[((long)v * G->nb + id) * NCELL + c];
    return;
  }
  if (id < 0) { /* restriction from the 8 children at lev+1 */
    double ch[8][NV];
    for (int o = 0; o < 8; o++) {
      long gc[3] = {2 * g[0] + (o & 1), 2 * g[1] + ((o >> 1) & 1), 2 * g[2] + ((o >> 2) & 1)};
      value_at(G, lev + 1, gc, ch[o]);
    }
    for (int v = 0; v < NV; v++) {
      double s = ((ch[0][v] + ch[1][v]) + (ch[2][v] + ch[3][v])) +
                 ((ch[4][v] + ch[5][v]) + (ch[6][v] + ch[7][v]));
      out[v] = 0.125 * s;
    }
    return;
  }
  /* prolongation from level lev-1 */
  if (ll < lev - 1) G->deep_prolong++;
  long gc[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
  double Vc[NV], slope[3][NV];
  value_at(G, lev - 1, gc, Vc);
  for (int a = 0; a < 3; a++) {
    double Vm[NV], Vp[NV];
    long gm[3] = {gc[0], gc[1], gc[2]}, gp[3] = {gc[0], gc[1], gc[2]};
    gm[a] -= 1;
    gp[a] += 1;
    value_at(G, lev - 1, gm, Vm);
    value_at(G, lev - 1, gp, Vp);
    for (int v = 0; v < NV; v++) slope[a][v] = minmod(Vc[v] - Vm[v], Vp[v] - Vc[v]);
  }
  double sx = (g[0] & 1) ? 0.25 : -0.25, sy = (g[1] & 1) ? 0.25 : -0.25, sz = (g[2] & 1) ? 0.25 : -0.25;
  for (int v = 0; v < NV; v++) out[v] = Vc[v] + sx * slope[0][v] + sy * slope[1][v] + sz * slope[2][v];
}

/* Classify a ghost cell (for message-size and recipe tests). */
static int ghost_class(const grid_t* G, int lev, const long g0[3], int32_t* src) {
  long g[3] = {g0[0], g0[1], g0[2]};
  if (apply_bc(G, lev, g)) { *src = -1; return GT_INFLOW; }
  int ll;
  int id = locate(G, lev, g, &ll);
  if (id >= 0 && ll == lev) { *src = id; return GT_COPY; }
  if (id < 0) {
    long gc[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
    int l2;
    *src = locate(G, lev + 1, gc, &l2);
    return GT_RESTRICT;
  }
  *src = id;
  return GT_PROLONG;
}

static int grid_init(grid_t* G, const or_desc* d, double dummy_unused) {
  (void)dummy_unused;
  memset(G, 0, sizeof(*G));
  G->d = d;
  if (!d || !d->leaves || d->n_leaves <= 0) return OR_EINVAL;
  if (!(d->gamma > 1.0)) return OR_EINVAL;
  if (d->flux < FLUX_RUSANOV || d->flux > FLUX_LINDE) return OR_EINVAL;
  if (d->flux != FLUX_RUSANOV && d->learned) return OR_EINVAL; /* the correction is defined on Rusanov */
  for (int a = 0; a < 3; a++) {
    if (d->root[a] <= 0 || !(d->hi[a] > d->lo[a])) return OR_EINVAL;
    int lo_p = d->bc[2 * a] == BC_PERIODIC, hi_p = d->bc[2 * a + 1] == BC_PERIODIC;
    if (lo_p != hi_p) return OR_EINVAL;
    for (int s = 0; s < 2; s++) if (d->bc[2 * a + s] < 0 || d->bc[2 * a + s] > 2) return OR_EINVAL;
  }
  G->nb = d->n_leaves;
  int maxlev = 0;
  for (int b = 0; b < G->nb; b++) {
    int l = d->leaves[4 * b];
    if (l < 0 || l > MAXLEV) return OR_EINVAL;
    if (l > maxlev) maxlev = l;
  }
  G->maxlev = maxlev;
  for (int l = 0; l <= MAXLEV; l++)
    for (int a = 0; a < 3; a++) {
      G->nblk[l][a] = (long)d->root[a] << l;
      G->ncell[l][a] = G->nblk[l][a] * NC;
      G->dx[l][a] = (d->hi[a] - d->lo[a]) / (double)G->ncell[l][a];
    }
  for (int l = 0; l <= maxlev; l++) {
    long n = G->nblk[l][0] * G->nblk[l][1] * G->nblk[l][2];
    G->map[l] = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!G->map[l]) { grid_free(G); return OR_ENOMEM; }
    for (long i = 0; i < n; i++) G->map[l][i] = -1;
  }
  /* place leaves; reject out-of-range and duplicates */
  double vol = 0.0;
  for (int b = 0; b < G->nb; b++) {
    const int32_t* L = d->leaves + 4 * b;
    int l = L[0];
    for (int a = 0; a < 3; a++)
      if (L[1 + a] < 0 || L[1 + a] >= G->nblk[l][a]) { grid_free(G); return OR_EINVAL; }
    long m = map_index(G, l, L[1], L[2], L[3]);
    if (G->map[l][m] >= 0) { grid_free(G); return OR_EINVAL; }
    G->map[l][m] = b;
    vol += ldexp(1.0, -3 * l);
  }
  /* exact tiling: volumes add up and no leaf lies inside another */
  if (vol != (double)d->root[0] * d->root[1] * d->root[2]) { grid_free(G); return OR_EINVAL; }
  for (int b = 0; b < G->nb; b++) {
    const int32_t* L = d->leaves + 4 * b;
    for (int l = L[0] - 1; l >= 0; l--) {
      int sh = L[0] - l;
      if (G->map[l][map_index(G, l, L[1] >> sh, L[2] >> sh, L[3] >> sh)] >= 0) { grid_free(G); return OR_EINVAL; }
    }
  }
  /* 2:1 balance across faces, edges and corners (through periodic wraps):
   * every cell adjacent to a leaf lies in a leaf at most one level apart. */
  for (int b = 0; b < G->nb; b++) {
    const int32_t* L = d->leaves + 4 * b;
    int l = L[0];
    for (int k = -1; k <= NC; k++)
      for (int j = -1; j <= NC; j++)
        for (int i = -1; i <= NC; i++) {
          if (i >= 0 && i < NC && j >= 0 && j < NC && k >= 0 && k < NC) continue;
          long g[3] = {(long)L[1] * NC + i, (long)L[2] * NC + j, (long)L[3] * NC + k};
          int out_of_domain = 0;
          for (int a = 0; a < 3; a++) {
            long n = G->ncell[l][a];
            if (g[a] < 0 || g[a] >= n) {
              if (d->bc[2 * a] != BC_PERIODIC) out_of_domain = 1;
              else g[a] = ((g[a] % n) + n) % n;
            }
          }
          if (out_of_domain) continue;
          int ll;
          int id = locate(G, l, g, &ll);
          if (id >= 0 && ll < l - 1) { grid_free(G); return OR_EUNBALANCED; }
          if (id < 0) {
            /* finer: every child at l+1 must be a leaf */
            for (int o = 0; o < 8; o++) {
              long gc[3] = {2 * g[0] + (o & 1), 2 * g[1] + ((o >> 1) & 1), 2 * g[2] + ((o >> 2) & 1)};
              int l2;
              int id2 = locate(G, l + 1, gc, &l2);
              if (id2 < 0 || l2 != l + 1) { grid_free(G); return OR_EUNBALANCED; }
            }
          }
        }
  }
  cons_from_prim(d->gamma, d->inflow, G->Uinflow);
  cons_from_prim(d->gamma, d->body, G->Ubody);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Fluxes.                                                                   */

static double limiter(int kind, double a, double b) {
  if (kind == LIM_NONE) return 0.0; /* first order: piecewise-constant faces */
  if (kind == LIM_MC) {
    /* monotonised central, beta = 2: sign(a) min(2|a|, 2|b|, |a+b|/2) */
    if (a > 0.0 && b > 0.0) {
      double m = 2.0 * a < 2.0 * b ? 2.0 * a : 2.0 * b;
      double c = 0.5 * (a + b);
      return m < c ? m : c;
    }
    if (a < 0.0 && b < 0.0) {
      double m = 2.0 * a > 2.0 * b ? 2.0 * a : 2.0 * b;
      double c = 0.5 * (a + b);
      return m > c ? m : c;
    }
    return 0.0;
  }
  return minmod(a, b);
}

/* Fast magnetosonic speed along axis dir with the total field B:
 * cf^2 = (a^2 + b^2 + sqrt(max(0, (a^2+b^2)^2 - 4 a^2 bn^2))) / 2. */
static double fast_speed(double gamma, const double W[NV], const double B[3], int dir) {
  double rho = W[0];
  double a2 = gamma * W[7] / rho;
  double b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho;
  double bn2 = B[dir] * B[dir] / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn2;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* Split-field physical flux along dir (Eqs. 1-4 with B = B0 + B1):
 *  F_rho = rho un
 *  F_m   = rho u un + (p + B1^2/2 + B0.B1) n - (B1 Bn + B0 B1n)
 *  F_B1  = un B - Bn u          (normal component vanishes identically)
 *  F_e1  = un (e1 + p + B1^2/2 + B0.B1) - (u.B1) Bn
 * Also returns U(W), the normal speed and the fast speed. */
static void phys_flux(const or_desc* d, int dir, const double W[NV], const double B0[3],
                      double F[NV], double U[NV], double* un_out, double* cf_out) {
  double gamma = d->gamma;
  double rho = W[0], u[3] = {W[1], W[2], W[3]}, B1[3] = {W[4], W[5], W[6]}, p = W[7];
  double B[3] = {B0[0] + B1[0], B0[1] + B1[1], B0[2] + B1[2]};
  double un = u[dir], Bn = B[dir], B1n = B1[dir];
  double b1sq = B1[0] * B1[0] + B1[1] * B1[1] + B1[2] * B1[2];
  double b0b1 = B0[0] * B1[0] + B0[1] * B1[1] + B0[2] * B1[2];
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double pt = p + 0.5 * b1sq + b0b1;
  double e1 = p * (1.0 / (gamma - 1.0)) + 0.5 * rho * usq + 0.5 * b1sq;
  double ub1 = u[0] * B1[0] + u[1] * B1[1] + u[2] * B1[2];
  F[0] = rho * un;
  for (int c = 0; c < 3; c++) {
    double f = rho * u[c] * un;
    if (c == dir) f = f + pt;
    F[1 + c] = f - (B1[c] * Bn + B0[c] * B1n);
    F[4 + c] = (c == dir) ? 0.0 : un * B[c] - Bn * u[c];
  }
  F[7] = un * (e1 + pt) - ub1 * Bn;
  U[0] = rho;
  U[1] = rho * u[0];
  U[2] = rho * u[1];
  U[3] = rho * u[2];
  U[4] = B1[0];
  U[5] = B1[1];
  U[6] = B1[2];
  U[7] = e1;
  *un_out = un;
  *cf_out = fast_speed(gamma, W, B, dir);
}

/* ------------------------------------------------------------------------ */
/* Learned flux correction (a4'): features, MLP, clipping.                   */

static double gelu_tanh(double x) {
  /* GELU, tanh form (Hendrycks & Gimpel 2016) */
  const double k = 0.7978845608028654; /* sqrt(2/pi) */
  return 0.5 * x * (1.0 + tanh(k * (x + 0.044715 * x * x * x)));
}

/* Face-normal frame: component order (normal, t1, t2) = cyclic from dir. */
static void rotate3(int dir, const double a[3], double r[3]) {
  r[0] = a[dir];
  r[1] = a[(dir + 1) % 3];
  r[2] = a[(dir + 2) % 3];
}

/* 40 normalised inputs: the 4 primitive states i-1..i+2 around the face (32)
 * and the mean reconstructed state (WL + WR)/2 (8), rotated into the face
 * frame; rho / rho_ref, u / c_ref, B1 / (sqrt(rho_ref) c_ref),
 * p / (rho_ref c_ref^2) with rho_ref = mean stencil density and c_ref =
 * the Rusanov c_max. */
void or_mlp_features(int dir, const double* Ws /* 4 x 8 */, const double WL[NV], const double WR[NV],
                     double cmax, double x[MLP_IN]) {
  double rho_ref = 0.25 * (Ws[0] + Ws[8] + Ws[16] + Ws[24]);
  double c_ref = cmax;
  double bref = sqrt(rho_ref) * c_ref;
  double pref = rho_ref * c_ref * c_ref;
  for (int s = 0; s < 5; s++) {
    double W[NV];
    if (s < 4) memcpy(W, Ws + 8 * s, sizeof(W));
    else for (int v = 0; v < NV; v++) W[v] = 0.5 * (WL[v] + WR[v]);
    double u[3], b[3], ur[3], br[3];
    u[0] = W[1]; u[1] = W[2]; u[2] = W[3];
    b[0] = W[4]; b[1] = W[5]; b[2] = W[6];
    rotate3(dir, u, ur);
    rotate3(dir, b, br);
    double* o = x + 8 * s;
    o[0] = W[0] / rho_ref;
    for (int c = 0; c < 3; c++) o[1 + c] = ur[c] / c_ref;
    for (int c = 0; c < 3; c++) o[4 + c] = br[c] / bref;
    o[7] = W[7] / pref;
  }
}

/* Plain FP64 MLP forward: h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), y = W3 h2 + b3. */
void or_mlp_forward(const double* P, const double x[MLP_IN], double h1[MLP_H], double h2[MLP_H], double y[MLP_OUT]) {
  const double* W1 = P;
  const double* b1 = W1 + MLP_H * MLP_IN;
  const double* W2 = b1 + MLP_H;
  const double* b2 = W2 + MLP_H * MLP_H;
  const double* W3 = b2 + MLP_H;
  const double* b3 = W3 + MLP_OUT * MLP_H;
  for (int o = 0; o < MLP_H; o++) {
    double s = 0.0;
    for (int i = 0; i < MLP_IN; i++) s += W1[o * MLP_IN + i] * x[i];
    h1[o] = gelu_tanh(s + b1[o]);
  }
  for (int o = 0; o < MLP_H; o++) {
    double s = 0.0;
    for (int i = 0; i < MLP_H; i++) s += W2[o * MLP_H + i] * h1[i];
    h2[o] = gelu_tanh(s + b2[o]);
  }
  for (int o = 0; o < MLP_OUT; o++) {
    double s = 0.0;
    for (int i = 0; i < MLP_H; i++) s += W3[o * MLP_H + i] * h2[i];
    y[o] = s + b3[o];
  }
}

/* Derivative of the tanh-form GELU. */
static double gelu_tanh_grad(double x) {
  const double k = 0.7978845608028654;
  double u = k * (x + 0.044715 * x * x * x);
  double t = tanh(u);
  double du = k * (1.0 + 3.0 * 0.044715 * x * x);
  return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du;
}

double or_gelu(double x) { return gelu_tanh(x); }

/* Mean-squared-error loss over n samples and its gradient by backpropagation
 * (chain rule through the three layers):
 *   L = (1/(8n)) sum_s sum_o (y_o(x_s) - t_so)^2.
 * X is n x 40, T is n x 8; grad has MLP_NPARAM entries in the parameter
 * layout (W1, b1, W2, b2, W3, b3).  Returns L. */
double or_mlp_loss_grad(const double* P, const double* X, const double* T, long n, double* grad) {
  const double* W1 = P;
  const double* b1 = W1 + MLP_H * MLP_IN;
  const double* W2 = b1 + MLP_H;
  const double* b2 = W2 + MLP_H * MLP_H;
  const double* W3 = b2 + MLP_H;
  const double* b3 = W3 + MLP_OUT * MLP_H;
  double* gW1 = grad;
  double* gb1 = gW1 + MLP_H * MLP_IN;
  double* gW2 = gb1 + MLP_H;
  double* gb2 = gW2 + MLP_H * MLP_H;
  double* gW3 = gb2 + MLP_H;
  double* gb3 = gW3 + MLP_OUT * MLP_H;
  memset(grad, 0, sizeof(double) * MLP_NPARAM);
  double loss = 0.0;
  for (long s = 0; s < n; s++) {
    const double* x = X + s * MLP_IN;
    const double* t = T + s * MLP_OUT;
    double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], y[MLP_OUT];
    for (int o = 0; o < MLP_H; o++) {
      double a = 0.0;
      for (int i = 0; i < MLP_IN; i++) a += W1[o * MLP_IN + i] * x[i];
      z1[o] = a + b1[o];
      h1[o] = gelu_tanh(z1[o]);
    }
    for (int o = 0; o < MLP_H; o++) {
      double a = 0.0;
      for (int i = 0; i < MLP_H; i++) a += W2[o * MLP_H + i] * h1[i];
      z2[o] = a + b2[o];
      h2[o] = gelu_tanh(z2[o]);
    }
    double dy[MLP_OUT];
    for (int o = 0; o < MLP_OUT; o++) {
      double a = 0.0;
      for (int i = 0; i < MLP_H; i++) a += W3[o * MLP_H + i] * h2[i];
      y[o] = a + b3[o];
      double e = y[o] - t[o];
      loss += e * e;
      dy[o] = 2.0 * e / (8.0 * (double)n);
    }
    double dh2[MLP_H], dz2[MLP_H], dh1[MLP_H], dz1[MLP_H];
    for (int i = 0; i < MLP_H; i++) dh2[i] = 0.0;
    for (int o = 0; o < MLP_OUT; o++) {
      gb3[o] += dy[o];
      for (int i = 0; i < MLP_H; i++) {
        gW3[o * MLP_H + i] += dy[o] * h2[i];
        dh2[i] += dy[o] * W3[o * MLP_H + i];
      }
    }
    for (int o = 0; o < MLP_H; o++) dz2[o] = dh2[o] * gelu_tanh_grad(z2[o]);
    for (int i = 0; i < MLP_H; i++) dh1[i] = 0.0;
    for (int o = 0; o < MLP_H; o++) {
      gb2[o] += dz2[o];
      for (int i = 0; i < MLP_H; i++) {
        gW2[o * MLP_H + i] += dz2[o] * h1[i];
        dh1[i] += dz2[o] * W2[o * MLP_H + i];
      }
    }
    for (int o = 0; o < MLP_H; o++) dz1[o] = dh1[o] * gelu_tanh_grad(z1[o]);
    for (int o = 0; o < MLP_H; o++) {
      gb1[o] += dz1[o];
      for (int i = 0; i < MLP_IN; i++) gW1[o * MLP_IN + i] += dz1[o] * x[i];
    }
  }
  return loss / (8.0 * (double)n);
}

/* Output scale per rotated flux component (flux units of each variable):
 * mass rho c, momentum rho c^2, B sqrt(rho) c^2, energy rho c^3. */
void or_mlp_out_scale(double rho_ref, double c_ref, double sc[MLP_OUT]) {
  sc[0] = rho_ref * c_ref;
  sc[1] = sc[2] = sc[3] = rho_ref * c_ref * c_ref;
  sc[4] = sc[5] = sc[6] = sqrt(rho_ref) * c_ref * c_ref;
  sc[7] = rho_ref * c_ref * c_ref * c_ref;
}

/* ------------------------------------------------------------------------ */
/* One stage.                                                                */

typedef struct {
  double F[NV];
  double bn;     /* face-averaged reconstructed normal B1 */
  double B0[3];  /* B0 at the face centre */
} face_t;

static void cell_centre(const grid_t* G, int lev, const int32_t* L, int i, int j, int k, double x[3]) {
  const or_desc* d = G->d;
  long gi[3] = {(long)L[1] * NC + i, (long)L[2] * NC + j, (long)L[3] * NC + k};
  for (int a = 0; a < 3; a++) x[a] = d->lo[a] + ((double)gi[a] + 0.5) * G->dx[lev][a];
}

static int in_body(const or_desc* d, const double x[3]) {
  if (!(d->body_r > 0.0)) return 0;
  return x[0] * x[0] + x[1] * x[1] + x[2] * x[2] < d->body_r * d->body_r;
}

/* Numerical flux from the two face states' physical fluxes F, states U,
 * primitives W (x, y, z components), normal speeds un and fast speeds cf.
 *  Rusanov: F = (F_L + F_R)/2 - cmax (U_R - U_L)/2,
 *           cmax = max(|un_L| + cf_L, |un_R| + cf_R).
 *  HLL (Harten, Lax and van Leer 1983), with the wave-speed bounds of Davis
 *  (1988) S_L = min(un_L - cf_L, un_R - cf_R), S_R = max(un_L + cf_L,
 *  un_R + cf_R): F = F_L where S_L >= 0, F = F_R where S_R <= 0, else
 *  F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
 *  Linde (the paper's flux, Section 5.1, cited to Linde 2002 without its
 *  formula): HLL with the contact (entropy) wave restored -- HLL's
 *  dissipation S_L S_R / (S_R - S_L) (U_R - U_L) smears a density jump that no
 *  wave but the flow carries; the part of the jump along the contact's
 *  eigenvector r = (1, u, 0, |u|^2 / 2) (density, momentum, field, energy at
 *  fixed pressure, velocity and field), of strength alpha =
 *  minmod((rho_R - rho_L) - (p_R - p_L) / c^2, rho_R - rho_L) (the density
 *  jump not carried by the pressure jump, never more than the density jump
 *  itself nor of the other sign), is taken back out with the weight
 *  delta = c / (c + |u_n|):  F = F_HLL - delta alpha S_L S_R / (S_R - S_L) r,
 *  with u, rho, p the means of the two face states and c^2 = gamma p / rho
 *  (reading 18).  `contact` scales the restored part (1 for the flux, 0 gives
 *  HLL). */
static void numerical_flux(int kind, int dir, double gamma, const double WL[NV], const double WR[NV],
                           const double FL[NV], const double FR[NV], const double UL[NV], const double UR[NV],
                           double unL, double unR, double cfL, double cfR, double contact, double F[NV]) {
  if (kind == FLUX_HLL || kind == FLUX_LINDE) {
    double SL = fmin(unL - cfL, unR - cfR);
    double SR = fmax(unL + cfL, unR + cfR);
    if (SL >= 0.0) {
      for (int v = 0; v < NV; v++) F[v] = FL[v];
    } else if (SR <= 0.0) {
      for (int v = 0; v < NV; v++) F[v] = FR[v];
    } else {
      for (int v = 0; v < NV; v++)
        F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
      if (kind == FLUX_LINDE) {
        double rho = 0.5 * (WL[0] + WR[0]), p = 0.5 * (WL[7] + WR[7]), u[3];
        for (int c = 0; c < 3; c++) u[c] = 0.5 * (WL[1 + c] + WR[1 + c]);
        double c2 = gamma * p / rho, cs = sqrt(c2);
        double alpha = minmod((WR[0] - WL[0]) - (WR[7] - WL[7]) / c2, WR[0] - WL[0]);
        double delta = cs / (cs + fabs(u[dir]));
        double q = contact * delta * alpha * SL * SR / (SR - SL);
        F[0] -= q;
        for (int c = 0; c < 3; c++) F[1 + c] -= q * u[c];
        F[7] -= q * 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      }
    }
    return;
  }
  double aL = fabs(unL) + cfL, aR = fabs(unR) + cfR;
  double cmax = aL > aR ? aL : aR;
  for (int v = 0; v < NV; v++) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * cmax * (UR[v] - UL[v]);
}

/* Face flux between tile cells m1 = p0 - e_dir and p0 (tile coords 0..11),
 * with the limited reconstruction of primitives, the numerical flux and, when
 * learned, the clipped MLP correction. */
static void face_flux(const grid_t* G, int dir, const double* Wt /* [12^3][8] */, int ti, int tj, int tk,
                      const double B0f[3], face_t* out) {
  const or_desc* d = G->d;
  int st = dir == 0 ? 1 : dir == 1 ? NT : NT * NT;
  int c0 = (tk * NT + tj) * NT + ti; /* cell p0 */
  const double* Wm2 = Wt + 8 * (c0 - 2 * st);
  const double* Wm1 = Wt + 8 * (c0 - st);
  const double* Wp0 = Wt + 8 * c0;
  const double* Wp1 = Wt + 8 * (c0 + st);
  double WL[NV], WR[NV];
  for (int v = 0; v < NV; v++) {
    double sl = limiter(d->limiter, Wm1[v] - Wm2[v], Wp0[v] - Wm1[v]);
    double sr = limiter(d->limiter, Wp0[v] - Wm1[v], Wp1[v] - Wp0[v]);
    WL[v] = Wm1[v] + 0.5 * sl;
    WR[v] = Wp0[v] - 0.5 * sr;
  }
  double FL[NV], FR[NV], UL[NV], UR[NV], unL, unR, cfL, cfR;
  phys_flux(d, dir, WL, B0f, FL, UL, &unL, &cfL);
  phys_flux(d, dir, WR, B0f, FR, UR, &unR, &cfR);
  double aL = fabs(unL) + cfL, aR = fabs(unR) + cfR;
  double cmax = aL > aR ? aL : aR;
  numerical_flux(d->flux, dir, d->gamma, WL, WR, FL, FR, UL, UR, unL, unR, cfL, cfR, 1.0, out->F);
  if (d->learned && d->mlp) {
    double Ws[32], x[MLP_IN], h1[MLP_H], h2[MLP_H], y[MLP_OUT], sc[MLP_OUT];
    memcpy(Ws, Wm2, 64); memcpy(Ws + 8, Wm1, 64); memcpy(Ws + 16, Wp0, 64); memcpy(Ws + 24, Wp1, 64);
    or_mlp_features(dir, Ws, WL, WR, cmax, x);
    or_mlp_forward(d->mlp, x, h1, h2, y);
    double rho_ref = 0.25 * (Ws[0] + Ws[8] + Ws[16] + Ws[24]);
    or_mlp_out_scale(rho_ref, cmax, sc);
    /* back from the face frame to x,y,z, then clip each component to the
     * Rusanov dissipation |cmax (UR-UL)/2| */
    double dF[NV];
    dF[0] = y[0] * sc[0];
    dF[7] = y[7] * sc[7];
    for (int c = 0; c < 3; c++) {
      dF[1 + (dir + c) % 3] = y[1 + c] * sc[1 + c];
      dF[4 + (dir + c) % 3] = y[4 + c] * sc[4 + c];
    }
    for (int v = 0; v < NV; v++) {
      double lim = fabs(0.5 * cmax * (UR[v] - UL[v]));
      double f = dF[v];
      if (f > lim) f = lim;
      if (f < -lim) f = -lim;
      out->F[v] = out->F[v] + f;
    }
  }
  out->bn = 0.5 * (WL[4 + dir] + WR[4 + dir]);
  out->B0[0] = B0f[0];
  out->B0[1] = B0f[1];
  out->B0[2] = B0f[2];
}

/* Kind of the neighbour region across face s (= 2 d + side) of block b: 0
 * same level or domain boundary, 1 one level coarser, 2 refined. */
static int face_kind(const grid_t* G, int b, int s) {
  const or_desc* d = G->d;
  const int32_t* L = d->leaves + 4 * b;
  int lev = L[0], dir = s >> 1, side = s & 1;
  long p[3] = {L[1], L[2], L[3]};
  p[dir] += side ? 1 : -1;
  long n = G->nblk[lev][dir];
  if (p[dir] < 0 || p[dir] >= n) {
    if (d->bc[s] != BC_PERIODIC) return 0;
    p[dir] = (p[dir] + n) % n;
  }
  if (G->map[lev][map_index(G, lev, p[0], p[1], p[2])] >= 0) return 0;
  if (lev >= 1 && G->map[lev - 1][map_index(G, lev - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1)] >= 0) return 1;
  return 2;
}

/* Refluxing (conservative flux correction at resolution changes): the flux
 * through a coarse face that borders a refined region is the mean of the 4
 * fine fluxes through it, so that what leaves the fine cells enters the
 * coarse cell.  fbound holds, per block, its face fluxes on the 6 block faces
 * [nb][6][64][8] ((q, r) = the two transverse cell indices, increasing axis
 * order), filled for every block that has a coarser neighbour. */
static void reflux_face(const grid_t* G, int b, int s, const double* fbound, face_t* Fx) {
  const or_desc* d = G->d;
  const int32_t* L = d->leaves + 4 * b;
  int lev = L[0], dir = s >> 1, side = s & 1;
  int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
  long fb[3];
  fb[dir] = side ? 2L * L[1 + dir] + 2 : 2L * L[1 + dir] - 1;
  long n = G->nblk[lev + 1][dir];
  fb[dir] = (fb[dir] + n) % n;
  for (int q = 0; q < NC; q++)
    for (int r = 0; r < NC; r++) {
      double f[2][2][NV];
      for (int eq = 0; eq < 2; eq++)
        for (int er = 0; er < 2; er++) {
          long gq = 2L * ((long)L[1 + t1] * NC + q) + eq, gr = 2L * ((long)L[1 + t2] * NC + r) + er;
          fb[t1] = gq / NC;
          fb[t2] = gr / NC;
          int fine = G->map[lev + 1][map_index(G, lev + 1, fb[0], fb[1], fb[2])];
          if (fine < 0) return; /* excluded by the 2:1 balance */
          int qf = (int)(gq - fb[t1] * NC), rf = (int)(gr - fb[t2] * NC);
          const double* src = fbound + (((long)fine * 6 + (s ^ 1)) * 64 + qf * NC + rf) * NV;
          for (int v = 0; v < NV; v++) f[eq][er][v] = src[v];
        }
      face_t* o = &Fx[(dir * 9 + (side ? NC : 0)) * 64 + q * 8 + r];
      for (int v = 0; v < NV; v++) o->F[v] = 0.25 * ((f[0][0][v] + f[1][0][v]) + (f[0][1][v] + f[1][1][v]));
    }
}

/* Residual R = -sum_d (F_{d,+} - F_{d,-}) / dx_d + S for every cell of block b,
 * from the padded tile of the stage input. R is [8][512] for this block.
 * bound_out (nullable, [6][64][8]): the block's face fluxes on its 6 faces;
 * fbound (nullable): refluxing with the fine blocks' boundary fluxes. */
static void block_residual_rf(grid_t* G, int b, double* R, double* bound_out, const double* fbound);
static void block_residual(grid_t* G, int b, double* R) { block_residual_rf(G, b, R, NULL, NULL); }
static void block_residual_rf(grid_t* G, int b, double* R, double* bound_out, const double* fbound) {
  const or_desc* d = G->d;
  const int32_t* L = d->leaves + 4 * b;
  int lev = L[0];
  double* T = (double*)malloc(sizeof(double) * NT * NT * NT * NV);   /* conservative, [cell][v] */
  double* Wt = (double*)malloc(sizeof(double) * NT * NT * NT * NV);  /* primitive, [cell][v] */
  face_t* Fx = (face_t*)malloc(sizeof(face_t) * 9 * 64 * 3);
  if (!T || !Wt || !Fx) { free(T); free(Wt); free(Fx); return; }
  /* 1. padded tile: interior copy, ghosts by point location */
  for (int k = -NG; k < NC + NG; k++)
    for (int j = -NG; j < NC + NG; j++)
      for (int i = -NG; i < NC + NG; i++) {
        double* o = T + 8 * (((k + NG) * NT + (j + NG)) * NT + (i + NG));
        if (i >= 0 && i < NC && j >= 0 && j < NC && k >= 0 && k < NC) {
          int c = (k * NC + j) * NC + i;
          for (int v = 0; v < NV; v++) o[v] = G->U[((long)v * G->nb + b) * NCELL + c];
        } else {
          long g[3] = {(long)L[1] * NC + i, (long)L[2] * NC + j, (long)L[3] * NC + k};
          value_at(G, lev, g, o);
        }
      }
  /* 2. primitives */
  for (int c = 0; c < NT * NT * NT; c++) prim_from_cons(d->gamma, T + 8 * c, Wt + 8 * c);
  /* 3. face values and fluxes, per direction; face f sits on the low side of
   *    interior cell f (f = 0..8) */
  for (int dir = 0; dir < 3; dir++) {
    for (int f = 0; f <= NC; f++)
      for (int q = 0; q < NC; q++)
        for (int r = 0; r < NC; r++) {
          int ci[3];
          /* (f along dir; q, r along the other two axes in increasing order) */
          if (dir == 0) { ci[0] = f; ci[1] = q; ci[2] = r; }
          else if (dir == 1) { ci[0] = q; ci[1] = f; ci[2] = r; }
          else { ci[0] = q; ci[1] = r; ci[2] = f; }
          long gi[3] = {(long)L[1] * NC + ci[0], (long)L[2] * NC + ci[1], (long)L[3] * NC + ci[2]};
          double xf[3], B0f[3];
          for (int a = 0; a < 3; a++) {
            double off = (a == dir) ? 0.0 : 0.5;
            xf[a] = d->lo[a] + ((double)gi[a] + off) * G->dx[lev][a];
          }
          b0_at(d, xf, B0f);
          face_flux(G, dir, Wt, ci[0] + NG, ci[1] + NG, ci[2] + NG, B0f, &Fx[(dir * 9 + f) * 64 + q * 8 + r]);
        }
  }
  if (bound_out)
    for (int s = 0; s < 6; s++)
      for (int qr = 0; qr < 64; qr++)
        memcpy(bound_out + (s * 64 + qr) * NV, Fx[((s >> 1) * 9 + ((s & 1) ? NC : 0)) * 64 + qr].F,
               sizeof(double) * NV);
  if (fbound)
    for (int s = 0; s < 6; s++)
      if (face_kind(G, b, s) == 2) reflux_face(G, b, s, fbound, Fx);
  /* 4. sources and residual per cell */
  double idx[3] = {1.0 / G->dx[lev][0], 1.0 / G->dx[lev][1], 1.0 / G->dx[lev][2]};
  for (int k = 0; k < NC; k++)
    for (int j = 0; j < NC; j++)
      for (int i = 0; i < NC; i++) {
        int cc[3] = {i, j, k};
        const face_t* fm[3];
        const face_t* fp[3];
        for (int dir = 0; dir < 3; dir++) {
          int q, r;
          if (dir == 0) { q = j; r = k; }
          else if (dir == 1) { q = i; r = k; }
          else { q = i; r = j; }
          fm[dir] = &Fx[(dir * 9 + cc[dir]) * 64 + q * 8 + r];
          fp[dir] = &Fx[(dir * 9 + cc[dir] + 1) * 64 + q * 8 + r];
        }
        double res[NV];
        for (int v = 0; v < NV; v++) {
          double s = -(fp[0]->F[v] - fm[0]->F[v]) * idx[0];
          s = s - (fp[1]->F[v] - fm[1]->F[v]) * idx[1];
          s = s - (fp[2]->F[v] - fm[2]->F[v]) * idx[2];
          res[v] = s;
        }
        const double* W = Wt + 8 * (((k + NG) * NT + (j + NG)) * NT + (i + NG));
        double S[NV] = {0, 0, 0, 0, 0, 0, 0, 0};
        double xc[3], B0c[3];
        cell_centre(G, lev, L, i, j, k, xc);
        b0_at(d, xc, B0c);
        double u[3] = {W[1], W[2], W[3]}, B1[3] = {W[4], W[5], W[6]};
        if (d->powell) {
          /* Powell 8-wave terms: -divB (0, B, u, u.B1) with the face-averaged
           * reconstructed normal B1 */
          double divb = (fp[0]->bn - fm[0]->bn) * idx[0] + (fp[1]->bn - fm[1]->bn) * idx[1] +
                        (fp[2]->bn - fm[2]->bn) * idx[2];
          double ub1 = u[0] * B1[0] + u[1] * B1[1] + u[2] * B1[2];
          for (int c = 0; c < 3; c++) {
            S[1 + c] = -divb * (B0c[c] + B1[c]);
            S[4 + c] = -divb * u[c];
          }
          S[7] = -divb * ub1;
        }
        if (d->b0 != B0_NONE) {
          /* split-field correction for the discrete div and curl of B0:
           * S_m += -B1 (div B0)_h + B1 x (curl B0)_h, from face-centre B0 */
          double divb0 = (fp[0]->B0[0] - fm[0]->B0[0]) * idx[0] + (fp[1]->B0[1] - fm[1]->B0[1]) * idx[1] +
                         (fp[2]->B0[2] - fm[2]->B0[2]) * idx[2];
          double cx = (fp[1]->B0[2] - fm[1]->B0[2]) * idx[1] - (fp[2]->B0[1] - fm[2]->B0[1]) * idx[2];
          double cy = (fp[2]->B0[0] - fm[2]->B0[0]) * idx[2] - (fp[0]->B0[2] - fm[0]->B0[2]) * idx[0];
          double cz = (fp[0]->B0[1] - fm[0]->B0[1]) * idx[0] - (fp[1]->B0[0] - fm[1]->B0[0]) * idx[1];
          S[1] = (S[1] - B1[0] * divb0) + (B1[1] * cz - B1[2] * cy);
          S[2] = (S[2] - B1[1] * divb0) + (B1[2] * cx - B1[0] * cz);
          S[3] = (S[3] - B1[2] * divb0) + (B1[0] * cy - B1[1] * cx);
        }
        int c = (k * NC + j) * NC + i;
        for (int v = 0; v < NV; v++) R[v * NCELL + c] = res[v] + S[v];
      }
  free(T);
  free(Wt);
  free(Fx);
}

/* ------------------------------------------------------------------------ */
/* Public entry points (ctypes).                                             */

int or_validate(const or_desc* d) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc == OR_OK) grid_free(&G);
  return rc;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Padded tiles [8][nb][12][12][12] of the conservative state, ghosts filled. */
int or_fill_ghosts(const or_desc* d, const double* U, double* T, long* deep_prolong) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  G.U = U;
  long deep = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : deep)
  for (int b = 0; b < G.nb; b++) {
    grid_t Gl = G;
    Gl.deep_prolong = 0;
    const int32_t* L = d->leaves + 4 * b;
    for (int k = -NG; k < NC + NG; k++)
      for (int j = -NG; j < NC + NG; j++)
        for (int i = -NG; i < NC + NG; i++) {
          double o[NV];
          if (i >= 0 && i < NC && j >= 0 && j < NC && k >= 0 && k < NC) {
            int c = (k * NC + j) * NC + i;
            for (int v = 0; v < NV; v++) o[v] = U[((long)v * G.nb + b) * NCELL + c];
          } else {
            long g[3] = {(long)L[1] * NC + i, (long)L[2] * NC + j, (long)L[3] * NC + k};
            value_at(&Gl, L[0], g, o);
          }
          long t = ((long)(k + NG) * NT + (j + NG)) * NT + (i + NG);
          for (int v = 0; v < NV; v++) T[((long)v * G.nb + b) * (NT * NT * NT) + t] = o[v];
        }
    deep += Gl.deep_prolong;
  }
  if (deep_prolong) *deep_prolong = deep;
  grid_free(&G);
  return OR_OK;
}

/* Ghost classification of block b: type and source leaf per tile cell. */
int or_ghost_info(const or_desc* d, int b, int32_t* type, int32_t* src) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  if (b < 0 || b >= G.nb) { grid_free(&G); return OR_EINVAL; }
  const int32_t* L = d->leaves + 4 * b;
  for (int k = -NG; k < NC + NG; k++)
    for (int j = -NG; j < NC + NG; j++)
      for (int i = -NG; i < NC + NG; i++) {
        long t = ((long)(k + NG) * NT + (j + NG)) * NT + (i + NG);
        if (i >= 0 && i < NC && j >= 0 && j < NC && k >= 0 && k < NC) { type[t] = GT_INTERIOR; src[t] = b; continue; }
        long g[3] = {(long)L[1] * NC + i, (long)L[2] * NC + j, (long)L[3] * NC + k};
        type[t] = ghost_class(&G, L[0], g, &src[t]);
      }
  grid_free(&G);
  return OR_OK;
}

/* R(Uin) for every block: R is [8][nb][512]. */
int or_residual(const or_desc* d, const double* Uin, double* R) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  G.U = Uin;
  int nb = G.nb;
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < nb; b++) {
    grid_t Gl = G;
    double Rb[NV * NCELL];
    block_residual(&Gl, b, Rb);
    for (int v = 0; v < NV; v++) memcpy(R + ((long)v * nb + b) * NCELL, Rb + v * NCELL, sizeof(double) * NCELL);
  }
  grid_free(&G);
  return OR_OK;
}

/* The stage output of block b from its residual Rb:
 *   kind 0: Uout = Ubase + c R(Uin)   (midpoint stages, SSP-RK2 stage 1)
 *   kind 1: Uout = 0.5 Ubase + 0.5 (Uin + c R(Uin))   (SSP-RK2 stage 2)
 * Body cells (centre radius < body_r) are set to the body state.  Ob is
 * [8][512].  Returns 1 when every non-body cell of the result is physical:
 * all 8 values finite, rho > 0 and p > 0 (p from Eq. 5). */
static int block_update(grid_t* G, int b, const double* Rb, const double* Uin, const double* Ubase, int kind,
                        double c, const double* dtc, double* Ob) {
  const or_desc* d = G->d;
  const int32_t* L = d->leaves + 4 * b;
  int nb = G->nb, ok = 1;
  for (int k = 0; k < NC; k++)
    for (int j = 0; j < NC; j++)
      for (int i = 0; i < NC; i++) {
        int cidx = (k * NC + j) * NC + i;
        double xc[3], Uc[NV], W[NV];
        cell_centre(G, L[0], L, i, j, k, xc);
        int body = in_body(d, xc);
        for (int v = 0; v < NV; v++) {
          long gidx = ((long)v * nb + b) * NCELL + cidx;
          double r = Rb[v * NCELL + cidx];
          double cc = dtc ? c * dtc[(long)b * NCELL + cidx] : c;
          double o;
          if (body) o = G->Ubody[v];
          else if (kind == 0) o = Ubase[gidx] + cc * r;
          else o = 0.5 * Ubase[gidx] + 0.5 * (Uin[gidx] + cc * r);
          Ob[v * NCELL + cidx] = o;
          Uc[v] = o;
        }
        if (body) continue;
        prim_from_cons(d->gamma, Uc, W);
        for (int v = 0; v < NV; v++) ok &= isfinite(Uc[v]) != 0;
        ok &= Uc[0] > 0.0;
        ok &= W[7] > 0.0;
      }
  return ok;
}

/* One stage (kinds as in block_update).  dtc (nullable, [nb][512]): local
 * time stepping, the coefficient of cell i is c * dtc[i] instead of c.  With
 * the learned correction, a block whose learned update leaves a non-physical
 * cell is recomputed with the plain Rusanov flux (the fallback of the learned
 * form); fb (nullable, one flag per block) records which blocks fell back. */
int or_stage_ex(const or_desc* d, const double* Uin, const double* Ubase, double* Uout, int kind, double c,
                const double* dtc, int32_t* fb) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  G.U = Uin;
  int nb = G.nb;
  or_desc plain = *d;
  plain.learned = 0;
  double* fbound = NULL;
  if (d->reflux) {
    if (d->learned) { grid_free(&G); return OR_EINVAL; }
    fbound = (double*)calloc((size_t)nb * 6 * 64 * NV, sizeof(double));
    if (!fbound) { grid_free(&G); return OR_ENOMEM; }
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < nb; b++) {
      int has_coarser = 0;
      for (int sf = 0; sf < 6; sf++) has_coarser |= face_kind(&G, b, sf) == 1;
      if (!has_coarser) continue;
      grid_t Gl = G;
      double Rb[NV * NCELL];
      block_residual_rf(&Gl, b, Rb, fbound + (size_t)b * 6 * 64 * NV, NULL);
    }
  }
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < nb; b++) {
    grid_t Gl = G;
    double Rb[NV * NCELL], Ob[NV * NCELL];
    block_residual_rf(&Gl, b, Rb, NULL, fbound);
    int ok = block_update(&Gl, b, Rb, Uin, Ubase, kind, c, dtc, Ob);
    int fell_back = 0;
    if (!ok && d->learned && d->mlp && !d->no_fallback) {
      Gl.d = &plain;
      block_residual(&Gl, b, Rb);
      block_update(&Gl, b, Rb, Uin, Ubase, kind, c, dtc, Ob);
      fell_back = 1;
    }
    if (fb) fb[b] = fell_back;
    for (int v = 0; v < NV; v++) memcpy(Uout + ((long)v * nb + b) * NCELL, Ob + v * NCELL, sizeof(double) * NCELL);
  }
  free(fbound);
  grid_free(&G);
  return OR_OK;
}

int or_stage(const or_desc* d, const double* Uin, const double* Ubase, double* Uout, int kind, double c) {
  return or_stage_ex(d, Uin, Ubase, Uout, kind, c, NULL, NULL);
}

/* Largest sum_d (|u_d| + cf_d) / dx_d over non-body cells; dt = cfl / smax. */
int or_cfl_smax(const or_desc* d, const double* U, double* smax_out) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  double smax = 0.0;
  int nb = G.nb;
#pragma omp parallel for schedule(static) reduction(max : smax)
  for (int b = 0; b < nb; b++) {
    const int32_t* L = d->leaves + 4 * b;
    int lev = L[0];
    for (int c = 0; c < NCELL; c++) {
      int i = c % NC, j = (c / NC) % NC, k = c / (NC * NC);
      double xc[3], B0c[3], Uc[NV], W[NV];
      cell_centre(&G, lev, L, i, j, k, xc);
      if (in_body(d, xc)) continue;
      for (int v = 0; v < NV; v++) Uc[v] = U[((long)v * nb + b) * NCELL + c];
      prim_from_cons(d->gamma, Uc, W);
      b0_at(d, xc, B0c);
      double B[3] = {B0c[0] + W[4], B0c[1] + W[5], B0c[2] + W[6]};
      double s = 0.0;
      for (int a = 0; a < 3; a++) s = s + (fabs(W[1 + a]) + fast_speed(d->gamma, W, B, a)) / G.dx[lev][a];
      if (s > smax) smax = s;
    }
  }
  *smax_out = smax;
  grid_free(&G);
  return OR_OK;
}

/* Local time step of every cell (steady-state runs): dt_i = cfl / s_i with
 * s_i = sum_d (|u_d| + cf_d) / dx_d of the cell, the bound whose global
 * maximum gives the time-accurate dt; body cells get 0.  dtc is [nb][512]. */
int or_local_dt(const or_desc* d, const double* U, double cfl, double* dtc) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  int nb = G.nb;
#pragma omp parallel for schedule(static)
  for (int b = 0; b < nb; b++) {
    const int32_t* L = d->leaves + 4 * b;
    int lev = L[0];
    for (int c = 0; c < NCELL; c++) {
      int i = c % NC, j = (c / NC) % NC, k = c / (NC * NC);
      double xc[3], B0c[3], Uc[NV], W[NV];
      cell_centre(&G, lev, L, i, j, k, xc);
      if (in_body(d, xc)) { dtc[(long)b * NCELL + c] = 0.0; continue; }
      for (int v = 0; v < NV; v++) Uc[v] = U[((long)v * nb + b) * NCELL + c];
      prim_from_cons(d->gamma, Uc, W);
      b0_at(d, xc, B0c);
      double B[3] = {B0c[0] + W[4], B0c[1] + W[5], B0c[2] + W[6]};
      double s = 0.0;
      for (int a = 0; a < 3; a++) s = s + (fabs(W[1 + a]) + fast_speed(d->gamma, W, B, a)) / G.dx[lev][a];
      dtc[(long)b * NCELL + c] = cfl / s;
    }
  }
  grid_free(&G);
  return OR_OK;
}

/* n full steps.  Two stages (midpoint or SSP-RK2) or one (forward Euler,
 * RK_EULER).  cfl > 0: dt = cfl / smax(U^n) each step; cfl <= 0: dt =
 * fixed_dt.  With local time stepping (and cfl > 0) every cell takes its own
 * dt_i from U^n (or_local_dt) in every stage of the step, and the elapsed
 * time advances by the global dt.  Returns the last dt, the elapsed time and
 * (nullable) the number of block-stages that fell back to the plain flux. */
int or_run_ex(const or_desc* d, double* U, int nsteps, double cfl, double fixed_dt, double* dt_last,
              double* t_total, long* n_fallback) {
  grid_t G;
  int rc = grid_init(&G, d, 0.0);
  if (rc) return rc;
  int nb = G.nb;
  size_t n = (size_t)NV * nb * NCELL;
  grid_free(&G);
  double* U1 = (double*)malloc(sizeof(double) * n);
  double* U2 = (double*)malloc(sizeof(double) * n);
  int32_t* fb = (int32_t*)malloc(sizeof(int32_t) * nb);
  const int lts = d->local_dt && cfl > 0.0;
  double* dtc = lts ? (double*)malloc(sizeof(double) * (size_t)nb * NCELL) : NULL;
  if (!U1 || !U2 || !fb || (lts && !dtc)) { free(U1); free(U2); free(fb); free(dtc); return OR_ENOMEM; }
  double t = 0.0, dt = fixed_dt;
  long nfb = 0;
  for (int s = 0; s < nsteps; s++) {
    if (cfl > 0.0) {
      double smax;
      rc = or_cfl_smax(d, U, &smax);
      if (rc) break;
      dt = cfl / smax;
      if (lts) rc = or_local_dt(d, U, cfl, dtc);
      if (rc) break;
    }
    /* with local time stepping the stage coefficients are beta * dt_i */
    const double f = lts ? 1.0 : dt;
    const int nst = d->rk == RK_EULER ? 1 : 2;
    /* the first of two stages without the correction when it is applied in the last stage only */
    or_desc first = *d;
    if (d->learned_last_only && nst == 2) first.learned = 0;
    for (int st = 0; st < nst && !rc; st++) {
      if (d->rk == RK_EULER) rc = or_stage_ex(d, U, U, U2, 0, f, dtc, fb);
      else if (d->rk == RK_SSP2)
        rc = st == 0 ? or_stage_ex(&first, U, U, U1, 0, f, dtc, fb) : or_stage_ex(d, U1, U, U2, 1, f, dtc, fb);
      else
        rc = st == 0 ? or_stage_ex(&first, U, U, U1, 0, 0.5 * f, dtc, fb) : or_stage_ex(d, U1, U, U2, 0, f, dtc, fb);
      for (int b = 0; b < nb && !rc; b++) nfb += fb[b];
    }
    if (rc) break;
    memcpy(U, U2, sizeof(double) * n);
    t += dt;
  }
  free(U1);
  free(U2);
  free(fb);
  free(dtc);
  if (dt_last) *dt_last = dt;
  if (t_total) *t_total = t;
  if (n_fallback) *n_fallback = nfb;
  return rc;
}

int or_run(const or_desc* d, double* U, int nsteps, double cfl, double fixed_dt, double* dt_last, double* t_total) {
  return or_run_ex(d, U, nsteps, cfl, fixed_dt, dt_last, t_total, NULL);
}

/* Test hooks for single formulas. */
double or_fast_speed(double gamma, const double W[NV], const double B[3], int dir) {
  return fast_speed(gamma, W, B, dir);
}

void or_prim_from_cons(double gamma, const double* U, double* W, long n) {
  for (long i = 0; i < n; i++) prim_from_cons(gamma, U + 8 * i, W + 8 * i);
}

void or_cons_from_prim(double gamma, const double* W, double* U, long n) {
  for (long i = 0; i < n; i++) cons_from_prim(gamma, W + 8 * i, U + 8 * i);
}

void or_b0_at(const or_desc* d, const double x[3], double B0[3]) { b0_at(d, x, B0); }

double or_limiter(int kind, double a, double b) { return limiter(kind, a, b); }

/* The numerical flux (d->flux) through a face along dir between the face
 * states WL, WR (primitive) with B0 at the face. */
void or_numerical_flux(const or_desc* d, int dir, const double WL[NV], const double WR[NV], const double B0[3],
                       double F[NV]) {
  double FL[NV], FR[NV], UL[NV], UR[NV], unL, unR, cfL, cfR;
  phys_flux(d, dir, WL, B0, FL, UL, &unL, &cfL);
  phys_flux(d, dir, WR, B0, FR, UR, &unR, &cfR);
  numerical_flux(d->flux, dir, d->gamma, WL, WR, FL, FR, UL, UR, unL, unR, cfL, cfR, 1.0, F);
}

/* The same with the Linde flux's restored contact part scaled by `contact`
 * (0: the HLL flux). */
void or_numerical_flux_contact(const or_desc* d, int dir, const double WL[NV], const double WR[NV],
                               const double B0[3], double contact, double F[NV]) {
  double FL[NV], FR[NV], UL[NV], UR[NV], unL, unR, cfL, cfR;
  phys_flux(d, dir, WL, B0, FL, UL, &unL, &cfL);
  phys_flux(d, dir, WR, B0, FR, UR, &unR, &cfR);
  numerical_flux(d->flux, dir, d->gamma, WL, WR, FL, FR, UL, UR, unL, unR, cfL, cfR, contact, F);
}
