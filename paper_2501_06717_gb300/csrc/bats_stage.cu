// bats_stage.cu -- sm_103a kernels of one explicit stage of the ideal-MHD
// finite-volume update (arXiv 2501.06717, Algorithms 1-2; Eqs. 1-5): the
// stage kernel's Rusanov and learned instantiations (the template is in
// bats_stage_kernel.h; bats_stage_flux.cu holds the HLL and Linde ones), the
// mixed form's ghost pre-pass at resolution changes, the layout, CFL, time
// step, refluxing and debug kernels, and their launchers.
#include "bats_stage_kernel.h"

namespace batsk {

// Mixed form: the face-slab ghosts of one face at a resolution change.  The
// tree does not change, so where each ghost's source lies is found once per
// handle (k_amr_ghost_table) and every stage's pre-pass (k_amr_ghosts) reads
// it instead of locating the source again.  Per task and thread one entry:
// the sample of thread k of a COARSER task (k < PSLOTS: coarse sample k of
// the prolongation) or the ghost cell of thread k of a FINER task (its
// restriction), encoded as leaf << 9 | cell (a leaf at the sample's level:
// load its cell), 1 << 30 | leaf << 9 | cell (refined there: restrict the 8
// cells of `leaf` from corner `cell`), -2 (an inflow face: the fixed state),
// -3 (no sample) or -1 (anything else: locate as the generic path does).
constexpr int32_t GT_RESTRICT = 1 << 30, GT_INFLOW = -2, GT_NONE = -3, GT_GENERIC = -1;
__device__ __forceinline__ int ghost_sample(const GhostTask& T, const BlockDev& B, int tid, int g[3]) {
  if (B.ftype[T.s] == FACE_COARSER) return tid < PSLOTS && psample(B, T.s, tid, g) ? B.level - 1 : -1;
  const int d = T.s >> 1, side = T.s & 1;
  const int layer = tid & 1, ta = (tid >> 1) & 7, tb = tid >> 4;
  const int c = side ? NC + layer : layer - 2;
  const int i = d == 0 ? c : ta, j = d == 1 ? c : (d == 0 ? ta : tb), k = d == 2 ? c : tb;
  g[0] = B.bi * NC + i;
  g[1] = B.bj * NC + j;
  g[2] = B.bk * NC + k;
  return B.level;
}
__global__ void __launch_bounds__(128) k_amr_ghost_table(const StageArgs a, const GhostTask* __restrict__ tasks,
                                                         int32_t* __restrict__ tab) {
  const GhostTask T = tasks[blockIdx.x];
  const BlockDev& B = a.blocks[chki(T.blk, 0, a.nblocks)];
  const GridDev& G = a.grids[B.grid];
  const int tid = threadIdx.x;
  int g[3];
  const int lev = ghost_sample(T, B, tid, g);
  int32_t e = GT_NONE;
  if (lev >= 0) {
    e = GT_GENERIC;
    int ll;
    if (bc_map(G, lev, g)) {
      e = GT_INFLOW;
    } else {
      const int leaf = locate(G, a.levmap, lev, g, ll);
      if (leaf >= 0 && ll == lev) {
        const BlockDev& L = a.blocks[leaf];
        const int li = g[0] - L.bi * NC, lj = g[1] - L.bj * NC, lk = g[2] - L.bk * NC;
        if (li >= 0 && li < NC && lj >= 0 && lj < NC && lk >= 0 && lk < NC && leaf < (1 << 21))
          e = leaf << 9 | ((lk * NC + lj) * NC + li);
      } else if (leaf < 0) {
        const int f[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
        const int fl = locate(G, a.levmap, lev + 1, f, ll);
        if (fl >= 0 && ll == lev + 1) {
          const BlockDev& L = a.blocks[fl];
          const int li = f[0] - L.bi * NC, lj = f[1] - L.bj * NC, lk = f[2] - L.bk * NC;
          if (li >= 0 && li < NC - 1 && lj >= 0 && lj < NC - 1 && lk >= 0 && lk < NC - 1 && fl < (1 << 21))
            e = GT_RESTRICT | fl << 9 | ((lk * NC + lj) * NC + li);
        }
      }
    }
  }
  tab[static_cast<int64_t>(blockIdx.x) * 128 + tid] = e;
}
// The sample of entry e (the generic point location for GT_GENERIC).
__device__ __forceinline__ void ghost_sample_w(const StageArgs& a, const GridDev& G, int32_t e, int lev, int g[3],
                                               float w[8]) {
  if (e >= 0) {
    const float* p = a.Win + static_cast<int64_t>((e & (GT_RESTRICT - 1)) >> 9) * (NV * NCELL) + (e & 511);
    if (e & GT_RESTRICT) {
      restrict_at(p, a.ph.gm1f, w);
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = p[v * NCELL];
    }
  } else if (e == GT_INFLOW) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = G.Winflow32[v];
  } else {
    sample_w(a.Win, G, a.blocks, a.levmap, lev, g, a.ph.gm1f, w, a.err);
  }
}

// One CTA of 128 threads per face, one ghost cell per thread, into
// gbuf[slot].  Coarser neighbour: the coarse samples into a shared table,
// then every fine ghost cell by the prolongation; finer neighbour: the
// restriction of each ghost cell's 8 children.
__global__ void __launch_bounds__(128) k_amr_ghosts(const StageArgs a, const GhostTask* __restrict__ tasks,
                                                    const int32_t* __restrict__ gtab) {
  __shared__ float tab[PSLOTS * PSTRIDE];
  const GhostTask T = tasks[blockIdx.x];
  const int tid = threadIdx.x;
  const int32_t ent = gtab[static_cast<int64_t>(blockIdx.x) * 128 + tid];
  const BlockDev& B = a.blocks[chki(T.blk, 0, a.nblocks)];
  const GridDev& G = a.grids[B.grid];
  float w[8];
  int g[3];
  if (B.ftype[T.s] == FACE_COARSER) {
    if (ent != GT_NONE) {
      const int lev = ghost_sample(T, B, tid, g);
      float ws[8], u[8];
      ghost_sample_w(a, G, ent, lev, g, ws);
      cons_from_prim<float>(ws, a.ph.inv_gm1f, u);
      float* e = tab + chki(tid, 0, PSLOTS) * PSTRIDE;
#pragma unroll
      for (int v = 0; v < NV; v++) e[v] = u[v];
      e[8] = ws[7];
      e[9] = ws[1];
      e[10] = ws[2];
      e[11] = ws[3];
    }
    __syncthreads();
    prolong_child_w(tab, T.s, tid, a.ph.gm1f, w);
  } else {
    const int lev = ghost_sample(T, B, tid, g);
    ghost_sample_w(a, G, ent, lev, g, w);
  }
  // slot layout: the generic tile's slab order [8][128] (layer fastest), or
  // the staged tile's slab layout of this face's axis
  const int d = T.s >> 1, side = T.s & 1;
  const int layer = tid & 1, ta = (tid >> 1) & 7, tb = tid >> 4;
  const int e = a.gbuf_mx ? mx_slab_elem(d, side, side ? NC + layer : layer - 2, ta, tb) : tid;
  const int vs = a.gbuf_mx ? mx_slab_vstride(d) : 128;
  float* o = a.gbuf + chk(T.slot, 0, a.nslots) * GSLOT + chki(e, 0, vs);
#pragma unroll
  for (int v = 0; v < NV; v++) o[v * vs] = w[v];
}

// ---------------------------------------------------------------------------
// The fused stage kernel.

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
                      const BlockDev* blocks, PhysDev ph, int b0, unsigned long long* smax, double* dtc, double cfl) {
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
  // local time stepping: the cell's own dt (0 in the body)
  if (dtc) dtc[static_cast<int64_t>(blk) * NCELL + c] = in_body ? 0.0 : cfl / s;
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((c & 31) == 0) sred[c >> 5] = s;
  __syncthreads();
  if (c == 0) {
    double m = 0.0;
    for (int w = 0; w < NCELL / 32; w++) m = fmax(m, sred[w]);
    if (m > 0.0) atomicMax(&smax[B.grid], static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// Refluxing after a stage.  One CTA per corrected block, one thread per face
// position (q, r) of a refined face: the coarse cell next to it trades its own
// face flux for the mean of the 4 fine fluxes through the face (summed in the
// oracle's order), i.e. its stage update gains c * dR with
// dR = -+ (mean - F_coarse) / dx.  Faces are taken one at a time (a cell on an
// edge of two refined faces gets both corrections in turn); in the last stage
// the corrected cells' CFL bounds follow from the final state.
__device__ __forceinline__ void reflux_cell(const StageArgs& a, const RefluxTask& T, int tid, int& c, bool& in_body) {
  const BlockDev& B = a.blocks[T.blk];
  const GridDev& G = a.grids[B.grid];
  const int d = T.s >> 1, side = T.s & 1;
  const int q = tid >> 3, r = tid & 7;
  int cc[3];
  cc[d] = side ? NC - 1 : 0;
  cc[d == 0 ? 1 : 0] = q;
  cc[d == 2 ? 1 : 2] = r;
  c = (cc[2] * NC + cc[1]) * NC + cc[0];
  in_body = false;
  if (B.body) {
    const int lev = B.level;
    double x = G.lo[0] + ((static_cast<double>(B.bi * NC) + cc[0]) + 0.5) * G.dx[lev][0];
    double y = G.lo[1] + ((static_cast<double>(B.bj * NC) + cc[1]) + 0.5) * G.dx[lev][1];
    double z = G.lo[2] + ((static_cast<double>(B.bk * NC) + cc[2]) + 0.5) * G.dx[lev][2];
    in_body = (x * x + y * y + z * z) < G.body_r * G.body_r;
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(64) k_reflux(const StageArgs a, const RefluxTask* __restrict__ tasks,
                                               const int32_t* __restrict__ rblocks) {
  const int first = rblocks[2 * blockIdx.x], cnt = rblocks[2 * blockIdx.x + 1];
  const int tid = threadIdx.x;
  const PhysDev& ph = a.ph;
  for (int t = first; t < first + cnt; t++) {
    const RefluxTask T = tasks[t];
    const BlockDev& B = a.blocks[T.blk];
    const GridDev& G = a.grids[B.grid];
    int c;
    bool in_body;
    reflux_cell(a, T, tid, c, in_body);
    if (!in_body) {
      const int d = T.s >> 1, side = T.s & 1;
      const int q = tid >> 3, r = tid & 7;
      const double* Fc = a.freg + (chk(T.cslot, 0, a.nslots) * 64 + tid) * NV;
      const double* Ff = a.freg + chk(T.fslot[(q >> 2) + 2 * (r >> 2)], 0, a.nslots) * 64 * NV;
      const int qf = 2 * (q & 3), rf = 2 * (r & 3);
      const double idx_d = G.idx[B.level][d];
      double dR[8];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const double f00 = Ff[(qf * NC + rf) * NV + v], f10 = Ff[((qf + 1) * NC + rf) * NV + v];
        const double f01 = Ff[(qf * NC + rf + 1) * NV + v], f11 = Ff[((qf + 1) * NC + rf + 1) * NV + v];
        const double dF = 0.25 * ((f00 + f10) + (f01 + f11)) - Fc[v];
        dR[v] = (side ? -dF : dF) * idx_d;
      }
      const int64_t cell = static_cast<int64_t>(T.blk) * NCELL + c;
      const int64_t base = static_cast<int64_t>(T.blk) * (NV * NCELL) + c;
      const double cdt = a.beta * (a.dtc ? a.dtc[cell] : a.dt[B.grid]);
      bool bad = false;
      if (MIXED && !(a.last || a.write_u_all)) {
        // first midpoint stage of the mixed form: only W* exists
        float Wo[8], dU[8], Wn[8];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          Wo[v] = a.Wout[base + v * NCELL];
          dU[v] = d2f_int(cdt * dR[v]);
        }
        prim_increment(Wo, dU, ph.gm1f, Wn);
        bad = !(Wn[0] > 0.f) || !(Wn[7] > 0.f);
#pragma unroll
        for (int v = 0; v < NV; v++) {
          bad |= !finite_f(Wn[v]);
          a.Wout[base + v * NCELL] = Wn[v];
        }
      } else {
        double Uo[8];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          double u = a.Uout[base + v * NCELL];
          u = a.kind == 1 ? u + 0.5 * (cdt * dR[v]) : fma(cdt, dR[v], u);
          Uo[v] = u;
          a.Uout[base + v * NCELL] = u;
          bad |= !finite_d(u);
        }
        bad |= !positive_d(Uo[0]);
        if constexpr (MIXED) {
          float Wn[8];
          double p64;
          prim_mixed(Uo, ph.gm1f, Wn, &p64);
          bad |= !positive_d(p64);
#pragma unroll
          for (int v = 0; v < NV; v++) a.Wout[base + v * NCELL] = Wn[v];
        } else {
          double Wn[8];
          prim64(Uo, ph.gm1, Wn);
          bad |= !positive_d(Wn[7]);
        }
      }
      if (bad) {
        atomicOr(&a.err[0], ERR_NONPHYSICAL);
        atomicMin(&a.err[1], T.blk);
      }
    }
    __syncthreads();
  }
  if (!a.last) return;
  // CFL bounds (and local dt) of the corrected cells, as in the stage epilogue
  for (int t = first; t < first + cnt; t++) {
    const RefluxTask T = tasks[t];
    const BlockDev& B = a.blocks[T.blk];
    const GridDev& G = a.grids[B.grid];
    int c;
    bool in_body;
    reflux_cell(a, T, tid, c, in_body);
    if (in_body) continue;
    const int ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;
    const int lev = B.level;
    const int gb0 = B.bi * NC, gb1 = B.bj * NC, gb2 = B.bk * NC;
    const int64_t base = static_cast<int64_t>(T.blk) * (NV * NCELL) + c;
    double md;
    if constexpr (MIXED) {
      float Wn[8], B0c[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int v = 0; v < NV; v++) Wn[v] = a.Wout[base + v * NCELL];
      if (ph.b0 != B0_NONE)
        b0_face<float>(ph, -1, ci, cj, ck, gb0, gb1, gb2, G.lof[0], G.lof[1], G.lof[2], G.dxf[lev][0],
                       G.dxf[lev][1], G.dxf[lev][2], B0c);
      const float Bt[3] = {B0c[0] + Wn[4], B0c[1] + Wn[5], B0c[2] + Wn[6]};
      float sacc = 0.f;
#pragma unroll
      for (int e = 0; e < 3; e++) {
        const float cf = fast_speed_n<float>(ph.gammaf, Wn[0], Wn[7], Bt[e], Bt[(e + 1) % 3], Bt[(e + 2) % 3]);
        sacc = sacc + (fabsf(Wn[1 + e]) + cf) * G.idxf[lev][e];
      }
      md = f2d_int(sacc);
    } else {
      double U[8], Wn[8], B0c[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int v = 0; v < NV; v++) U[v] = a.Uout[base + v * NCELL];
      prim64(U, ph.gm1, Wn);
      if (ph.b0 != B0_NONE)
        b0_face<double>(ph, -1, ci, cj, ck, gb0, gb1, gb2, G.lo[0], G.lo[1], G.lo[2], G.dx[lev][0], G.dx[lev][1],
                        G.dx[lev][2], B0c);
      const double Bt[3] = {B0c[0] + Wn[4], B0c[1] + Wn[5], B0c[2] + Wn[6]};
      double sacc = 0.0;
#pragma unroll
      for (int e = 0; e < 3; e++) {
        const double cf = fast_speed_exact(ph.gamma, Wn[0], Wn[7], Bt[e], Bt[(e + 1) % 3], Bt[(e + 2) % 3]);
        sacc = sacc + (fabs(Wn[1 + e]) + cf) / G.dx[lev][e];
      }
      md = sacc;
    }
    if (md > 0.0) atomicMax(&a.smax_next[B.grid], static_cast<unsigned long long>(__double_as_longlong(md)));
    if (a.dtc) a.dtc[static_cast<int64_t>(T.blk) * NCELL + c] = a.cfl / md;
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

// Padded tiles [8][nb][12][12][12] (external layout) of the shared-memory
// tile of block blockIdx.x: the interior and the face slabs; edge and corner
// cells are 0.
template <class R>
__device__ void write_debug_tile(const R* sT, int nb, double* T) {
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
      T[(static_cast<int64_t>(v) * nb + blockIdx.x) * tile + e] = t >= 0 ? static_cast<double>(sT[v * NTILE + t]) : 0.0;
  }
}

// Debug view of the ghost fill of blocks [b0, b0+nb), filled by the same code
// as the stage kernel: FP64 form, conservative variables.
__global__ void k_debug_fill(const StageArgs a, int b0, int nb, double* T) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* sT = reinterpret_cast<double*>(smem_raw);
  const int blk = b0 + blockIdx.x;
  const BlockDev& B = a.blocks[blk];
  GhostCtx cx{&a.grids[B.grid], a.blocks, a.levmap, a.Uin, a.err};
  for (int e = threadIdx.x; e < NV * NCELL; e += blockDim.x)
    sT[(e / NCELL) * NTILE + (e % NCELL)] = a.Uin[static_cast<int64_t>(blk) * NV * NCELL + e];
  fill_ghosts_block<false, double>(a, cx, B, blk, sT, sT + NV * NTILE, threadIdx.x, blockDim.x);
  __syncthreads();
  write_debug_tile(sT, nb, T);
}

// The same for the mixed form: FP32 primitives from W.
constexpr size_t kDebugFillWSmem = sizeof(float) * NV * NTILE;
__global__ void k_debug_fill_w(const StageArgs a, int b0, int nb, double* T) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sT = reinterpret_cast<float*>(smem_raw);
  const int blk = b0 + blockIdx.x;
  const BlockDev& B = a.blocks[blk];
  GhostCtx cx{&a.grids[B.grid], a.blocks, a.levmap, a.Uin, a.err};
  for (int e = threadIdx.x; e < NV * NCELL; e += blockDim.x)
    sT[(e / NCELL) * NTILE + (e % NCELL)] = a.Win[static_cast<int64_t>(blk) * NV * NCELL + e];
  fill_ghosts_block_mixed(a, cx, B, blk, sT, threadIdx.x, blockDim.x, true);
  __syncthreads();
  write_debug_tile(sT, nb, T);
}

// The same for the mixed plain kernel's staged tile: block blockIdx.x staged
// exactly as the stage kernel stages it (tensor copies or thread gathers, as
// stage_tma says, and the precomputed slabs of faces at resolution changes),
// then written out through the tile's layout.
constexpr size_t kDebugFillMxSmem = sizeof(float) * MX_TILE + 1024;
__global__ void k_debug_fill_mx(const __grid_constant__ StageArgs a, int b0, int nb, double* T) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  float* sT = reinterpret_cast<float*>(smem_raw + pad);
  const int blk = b0 + blockIdx.x;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  mx_stage_tile(a, a.blocks[blk], blk, sT, &bar, threadIdx.x, blockDim.x);
  if (!mbar_wait_bounded(&bar, 0, a.err)) mbar_wait_bounded(&bar, 0, a.err);
  __syncthreads();
  const int tile = 12 * 12 * 12;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int i = e % 12 - 2, j = (e / 12) % 12 - 2, k = e / 144 - 2;
    const int oi = (i < 0 || i >= NC), oj = (j < 0 || j >= NC), ok = (k < 0 || k >= NC);
    int t = -1, vs = 0;
    if (oi + oj + ok == 0) {
      t = mx_int(i, j, k);
      vs = NCELL;
    } else if (oi + oj + ok == 1) {
      const int d = oi ? 0 : (oj ? 1 : 2);
      const int c = d == 0 ? i : (d == 1 ? j : k);
      const int ta = d == 0 ? j : i, tb = d == 2 ? j : k;
      const int side = c >= NC ? 1 : 0;
      t = mx_slab_base(2 * d + side) + mx_slab_elem(d, side, c, ta, tb);
      vs = mx_slab_vstride(d);
    }
    for (int v = 0; v < NV; v++)
      T[(static_cast<int64_t>(v) * nb + blockIdx.x) * tile + e] = t >= 0 ? static_cast<double>(sT[t + v * vs]) : 0.0;
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
// dynamic shared memory of a stage kernel: the mixed plain kernel stages
// its own tile layout
static size_t stage_smem(bool mixed, bool lrn) {
  return mixed ? (lrn ? kSmemLx : StageCfg<true>::SMEM_MX) : StageCfg<false>::SMEM;
}

using StageFn = void (*)(const StageArgs);
template <bool MIXED, bool LRN, int FLX>
StageFn stage_fn_l(int lim, bool b0) {
  if (lim == 2) return b0 ? k_stage<MIXED, 2, true, LRN, FLX> : k_stage<MIXED, 2, false, LRN, FLX>;
  if (lim == 1) return b0 ? k_stage<MIXED, 1, true, LRN, FLX> : k_stage<MIXED, 1, false, LRN, FLX>;
  return b0 ? k_stage<MIXED, 0, true, LRN, FLX> : k_stage<MIXED, 0, false, LRN, FLX>;
}
// The learned correction is defined on the Rusanov flux only (the host rejects
// learned + HLL or Linde), so the other fluxes are instantiated for the plain
// kernels only, in bats_stage_flux.cu.
StageFn stage_fn_flux(bool mixed, int lim, bool b0, int flux);
cudaError_t read_index_flag_flux(int32_t* out);
template <bool MIXED>
StageFn stage_fn(int lim, bool b0, bool lrn = false, int flux = FLUX_RUSANOV) {
  if (lrn) return stage_fn_l<MIXED, true, FLUX_RUSANOV>(lim, b0);
  if (flux != FLUX_RUSANOV) return stage_fn_flux(MIXED, lim, b0, flux);
  return stage_fn_l<MIXED, false, FLUX_RUSANOV>(lim, b0);
}

cudaError_t stage_setup(int occ[2]) {
  cudaError_t e = cudaSuccess;
  for (int lim = 0; lim < 3 && e == cudaSuccess; lim++)
    for (int b0 = 0; b0 < 2 && e == cudaSuccess; b0++)
      for (int kv = 0; kv < 4 && e == cudaSuccess; kv++) {  // Rusanov, learned, HLL, Linde
        const bool lrn = kv == 1;
        const int flux = kv == 2 ? FLUX_HLL : (kv == 3 ? FLUX_LINDE : FLUX_RUSANOV);
        e = cudaFuncSetAttribute(stage_fn<false>(lim, b0, lrn, flux), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(StageCfg<false>::SMEM));
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(stage_fn<true>(lim, b0, lrn, flux), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(stage_smem(true, lrn)));
      }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_debug_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(double) * (NV * NTILE + 3 * 128 * NV)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_debug_fill_w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kDebugFillWSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_debug_fill_mx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kDebugFillMxSmem));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], stage_fn<false>(0, false), StageCfg<false>::THREADS,
                                                      StageCfg<false>::SMEM);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], stage_fn<true>(0, false), StageCfg<true>::THREADS,
                                                      stage_smem(true, false));
  return e;
}

cudaError_t launch_stage_kernel(bool mixed, int grid, cudaStream_t st, const StageArgs& a) {
  const bool b0 = a.ph.b0 != B0_NONE;
  const bool lrn = a.learned || a.kind >= 3;
  const int flux = a.ph.flux;
  if (mixed)
    stage_fn<true>(a.ph.limiter, b0, lrn, flux)<<<grid, StageCfg<true>::THREADS, stage_smem(true, lrn), st>>>(a);
  else
    stage_fn<false>(a.ph.limiter, b0, lrn, flux)<<<grid, StageCfg<false>::THREADS, StageCfg<false>::SMEM, st>>>(a);
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
cudaError_t launch_cfl_dt(bool mixed, const double* U, const float* Wt, const GridDev* grids,
                          const BlockDev* blocks, const PhysDev& ph, int b0, int nb, unsigned long long* smax,
                          double* dtc, double cfl, cudaStream_t st) {
  if (mixed) k_cfl<true><<<nb, NCELL, 0, st>>>(U, Wt, grids, blocks, ph, b0, smax, dtc, cfl);
  else k_cfl<false><<<nb, NCELL, 0, st>>>(U, Wt, grids, blocks, ph, b0, smax, dtc, cfl);
  return cudaGetLastError();
}
cudaError_t launch_amr_ghost_table(const StageArgs& a, const GhostTask* tasks, int32_t* gtab, int ntasks,
                                   cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  k_amr_ghost_table<<<ntasks, 128, 0, st>>>(a, tasks, gtab);
  return cudaGetLastError();
}
cudaError_t launch_amr_ghosts(const StageArgs& a, const GhostTask* tasks, const int32_t* gtab, int ntasks,
                              cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  k_amr_ghosts<<<ntasks, 128, 0, st>>>(a, tasks, gtab);
  return cudaGetLastError();
}
cudaError_t launch_reflux(bool mixed, const StageArgs& a, const RefluxTask* tasks, const int32_t* rblocks, int nrb,
                          cudaStream_t st) {
  if (nrb <= 0) return cudaSuccess;
  if (mixed) k_reflux<true><<<nrb, 64, 0, st>>>(a, tasks, rblocks);
  else k_reflux<false><<<nrb, 64, 0, st>>>(a, tasks, rblocks);
  return cudaGetLastError();
}
cudaError_t launch_cfl(bool mixed, const double* U, const float* Wt, const GridDev* grids, const BlockDev* blocks,
                       const PhysDev& ph, int b0, int nb, unsigned long long* smax, cudaStream_t st) {
  return launch_cfl_dt(mixed, U, Wt, grids, blocks, ph, b0, nb, smax, nullptr, 0.0, st);
}
cudaError_t launch_dt(int ngrids, int mode, double cfl, double fixed_dt, double* dt, double* t,
                      unsigned long long* smax, unsigned long long* smax_next, cudaStream_t st) {
  k_dt<<<(ngrids + 127) / 128, 128, 0, st>>>(ngrids, mode, cfl, fixed_dt, dt, t, smax, smax_next);
  return cudaGetLastError();
}
cudaError_t launch_debug_fill(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st) {
  k_debug_fill<<<nb, 256, sizeof(double) * (NV * NTILE + 3 * 128 * NV), st>>>(a, b0, nb, T);
  return cudaGetLastError();
}
cudaError_t launch_debug_fill_w(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st) {
  k_debug_fill_w<<<nb, 256, kDebugFillWSmem, st>>>(a, b0, nb, T);
  return cudaGetLastError();
}
cudaError_t launch_debug_fill_mx(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st) {
  k_debug_fill_mx<<<nb, 256, kDebugFillMxSmem, st>>>(a, b0, nb, T);
  return cudaGetLastError();
}
// Checked build: read and clear the index-check flag (always 0 otherwise).
cudaError_t read_index_flag(int32_t* out) {
#ifdef BATS_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(out, g_index_err, sizeof(int32_t));
  const int32_t zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_index_err, &zero, sizeof(int32_t));
  int32_t other = 0;  // the flag of the HLL and Linde kernels' module
  if (e == cudaSuccess) e = read_index_flag_flux(&other);
  *out |= other;
  return e;
#else
  *out = 0;
  return cudaSuccess;
#endif
}

// Bounded-wait test hook: one thread waits on an mbarrier that nothing
// arrives at; after the wait's limit it records ERR_TIMEOUT and returns.
__global__ void k_debug_wait_timeout(int32_t* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_wait_bounded(&bar, 0, err);
  }
}
cudaError_t launch_debug_wait_timeout(int32_t* err, cudaStream_t st) {
  k_debug_wait_timeout<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

// FP64 FMA throughput probe (the FP64 form's roofline): every thread runs
// `iters` rounds of eight independent FMA chains x = x * b + c, so that the
// FP64 pipe's issue rate, not an FMA's latency, sets the time.  The chains'
// sum is stored only in the (never taken) case that it equals `never`,
// which keeps all of them live.
__global__ void __launch_bounds__(256) k_fp64_fma_rate(double* out, int iters, double b, double c, double never) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = fma(x[k], b, c);
  }
  double s = ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
  if (s == never) out[0] = s;
}
cudaError_t launch_fp64_fma_rate(double* out, int ctas, int iters, cudaStream_t st) {
  k_fp64_fma_rate<<<ctas, 256, 0, st>>>(out, iters, 0.9999999, 1e-7, -1.0);
  return cudaGetLastError();
}

cudaError_t launch_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out) {
  k_check_conversions<<<(n + 255) / 256, 256>>>(f, d, n, f2d_out, d2f_out);
  return cudaGetLastError();
}

}  // namespace batsk
