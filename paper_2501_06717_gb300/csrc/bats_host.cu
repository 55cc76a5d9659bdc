// bats_host.cu -- host side of libbats: the C ABI of include/bats.h, tree
// validation (exact tiling, 2:1 balance across faces, edges and corners,
// through periodic wraps), the per-block neighbour table and per-level block
// maps built once per grid on the host and uploaded (the memory-map idea of
// arXiv 2501.06717 Section 4.4 applied to the on-device ghost exchange), and
// the launch sequence of a time step.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bats.h"
#include "bats_internal.h"

namespace batsk {

// launchers defined next to the kernels (bats_stage.cu)
size_t stage_smem_bytes(bool mixed);
cudaError_t stage_setup(int occ[2]);
cudaError_t launch_stage_kernel(bool mixed, int grid, cudaStream_t st, const StageArgs& a);
cudaError_t launch_to_internal(const double* ext, double* in, int block0, int nb, cudaStream_t st);
cudaError_t launch_to_external(const double* in, double* ext, int block0, int nb, cudaStream_t st);
cudaError_t launch_init_grid_states(GridDev* grids, int ngrids, double inv_gm1, double gm1, cudaStream_t st);
cudaError_t launch_prim_mixed(const double* U, float* Wt, int b0, int nb, float gm1f, cudaStream_t st);
cudaError_t launch_cfl(bool mixed, const double* U, const float* Wt, const GridDev* grids, const BlockDev* blocks,
                       const PhysDev& ph, int b0, int nb, unsigned long long* smax, cudaStream_t st);
cudaError_t launch_amr_ghosts(const StageArgs& a, const GhostTask* tasks, const int32_t* gtab, int ntasks,
                              cudaStream_t st);
cudaError_t launch_amr_ghost_table(const StageArgs& a, const GhostTask* tasks, int32_t* gtab, int ntasks,
                                   cudaStream_t st);
cudaError_t launch_reflux(bool mixed, const StageArgs& a, const RefluxTask* tasks, const int32_t* rblocks, int nrb,
                          cudaStream_t st);
cudaError_t launch_cfl_dt(bool mixed, const double* U, const float* Wt, const GridDev* grids,
                          const BlockDev* blocks, const PhysDev& ph, int b0, int nb, unsigned long long* smax,
                          double* dtc, double cfl, cudaStream_t st);
cudaError_t launch_dt(int ngrids, int mode, double cfl, double fixed_dt, double* dt, double* t,
                      unsigned long long* smax, unsigned long long* smax_next, cudaStream_t st);
cudaError_t launch_debug_fill(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st);
cudaError_t launch_debug_fill_w(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st);
cudaError_t launch_debug_fill_mx(const StageArgs& a, int b0, int nb, double* T, cudaStream_t st);
cudaError_t launch_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out);
cudaError_t launch_fp64_fma_rate(double* out, int ctas, int iters, cudaStream_t st);
cudaError_t read_index_flag(int32_t* out);
cudaError_t launch_debug_wait_timeout(int32_t* err, cudaStream_t st);
cudaError_t mlp_alloc(MlpDev* w);
cudaError_t mlp_setup();
void mlp_free(MlpDev* w);
cudaError_t launch_mlp_pack(const float* P, const MlpDev& m, cudaStream_t st);
cudaError_t launch_mlp_infer(const uint32_t* X, float* Y, int64_t n, const MlpDev& m, int nsm, int32_t* err,
                             cudaStream_t st);

}  // namespace batsk

using namespace batsk;

struct bats {
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int ngrids = 0, nbt = 0, num_sms = 0;
  std::vector<GridDev> grids_h;
  std::vector<BlockDev> blocks_h;
  std::vector<int32_t> levmap_h;
  PhysDev ph{};
  GridDev* grids_d = nullptr;
  BlockDev* blocks_d = nullptr;
  int32_t* levmap_d = nullptr;
  double *U = nullptr, *U1 = nullptr;
  float *W = nullptr, *W1 = nullptr;
  double *dt = nullptr, *t = nullptr;
  unsigned long long *smax = nullptr, *smax_next = nullptr;
  int32_t* errw = nullptr;
  double* staging = nullptr;
  size_t staging_n = 0;
  int persistent = 0, bpc = 1, ctas_per_sm = 0, use_graph = 0;
  int local_dt = 0;
  double* dtc = nullptr;  // local time stepping: per-cell dt [nbt][512]
  // refluxing
  int reflux = 0, nslots = 0;
  std::vector<RefluxTask> rtasks_h;
  std::vector<int32_t> rblocks_h;        // per corrected block: first task, task count
  double* freg = nullptr;
  RefluxTask* rtasks_d = nullptr;
  int32_t* rblocks_d = nullptr;
  // mixed form: ghost slabs of faces at resolution changes, computed ahead of each stage
  std::vector<GhostTask> gtasks_h;
  GhostTask* gtasks_d = nullptr;
  int32_t* gtab_d = nullptr;   // where each pre-pass thread's sample lies (built once per handle)
  float* gbuf = nullptr;
  // mixed form: tensor maps of W and W1 for the plain stage kernel's tile
  // staging (interior, x, y, z slab boxes), and the staging layout
  CUtensorMap tmW[4], tmW1[4];
  int stage_tma = 1;
  int occ[2] = {1, 1};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> stage_ev;   // pairs around the two stage launches of each step
  int timed_steps = 0;
  double ms_last[BATS_NUM_PHASES] = {0, 0, 0};
  long long launches = 0;
  long long fallbacks = 0;  // learned block-stages recomputed with the plain flux
  cudaGraphExec_t graph = nullptr;
  int graph_n = -1;
  double graph_cfl = 0, graph_dt = 0;
  long long graph_launches = 0;
  int graph_timed = 0;                 // steps whose stage events the graph records
  // learned form
  bool learned_requested = false, learned = false;
  bool learned_last_only = false;  // the correction in the last stage of a step only
  MlpDev mlp{};
  float* mlp_params = nullptr;
  uint32_t* Xb = nullptr;   // BF16 network inputs of every face
  float* Yb = nullptr;      // network outputs of every face
};

static std::string g_create_error;

static int fail(bats_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}
static int cuda_fail(bats_t* h, cudaError_t e, const char* what) {
  return fail(h, BATS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(h, call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// Grid construction (host).

namespace {

struct HostGrid {
  const bats_grid_desc* d;
  int maxlev = 0;
  std::vector<std::vector<int32_t>> map;  // per level, dense block map (local leaf index or -1)
  int64_t nblk(int l, int a) const { return static_cast<int64_t>(d->root[a]) << l; }
  int32_t at(int l, int64_t i, int64_t j, int64_t k) const {
    if (l < 0 || l > maxlev) return -1;
    return map[l][(k * nblk(l, 1) + j) * nblk(l, 0) + i];
  }
};

// Covering leaf of block position p (level l): returns local leaf index and
// its level (l or coarser), or -1 if the region is refined.
int cover(const HostGrid& H, int l, const int64_t p[3], int& lev_out) {
  for (int lc = l; lc >= 0; lc--) {
    int sh = l - lc;
    int32_t id = H.at(lc, p[0] >> sh, p[1] >> sh, p[2] >> sh);
    if (id >= 0) { lev_out = lc; return id; }
  }
  lev_out = l + 1;
  return -1;
}

int build_grid(bats_t* h, const bats_grid_desc& d, int gidx, int block0, std::vector<BlockDev>& blocks,
               GridDev& gd, std::vector<int32_t>& levmap) {
  if (d.n_leaves <= 0 || !d.leaves) return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": no leaves");
  for (int a = 0; a < 3; a++) {
    if (d.root[a] <= 0 || !(d.hi[a] > d.lo[a]))
      return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": bad root or extent");
    for (int s = 0; s < 2; s++)
      if (d.bc[2 * a + s] < 0 || d.bc[2 * a + s] > 2)
        return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": bad boundary code");
    if ((d.bc[2 * a] == BATS_BC_PERIODIC) != (d.bc[2 * a + 1] == BATS_BC_PERIODIC))
      return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": periodic on one side only");
  }
  HostGrid H;
  H.d = &d;
  for (int b = 0; b < d.n_leaves; b++) {
    int l = d.leaves[4 * b];
    if (l < 0 || l > MAXLEV) return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": level out of range");
    H.maxlev = std::max(H.maxlev, l);
  }
  H.map.resize(H.maxlev + 1);
  for (int l = 0; l <= H.maxlev; l++) {
    int64_t n = H.nblk(l, 0) * H.nblk(l, 1) * H.nblk(l, 2);
    if (n > (int64_t(1) << 31)) return fail(h, BATS_ERR_INVALID_ARG, "grid too large");
    H.map[l].assign(static_cast<size_t>(n), -1);
  }
  long double vol = 0;
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    for (int a = 0; a < 3; a++)
      if (L[1 + a] < 0 || L[1 + a] >= H.nblk(L[0], a))
        return fail(h, BATS_ERR_INVALID_ARG, "grid " + std::to_string(gidx) + ": leaf outside the domain");
    int64_t m = (static_cast<int64_t>(L[3]) * H.nblk(L[0], 1) + L[2]) * H.nblk(L[0], 0) + L[1];
    if (H.map[L[0]][m] >= 0) return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": duplicate leaf");
    H.map[L[0]][m] = b;
    vol += std::ldexp(1.0L, -3 * L[0]);
  }
  if (vol != static_cast<long double>(d.root[0]) * d.root[1] * d.root[2])
    return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": leaves do not tile the domain");
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    for (int lc = L[0] - 1; lc >= 0; lc--) {
      int sh = L[0] - lc;
      if (H.at(lc, L[1] >> sh, L[2] >> sh, L[3] >> sh) >= 0)
        return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": nested leaves");
    }
  }
  // neighbour relations through the 26 directions, 2:1 balance, face table
  blocks.resize(block0 + d.n_leaves);
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    int l = L[0];
    BlockDev B{};
    B.grid = gidx;
    B.level = l;
    B.bi = L[1];
    B.bj = L[2];
    B.bk = L[3];
    for (int f = 0; f < 6; f++) B.rslot[f] = -1;
    for (int dk = -1; dk <= 1; dk++)
      for (int dj = -1; dj <= 1; dj++)
        for (int di = -1; di <= 1; di++) {
          if (!di && !dj && !dk) continue;
          int dd[3] = {di, dj, dk};
          int64_t p[3] = {L[1] + di, L[2] + dj, L[3] + dk};
          int outside_axis = -1, outside_side = 0;
          bool off = false;
          for (int a = 0; a < 3; a++) {
            int64_t n = H.nblk(l, a);
            if (p[a] < 0 || p[a] >= n) {
              if (d.bc[2 * a] == BATS_BC_PERIODIC) p[a] = (p[a] % n + n) % n;
              else { off = true; outside_axis = a; outside_side = p[a] < 0 ? 0 : 1; }
            }
          }
          int nz = (di != 0) + (dj != 0) + (dk != 0);
          int face = -1;
          if (nz == 1) face = di ? (di < 0 ? 0 : 1) : dj ? (dj < 0 ? 2 : 3) : (dk < 0 ? 4 : 5);
          if (off) {
            if (face >= 0) {
              int bc = d.bc[2 * outside_axis + outside_side];
              B.ftype[face] = bc == BATS_BC_INFLOW ? FACE_INFLOW : FACE_OUTFLOW;
              B.fnb[face] = -1;
            }
            continue;
          }
          int lc;
          int id = cover(H, l, p, lc);
          if (id >= 0) {
            if (lc < l - 1)
              return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": neighbours differ by more than one level");
            if (face >= 0) {
              B.ftype[face] = lc == l ? FACE_SAME : FACE_COARSER;
              B.fnb[face] = block0 + id;
            }
          } else {
            // refined: the children of p touching this block must be leaves
            for (int o = 0; o < 8; o++) {
              int oo[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
              bool ok = true;
              for (int a = 0; a < 3; a++) {
                if (dd[a] < 0 && oo[a] != 1) ok = false;
                if (dd[a] > 0 && oo[a] != 0) ok = false;
              }
              if (!ok) continue;
              int32_t cid = H.at(l + 1, 2 * p[0] + oo[0], 2 * p[1] + oo[1], 2 * p[2] + oo[2]);
              if (cid < 0)
                return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": neighbours differ by more than one level");
            }
            if (face >= 0) {
              B.ftype[face] = FACE_FINER;
              B.fnb[face] = -1;
            }
          }
        }
    for (int s = 0; s < 6; s++)
      if (B.ftype[s] == FACE_COARSER || B.ftype[s] == FACE_FINER) B.amr = 1;
    blocks[block0 + b] = B;
  }
  // refluxing: a flux-register slot for every face at a resolution change,
  // and one task per coarse face that borders a refined region
  for (int b = 0; b < d.n_leaves; b++) {
    BlockDev& B = blocks[block0 + b];
    for (int f = 0; f < 6; f++)
      if (B.ftype[f] == FACE_COARSER || B.ftype[f] == FACE_FINER) {
        B.rslot[f] = h->nslots++;
        h->gtasks_h.push_back(GhostTask{block0 + b, f, B.rslot[f]});
      }
  }
  for (int b = 0; b < d.n_leaves; b++) {
    const BlockDev& B = blocks[block0 + b];
    int first = static_cast<int>(h->rtasks_h.size());
    for (int f = 0; f < 6; f++) {
      if (B.ftype[f] != FACE_FINER) continue;
      const int dir = f >> 1, side = f & 1, l = B.level;
      const int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
      const int64_t bc[3] = {B.bi, B.bj, B.bk};
      RefluxTask T{};
      T.blk = block0 + b;
      T.s = f;
      T.cslot = B.rslot[f];
      for (int q = 0; q < 4; q++) {
        int64_t p[3];
        const int64_t n = H.nblk(l + 1, dir);
        p[dir] = ((side ? 2 * bc[dir] + 2 : 2 * bc[dir] - 1) + n) % n;
        p[t1] = 2 * bc[t1] + (q & 1);
        p[t2] = 2 * bc[t2] + (q >> 1);
        int32_t id = H.at(l + 1, p[0], p[1], p[2]);
        if (id < 0) return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": refined face without fine leaves");
        T.fslot[q] = blocks[block0 + id].rslot[f ^ 1];
        if (T.fslot[q] < 0) return fail(h, BATS_ERR_UNBALANCED_TREE, "grid " + std::to_string(gidx) + ": fine face without a slot");
      }
      h->rtasks_h.push_back(T);
    }
    int cnt = static_cast<int>(h->rtasks_h.size()) - first;
    if (cnt) {
      h->rblocks_h.push_back(first);
      h->rblocks_h.push_back(cnt);
    }
  }
  // grid record + level maps with global block indices
  std::memset(&gd, 0, sizeof(gd));
  for (int a = 0; a < 3; a++) {
    gd.lo[a] = d.lo[a];
    gd.hi[a] = d.hi[a];
    gd.root[a] = d.root[a];
  }
  for (int s = 0; s < 6; s++) gd.bc[s] = d.bc[s];
  gd.maxlev = H.maxlev;
  gd.block0 = block0;
  gd.nb = d.n_leaves;
  gd.body_r = d.body_r;
  for (int v = 0; v < 8; v++) {
    gd.Winflow[v] = d.inflow[v];
    gd.Wbody[v] = d.body[v];
  }
  for (int l = 0; l <= MAXLEV; l++) {
    gd.map_off[l] = -1;
    for (int a = 0; a < 3; a++) {
      double ncell = static_cast<double>((static_cast<int64_t>(d.root[a]) << l) * NC);
      gd.dx[l][a] = (d.hi[a] - d.lo[a]) / ncell;
      gd.idx[l][a] = 1.0 / gd.dx[l][a];
      gd.dxf[l][a] = static_cast<float>(gd.dx[l][a]);
      gd.idxf[l][a] = static_cast<float>(gd.idx[l][a]);
    }
  }
  for (int a = 0; a < 3; a++) gd.lof[a] = static_cast<float>(d.lo[a]);
  // blocks with a cell centre inside the body (same FP64 centre formula as the kernels)
  if (d.body_r > 0.0) {
    for (int b = 0; b < d.n_leaves; b++) {
      BlockDev& B = blocks[block0 + b];
      for (int c = 0; c < NCELL && !B.body; c++) {
        int ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;
        double x = d.lo[0] + ((static_cast<double>(B.bi * NC) + ci) + 0.5) * gd.dx[B.level][0];
        double y = d.lo[1] + ((static_cast<double>(B.bj * NC) + cj) + 0.5) * gd.dx[B.level][1];
        double z = d.lo[2] + ((static_cast<double>(B.bk * NC) + ck) + 0.5) * gd.dx[B.level][2];
        if (x * x + y * y + z * z < d.body_r * d.body_r) B.body = 1;
      }
    }
  }
  for (int l = 0; l <= H.maxlev; l++) {
    gd.map_off[l] = static_cast<int64_t>(levmap.size());
    for (int32_t id : H.map[l]) levmap.push_back(id >= 0 ? block0 + id : -1);
  }
  return BATS_OK;
}

template <class T>
int dev_alloc(bats_t* h, T** p, size_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(h, BATS_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return BATS_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear: an unregistered host pointer is not an error here
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Page-locked host memory the device can address directly (kernels then move
// it across the host link themselves, fused with the layout change).
const void* device_view_of_pinned(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

void free_all(bats_t* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  cudaFree(h->grids_d);
  cudaFree(h->blocks_d);
  cudaFree(h->levmap_d);
  cudaFree(h->U);
  cudaFree(h->U1);
  cudaFree(h->W);
  cudaFree(h->W1);
  cudaFree(h->dtc);
  cudaFree(h->freg);
  cudaFree(h->gbuf);
  cudaFree(h->gtasks_d);
  cudaFree(h->gtab_d);
  cudaFree(h->rtasks_d);
  cudaFree(h->rblocks_d);
  cudaFree(h->dt);
  cudaFree(h->t);
  cudaFree(h->smax);
  cudaFree(h->smax_next);
  cudaFree(h->errw);
  cudaFree(h->staging);
  mlp_free(&h->mlp);
  cudaFree(h->mlp_params);
  cudaFree(h->Xb);
  cudaFree(h->Yb);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  for (cudaEvent_t e : h->stage_ev) cudaEventDestroy(e);
  h->stage_ev.clear();
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  h->stream = nullptr;
}

int grid_check(bats_t* h, int grid) {
  if (!h) return BATS_ERR_INVALID_ARG;
  if (grid < 0 || grid >= h->ngrids) return fail(h, BATS_ERR_INVALID_ARG, "grid index out of range");
  return BATS_OK;
}

StageArgs base_args(bats_t* h) {
  StageArgs a{};
  a.grids = h->grids_d;
  a.blocks = h->blocks_d;
  a.levmap = h->levmap_d;
  a.dt = h->dt;
  a.smax_next = h->smax_next;
  a.err = h->errw;
  a.nblocks = h->nbt;
  a.nslots = h->nslots;
  a.blocks_per_item = std::max(1, h->bpc);
  a.ph = h->ph;
  return a;
}

// make_ghosts = false: the ghost slabs in gbuf already hold this stage input's
// values (the learned form's second launch of a stage reads the same input).
// one_per_sm: a persistent launch of one CTA per SM (the mixed learned
// kernel, whose network weights and tensor memory each CTA sets up once).
int launch_stage_one(bats_t* h, const StageArgs& a0, bool make_ghosts = true, bool one_per_sm = false) {
  bool mixed = h->ph.precision == BATS_MIXED;
  StageArgs a = a0;
  if (mixed) {
    // the plain kernel stages its tile with tensor copies of the stage input
    const bool lrn = a.learned || a.kind >= 3;
    a.gbuf_mx = lrn ? 0 : 1;
    a.stage_tma = h->stage_tma;
    const CUtensorMap* m = a.Win == h->W1 ? h->tmW1 : h->tmW;
    for (int k = 0; k < 4; k++) a.tm[k] = m[k];
  }
  if (mixed && h->gbuf) {
    // the ghost slabs of faces at resolution changes, from this stage's input
    a.gbuf = h->gbuf;
    if (make_ghosts) {
      h->launches++;
      CK(h, launch_amr_ghosts(a, h->gtasks_d, h->gtab_d, static_cast<int>(h->gtasks_h.size()), h->stream));
    }
  }
  int nitems = (a.nblocks + a.blocks_per_item - 1) / a.blocks_per_item;
  int grid = nitems;
  if (one_per_sm) {
    grid = std::min(nitems, h->num_sms);
  } else if (h->persistent) {
    int per_sm = h->ctas_per_sm > 0 ? std::min(h->ctas_per_sm, h->occ[mixed]) : h->occ[mixed];
    grid = std::min(nitems, h->num_sms * std::max(1, per_sm));
  }
  if (grid <= 0) return BATS_OK;
  h->launches++;
  CK(h, launch_stage_kernel(mixed, grid, h->stream, a));
  return BATS_OK;
}

// Refluxing after a stage (kinds 0, 1): the coarse cells at refined faces
// take the fine fluxes' mean instead of their own face flux.
int launch_reflux(bats_t* h, const StageArgs& a) {
  if (!a.freg || a.kind > 1) return BATS_OK;
  h->launches++;
  CK(h, launch_reflux(h->ph.precision == BATS_MIXED, a, h->rtasks_d, h->rblocks_d,
                      static_cast<int>(h->rblocks_h.size() / 2), h->stream));
  return BATS_OK;
}

// One stage; with the learned form in FP64, three launches: the network
// inputs of every face, the network, and the stage with the correction; in
// the mixed form one (after the ghost pre-pass), the network run inside the
// stage kernel on the tensor cores.
int launch_stage(bats_t* h, const StageArgs& a) {
  if (!h->learned || a.kind >= 3 || (h->learned_last_only && !a.last)) {
    int rc = launch_stage_one(h, a);
    return rc ? rc : launch_reflux(h, a);
  }
  if (h->ph.precision == BATS_MIXED) {
    // mixed form: one launch, the network fused into the stage kernel
    StageArgs u = a;
    u.learned = 1;
    u.mlp = h->mlp;
    u.Y = nullptr;
    return launch_stage_one(h, u, true, true);
  }
  StageArgs f = a;
  f.kind = 3;
  f.learned = 0;
  f.Xb = h->Xb;
  int rc = launch_stage_one(h, f);
  if (rc) return rc;
  h->launches++;
  CK(h, launch_mlp_infer(h->Xb, h->Yb, static_cast<int64_t>(h->nbt) * 3 * NFACE, h->mlp, h->num_sms, h->errw,
                         h->stream));
  StageArgs u = a;
  u.learned = 1;
  u.Y = h->Yb;
  return launch_stage_one(h, u, false);  // same stage input: the ghost slabs are in place
}

// CFL bound of grid g's current state into smax[g]; with dtc, also every
// cell's local dt = cfl / s_i.
int launch_cfl(bats_t* h, int g, double* dtc = nullptr, double cfl = 0.0) {
  const GridDev& G = h->grids_h[g];
  CK(h, cudaMemsetAsync(h->smax + g, 0, sizeof(unsigned long long), h->stream));
  h->launches++;
  CK(h, launch_cfl_dt(h->ph.precision == BATS_MIXED, h->U, h->W, h->grids_d, h->blocks_d, h->ph, G.block0, G.nb,
                      h->smax, dtc, cfl, h->stream));
  return BATS_OK;
}

constexpr int kMaxTimedSteps = 256;

int ensure_stage_events(bats_t* h, int n) {
  int want = 2 * std::min(n, kMaxTimedSteps);
  while (static_cast<int>(h->stage_ev.size()) < want) {
    cudaEvent_t e;
    CK(h, cudaEventCreate(&e));
    h->stage_ev.push_back(e);
  }
  return BATS_OK;
}

// Enqueue n steps (no synchronisation).  The stage launches of each of the
// first kMaxTimedSteps steps are bracketed by an event pair: recorded on the
// stream (timed) or, while a CUDA graph is captured (captured), as event
// nodes of the graph, which its every replay records.
int enqueue_steps(bats_t* h, int n, double cfl, double fixed_dt, bool timed, bool captured = false) {
  const bool mixed = h->ph.precision == BATS_MIXED;
  const bool ssp = h->ph.rk == BATS_RK_SSP2;
  const bool euler = h->ph.rk == BATS_RK_EULER;
  const bool lts = h->local_dt && cfl > 0.0;
  if (timed) {
    int rc0 = ensure_stage_events(h, n);
    if (rc0) return rc0;
  }
  h->timed_steps = (timed || captured) ? std::min(n, kMaxTimedSteps) : 0;
  const int ntimed = h->timed_steps;
  auto record = [&](cudaEvent_t ev) {
    return captured ? cudaEventRecordWithFlags(ev, h->stream, cudaEventRecordExternal) : cudaEventRecord(ev, h->stream);
  };
  if (lts && n > 0) {
    // every cell's dt from the current state (later steps take it from the
    // last stage of the step before)
    for (int g = 0; g < h->ngrids; g++) {
      int rc = launch_cfl(h, g, h->dtc, cfl);
      if (rc) return rc;
    }
  }
  // the one-stage scheme cannot write in place (other blocks read this
  // block's cells as ghosts): it alternates between the two state buffers
  double* Ucur = h->U;
  double* Uoth = h->U1;
  float* Wcur = h->W;
  float* Woth = h->W1;
  for (int s = 0; s < n; s++) {
    CK(h, launch_dt(h->ngrids, 0, cfl, fixed_dt, h->dt, h->t, h->smax, h->smax_next, h->stream));
    h->launches++;
    if (s < ntimed) CK(h, record(h->stage_ev[2 * s]));
    StageArgs a = base_args(h);
    a.dtc = lts ? h->dtc : nullptr;
    a.cfl = cfl;
    a.freg = h->freg;
    if (euler) {
      // U^{n+1} = U^n + dt R(U^n)
      a.Uin = Ucur;
      a.Ubase = Ucur;
      a.Uout = Uoth;
      a.Win = Wcur;
      a.Wout = Woth;
      a.kind = 0;
      a.last = 1;
      a.beta = 1.0;
      a.write_u_all = 1;
      int rc = launch_stage(h, a);
      if (rc) return rc;
      std::swap(Ucur, Uoth);
      std::swap(Wcur, Woth);
    } else {
      // stage 1: U* = U^n + (dt/2) R(U^n)   [SSP-RK2: U^n + dt R(U^n)]
      a.Uin = h->U;
      a.Ubase = h->U;
      a.Uout = h->U1;
      a.Win = h->W;
      a.Wout = h->W1;
      a.kind = 0;
      a.last = 0;
      a.beta = ssp ? 1.0 : 0.5;
      a.write_u_all = (!mixed || ssp) ? 1 : 0;
      int rc = launch_stage(h, a);
      if (rc) return rc;
      // stage 2: U^{n+1} = U^n + dt R(U*)   [SSP-RK2: U^n/2 + (U* + dt R(U*))/2]
      a.Uin = h->U1;
      a.Ubase = h->U;
      a.Uout = h->U;
      a.Win = h->W1;
      a.Wout = h->W;
      a.kind = ssp ? 1 : 0;
      a.last = 1;
      a.beta = 1.0;
      a.write_u_all = 1;
      rc = launch_stage(h, a);
      if (rc) return rc;
    }
    if (s < ntimed) CK(h, record(h->stage_ev[2 * s + 1]));
    CK(h, launch_dt(h->ngrids, 1, cfl, fixed_dt, h->dt, h->t, h->smax, h->smax_next, h->stream));
    h->launches++;
  }
  if (Ucur != h->U) {
    const size_t ncell = static_cast<size_t>(h->nbt) * NV * NCELL;
    CK(h, cudaMemcpyAsync(h->U, Ucur, ncell * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (mixed) CK(h, cudaMemcpyAsync(h->W, Wcur, ncell * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  }
  CK(h, cudaGetLastError());
  return BATS_OK;
}

// Checked build: an index outside its range anywhere in the kernels since the
// last call is an error (the flag is always clear in the normal build).
int index_check(bats_t* h) {
  int32_t f = 0;
  CK(h, read_index_flag(&f));
  if (f) return fail(h, BATS_ERR_CUDA, "index check failed (checked build): an index left its range");
  return BATS_OK;
}

int run_steps(bats_t* h, int n, double cfl, double fixed_dt, double* t_out) {
  if (n < 0) return fail(h, BATS_ERR_INVALID_ARG, "negative step count");
  if (h->learned_requested && !h->learned)
    return fail(h, BATS_ERR_NOT_TRAINED, "learned form requested but no weights set (bats_set_mlp)");
  h->launches = 0;
  CK(h, cudaGetLastError());  // report (and clear) anything left from an earlier call
  int32_t init[3] = {0, INT_MAX, 0};
  CK(h, cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaEventRecord(h->ev0, h->stream));
  if (h->use_graph && n > 0) {
    if (!h->graph || h->graph_n != n || h->graph_cfl != cfl || h->graph_dt != fixed_dt) {
      if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
      // the events the graph's event nodes record exist before the capture
      if (int rc0 = ensure_stage_events(h, n)) return rc0;
      cudaGraph_t g;
      CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      h->launches = 0;
      int rc = enqueue_steps(h, n, cfl, fixed_dt, false, true);
      cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
      h->graph_n = n;
      h->graph_cfl = cfl;
      h->graph_dt = fixed_dt;
      h->graph_launches = h->launches;
      h->graph_timed = h->timed_steps;
    }
    CK(h, cudaGraphLaunch(h->graph, h->stream));
    h->launches = h->graph_launches;
    h->timed_steps = h->graph_timed;
  } else {
    int rc = enqueue_steps(h, n, cfl, fixed_dt, true);
    if (rc) return rc;
  }
  CK(h, cudaEventRecord(h->ev1, h->stream));
  int32_t ew[3];
  CK(h, cudaMemcpyAsync(ew, h->errw, sizeof(ew), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->fallbacks += ew[2];
  float ms = 0.f;
  CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  double stage_ms = 0.0;
  for (int s = 0; s < h->timed_steps && n > 0; s++) {
    float m = 0.f;
    CK(h, cudaEventElapsedTime(&m, h->stage_ev[2 * s], h->stage_ev[2 * s + 1]));
    stage_ms += m;
  }
  if (h->timed_steps > 0 && n > h->timed_steps) stage_ms *= static_cast<double>(n) / h->timed_steps;
  h->ms_last[BATS_PHASE_STAGE] = h->timed_steps > 0 ? stage_ms : -1.0;
  h->ms_last[BATS_PHASE_DT] = h->timed_steps > 0 ? ms - stage_ms : -1.0;
  h->ms_last[BATS_PHASE_TOTAL] = ms;
  if (t_out) CK(h, cudaMemcpy(t_out, h->t, sizeof(double), cudaMemcpyDeviceToHost));
  if (int rc = index_check(h)) return rc;
  if (ew[0] & ERR_TIMEOUT) return fail(h, BATS_ERR_TIMEOUT, "a bounded device wait ran out");
  if (ew[0] & ERR_BOUNDS) return fail(h, BATS_ERR_CUDA, "ghost fill met a source two levels away (unbalanced tree)");
  if (ew[0] & ERR_NONPHYSICAL)
    return fail(h, BATS_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN) in block " + std::to_string(ew[1]));
  h->err.clear();
  return BATS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

// cuTensorMapEncodeTiled, looked up through the runtime (no link against the
// driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The four tensor maps of an FP32 state buffer W (block-major [block][8][512])
// viewed as the 4-D tensor (i, j, k, 8 * block + v): the interior box
// 8 x 8 x 8 x 8 with the 32-byte swizzle, and the face-slab boxes of the
// neighbour's cells nearest a face, 4 x 8 x 8 x 8 (x; a TMA box row is at
// least 16 bytes), 8 x 2 x 8 x 8 (y) and 8 x 8 x 2 x 8 (z).
static int encode_tile_maps(bats_t* h, float* W, CUtensorMap tm[4]) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(h, BATS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[4] = {NC, NC, NC, static_cast<cuuint64_t>(h->nbt) * NV};
  const cuuint64_t strides[3] = {NC * sizeof(float), NC * NC * sizeof(float), NCELL * sizeof(float)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t boxes[4][4] = {{NC, NC, NC, NV}, {4, NC, NC, NV}, {NC, 2, NC, NV}, {NC, NC, 2, NV}};
  for (int m = 0; m < 4; m++) {
    CUresult r = encode(&tm[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, W, dims, strides, boxes[m], estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, m == 0 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, BATS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a state buffer");
  }
  return BATS_OK;
}

int bats_create(const bats_grid_desc* grids, int n_grids, const bats_physics* phys, void* cuda_stream,
                bats_t** out) {
  if (!out) return fail(nullptr, BATS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grids || n_grids <= 0 || !phys) return fail(nullptr, BATS_ERR_INVALID_ARG, "grids/phys missing");
  if (!(phys->gamma > 1.0)) return fail(nullptr, BATS_ERR_INVALID_ARG, "gamma must exceed 1");
  if (phys->reflux && phys->learned)
    return fail(nullptr, BATS_ERR_INVALID_ARG, "refluxing is not available with the learned correction");
  if (phys->flux < BATS_FLUX_RUSANOV || phys->flux > BATS_FLUX_LINDE)
    return fail(nullptr, BATS_ERR_INVALID_ARG, "bad flux kind");
  if (phys->flux != BATS_FLUX_RUSANOV && phys->learned)
    return fail(nullptr, BATS_ERR_INVALID_ARG, "the learned correction is defined on the Rusanov flux only");
  if (phys->limiter < 0 || phys->limiter > 2 || phys->rk < 0 || phys->rk > 2 || phys->local_dt < 0 ||
      phys->local_dt > 1 || phys->precision < 0 ||
      phys->precision > 1 || phys->b0 < 0 || phys->b0 > 3)
    return fail(nullptr, BATS_ERR_INVALID_ARG, "bad physics enumeration");
  bats_t* h = new bats_t();
  h->learned_requested = phys->learned != 0;
  h->learned_last_only = phys->learned_last_only != 0;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->ngrids = n_grids;
  h->grids_h.resize(n_grids);
  int block0 = 0;
  for (int g = 0; g < n_grids; g++) {
    int rc = build_grid(h, grids[g], g, block0, h->blocks_h, h->grids_h[g], h->levmap_h);
    if (rc) {
      g_create_error = h->err;
      delete h;
      return rc;
    }
    block0 += grids[g].n_leaves;
  }
  h->nbt = block0;
  h->ph.gamma = phys->gamma;
  h->ph.gm1 = phys->gamma - 1.0;
  h->ph.inv_gm1 = 1.0 / (phys->gamma - 1.0);
  h->ph.gammaf = static_cast<float>(h->ph.gamma);
  h->ph.gm1f = static_cast<float>(h->ph.gm1);
  h->ph.inv_gm1f = static_cast<float>(h->ph.inv_gm1);
  h->ph.limiter = phys->limiter;
  h->ph.rk = phys->rk;
  h->ph.precision = phys->precision;
  h->ph.b0 = phys->b0;
  h->ph.powell = phys->powell ? 1 : 0;
  h->ph.learned = 0;
  h->ph.flux = phys->flux;
  for (int i = 0; i < 12; i++) h->ph.b0p[i] = phys->b0_param[i];
  h->persistent = phys->persistent;
  h->bpc = std::max(1, phys->blocks_per_cta);
  h->ctas_per_sm = phys->ctas_per_sm;
  h->use_graph = phys->use_graph;
  h->local_dt = phys->local_dt ? 1 : 0;
  h->reflux = phys->reflux ? 1 : 0;

  int rc = BATS_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && !h->stream) {
    // a blocking stream of our own: ordered with the legacy default stream,
    // and capturable into a CUDA graph
    e = cudaStreamCreate(&h->stream);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = stage_setup(h->occ);
  if (e != cudaSuccess) {
    rc = cuda_fail(h, e, "device setup");
    g_create_error = h->err;
    delete h;
    return rc;
  }
  size_t nstate = static_cast<size_t>(h->nbt) * NV * NCELL;
  size_t maxnb = 0;
  for (auto& G : h->grids_h) maxnb = std::max<size_t>(maxnb, G.nb);
  h->staging_n = maxnb * NV * 12 * 12 * 12;
  if ((rc = dev_alloc(h, &h->grids_d, h->ngrids)) || (rc = dev_alloc(h, &h->blocks_d, h->nbt)) ||
      (rc = dev_alloc(h, &h->levmap_d, h->levmap_h.size())) || (rc = dev_alloc(h, &h->U, nstate)) ||
      (rc = dev_alloc(h, &h->U1, nstate)) || (rc = dev_alloc(h, &h->dt, h->ngrids)) ||
      (rc = dev_alloc(h, &h->t, h->ngrids)) || (rc = dev_alloc(h, &h->smax, h->ngrids)) ||
      (rc = dev_alloc(h, &h->smax_next, h->ngrids)) || (rc = dev_alloc(h, &h->errw, 3)) ||
      (rc = dev_alloc(h, &h->staging, h->staging_n))) {
    free_all(h);
    g_create_error = h->err;
    delete h;
    return rc;
  }
  if (h->reflux && !h->rtasks_h.empty() &&
      ((rc = dev_alloc(h, &h->freg, static_cast<size_t>(h->nslots) * 64 * NV)) ||
       (rc = dev_alloc(h, &h->rtasks_d, h->rtasks_h.size())) || (rc = dev_alloc(h, &h->rblocks_d, h->rblocks_h.size())))) {
    free_all(h);
    g_create_error = h->err;
    delete h;
    return rc;
  }
  if (h->ph.precision == BATS_MIXED && !h->gtasks_h.empty() &&
      ((rc = dev_alloc(h, &h->gbuf, static_cast<size_t>(h->nslots) * GSLOT)) ||
       (rc = dev_alloc(h, &h->gtasks_d, h->gtasks_h.size())) ||
       (rc = dev_alloc(h, &h->gtab_d, h->gtasks_h.size() * 128)))) {
    free_all(h);
    g_create_error = h->err;
    delete h;
    return rc;
  }
  if (h->local_dt && (rc = dev_alloc(h, &h->dtc, static_cast<size_t>(h->nbt) * NCELL))) {
    free_all(h);
    g_create_error = h->err;
    delete h;
    return rc;
  }
  if (h->ph.precision == BATS_MIXED) {
    if ((rc = dev_alloc(h, &h->W, nstate)) || (rc = dev_alloc(h, &h->W1, nstate)) ||
        (rc = encode_tile_maps(h, h->W, h->tmW)) || (rc = encode_tile_maps(h, h->W1, h->tmW1))) {
      free_all(h);
      g_create_error = h->err;
      delete h;
      return rc;
    }
  }
  e = cudaMemcpyAsync(h->grids_d, h->grids_h.data(), sizeof(GridDev) * h->ngrids, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->blocks_d, h->blocks_h.data(), sizeof(BlockDev) * h->nbt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->levmap_d, h->levmap_h.data(), sizeof(int32_t) * h->levmap_h.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->gtasks_d)
    e = cudaMemcpyAsync(h->gtasks_d, h->gtasks_h.data(), sizeof(GhostTask) * h->gtasks_h.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->rtasks_d)
    e = cudaMemcpyAsync(h->rtasks_d, h->rtasks_h.data(), sizeof(RefluxTask) * h->rtasks_h.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->rblocks_d)
    e = cudaMemcpyAsync(h->rblocks_d, h->rblocks_h.data(), sizeof(int32_t) * h->rblocks_h.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->t, 0, sizeof(double) * h->ngrids, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->smax, 0, sizeof(unsigned long long) * h->ngrids, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->U, 0, sizeof(double) * nstate, h->stream);
  if (e == cudaSuccess) e = launch_init_grid_states(h->grids_d, h->ngrids, h->ph.inv_gm1, h->ph.gm1, h->stream);
  // the static tree: where every ghost-slab sample of the pre-pass lies
  if (e == cudaSuccess && h->gtab_d)
    e = launch_amr_ghost_table(base_args(h), h->gtasks_d, h->gtab_d, static_cast<int>(h->gtasks_h.size()), h->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(h->grids_h.data(), h->grids_d, sizeof(GridDev) * h->ngrids, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    rc = cuda_fail(h, e, "upload");
    free_all(h);
    g_create_error = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return BATS_OK;
}

void bats_destroy(bats_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

const char* bats_last_error(const bats_t* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int bats_set_state(bats_t* h, int grid, const double* U, size_t n) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  const GridDev& G = h->grids_h[grid];
  size_t need = static_cast<size_t>(G.nb) * NV * NCELL;
  if (!U || n != need) return fail(h, BATS_ERR_INVALID_ARG, "state size mismatch: expected " + std::to_string(need));
  const double* src = U;
  if (!is_device_ptr(U)) {
    CK(h, cudaMemcpyAsync(h->staging, U, need * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    src = h->staging;
  }
  CK(h, launch_to_internal(src, h->U, G.block0, G.nb, h->stream));
  if (h->ph.precision == BATS_MIXED)
    CK(h, launch_prim_mixed(h->U, h->W, G.block0, G.nb, static_cast<float>(h->ph.gm1), h->stream));
  rc = launch_cfl(h, grid);
  if (rc) return rc;
  CK(h, cudaMemsetAsync(h->t + grid, 0, sizeof(double), h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return BATS_OK;
}

int bats_get_state(bats_t* h, int grid, double* U, size_t n) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  const GridDev& G = h->grids_h[grid];
  size_t need = static_cast<size_t>(G.nb) * NV * NCELL;
  if (!U || n != need) return fail(h, BATS_ERR_INVALID_ARG, "state size mismatch: expected " + std::to_string(need));
  bool dev = is_device_ptr(U);
  double* dst = dev ? U : h->staging;
  CK(h, launch_to_external(h->U, dst, G.block0, G.nb, h->stream));
  if (!dev) CK(h, cudaMemcpyAsync(U, h->staging, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return BATS_OK;
}

int bats_set_states(bats_t* h, const double* U, size_t n) {
  if (!h) return BATS_ERR_INVALID_ARG;
  const size_t need = static_cast<size_t>(h->nbt) * NV * NCELL;
  if (!U || n != need) return fail(h, BATS_ERR_INVALID_ARG, "state size mismatch: expected " + std::to_string(need));
  // device or page-locked host memory: the layout change reads it directly;
  // pageable host memory: staged through the second state buffer, free
  // between steps
  const double* src = U;
  if (!is_device_ptr(U)) {
    const void* view = device_view_of_pinned(U);
    if (view) {
      src = static_cast<const double*>(view);
    } else {
      CK(h, cudaMemcpyAsync(h->U1, U, need * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      src = h->U1;
    }
  }
  for (int g = 0; g < h->ngrids; g++) {
    const GridDev& G = h->grids_h[g];
    CK(h, launch_to_internal(src + static_cast<size_t>(G.block0) * NV * NCELL, h->U, G.block0, G.nb, h->stream));
  }
  if (h->ph.precision == BATS_MIXED)
    CK(h, launch_prim_mixed(h->U, h->W, 0, h->nbt, static_cast<float>(h->ph.gm1), h->stream));
  for (int g = 0; g < h->ngrids; g++) {
    int rc = launch_cfl(h, g);
    if (rc) return rc;
  }
  CK(h, cudaMemsetAsync(h->t, 0, sizeof(double) * h->ngrids, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return BATS_OK;
}

int bats_get_states(bats_t* h, double* U, size_t n) {
  if (!h) return BATS_ERR_INVALID_ARG;
  const size_t need = static_cast<size_t>(h->nbt) * NV * NCELL;
  if (!U || n != need) return fail(h, BATS_ERR_INVALID_ARG, "state size mismatch: expected " + std::to_string(need));
  const bool dev = is_device_ptr(U);
  double* pinned = dev ? nullptr : static_cast<double*>(const_cast<void*>(device_view_of_pinned(U)));
  double* dst = dev ? U : (pinned ? pinned : h->U1);
  for (int g = 0; g < h->ngrids; g++) {
    const GridDev& G = h->grids_h[g];
    CK(h, launch_to_external(h->U, dst + static_cast<size_t>(G.block0) * NV * NCELL, G.block0, G.nb, h->stream));
  }
  if (!dev && !pinned) CK(h, cudaMemcpyAsync(U, h->U1, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return BATS_OK;
}

int bats_step(bats_t* h, int n, double cfl, double* t_out) {
  if (!h) return BATS_ERR_INVALID_ARG;
  if (!(cfl > 0.0)) return fail(h, BATS_ERR_INVALID_ARG, "cfl must be positive");
  return run_steps(h, n, cfl, 0.0, t_out);
}

int bats_step_dt(bats_t* h, int n, double dt, double* t_out) {
  if (!h) return BATS_ERR_INVALID_ARG;
  if (!(dt > 0.0)) return fail(h, BATS_ERR_INVALID_ARG, "dt must be positive");
  return run_steps(h, n, -1.0, dt, t_out);
}

int bats_get_dt(bats_t* h, int grid, double cfl, double* dt) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  if (!dt || !(cfl > 0.0)) return fail(h, BATS_ERR_INVALID_ARG, "bad dt pointer or cfl");
  unsigned long long s;
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(&s, h->smax + grid, sizeof(s), cudaMemcpyDeviceToHost));
  double sm;
  std::memcpy(&sm, &s, sizeof(sm));
  *dt = cfl / sm;
  return BATS_OK;
}

int bats_get_time(bats_t* h, int grid, double* t) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  if (!t) return fail(h, BATS_ERR_INVALID_ARG, "t is NULL");
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(t, h->t + grid, sizeof(double), cudaMemcpyDeviceToHost));
  return BATS_OK;
}

int bats_get_timings(bats_t* h, double* ms, int n) {
  if (!h || !ms || n <= 0) return BATS_ERR_INVALID_ARG;
  for (int i = 0; i < n && i < BATS_NUM_PHASES; i++) ms[i] = h->ms_last[i];
  return BATS_OK;
}

int bats_debug_fill_ghosts(bats_t* h, int grid, double* T, size_t n) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  const GridDev& G = h->grids_h[grid];
  size_t need = static_cast<size_t>(G.nb) * NV * 1728;
  if (!T || n != need) return fail(h, BATS_ERR_INVALID_ARG, "tile size mismatch");
  bool dev = is_device_ptr(T);
  double* dst = dev ? T : h->staging;
  StageArgs a = base_args(h);
  a.Uin = h->U;
  int32_t init[3] = {0, INT_MAX, 0};
  CK(h, cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  CK(h, launch_debug_fill(a, G.block0, G.nb, dst, h->stream));
  if (!dev) CK(h, cudaMemcpyAsync(T, h->staging, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return index_check(h);
}

int bats_debug_fill_ghosts_w(bats_t* h, int grid, double* T, size_t n) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  if (h->ph.precision != BATS_MIXED) return fail(h, BATS_ERR_INVALID_ARG, "mixed form only");
  const GridDev& G = h->grids_h[grid];
  size_t need = static_cast<size_t>(G.nb) * NV * 1728;
  if (!T || n != need) return fail(h, BATS_ERR_INVALID_ARG, "tile size mismatch");
  bool dev = is_device_ptr(T);
  double* dst = dev ? T : h->staging;
  StageArgs a = base_args(h);
  a.Uin = h->U;
  a.Win = h->W;
  a.gbuf = h->gbuf;
  // the tile as the stage kernel stages it: the plain kernel's staged layout,
  // the learned kernel's generic one
  const bool staged = !h->learned;
  a.gbuf_mx = staged ? 1 : 0;
  a.stage_tma = h->stage_tma;
  for (int k = 0; k < 4; k++) a.tm[k] = h->tmW[k];
  int32_t init[3] = {0, INT_MAX, 0};
  CK(h, cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  if (h->gbuf) CK(h, launch_amr_ghosts(a, h->gtasks_d, h->gtab_d, static_cast<int>(h->gtasks_h.size()), h->stream));
  if (staged) CK(h, launch_debug_fill_mx(a, G.block0, G.nb, dst, h->stream));
  else CK(h, launch_debug_fill_w(a, G.block0, G.nb, dst, h->stream));
  if (!dev) CK(h, cudaMemcpyAsync(T, h->staging, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return index_check(h);
}

int bats_debug_residual(bats_t* h, int grid, double* R, size_t n) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  const GridDev& G = h->grids_h[grid];
  size_t need = static_cast<size_t>(G.nb) * NV * NCELL;
  if (!R || n != need) return fail(h, BATS_ERR_INVALID_ARG, "size mismatch");
  StageArgs a = base_args(h);
  a.Uin = h->U;
  a.Ubase = h->U;
  a.Uout = h->U1;
  a.Win = h->W;
  a.Wout = h->W1;
  a.kind = 2;
  a.last = 0;
  a.beta = 1.0;
  a.write_u_all = 1;
  int32_t init[3] = {0, INT_MAX, 0};
  CK(h, cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  rc = launch_stage(h, a);
  if (rc) return rc;
  bool dev = is_device_ptr(R);
  double* dst = dev ? R : h->staging;
  CK(h, launch_to_external(h->U1, dst, G.block0, G.nb, h->stream));
  if (!dev) CK(h, cudaMemcpyAsync(R, h->staging, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return index_check(h);
}

int bats_debug_wait_timeout(bats_t* h) {
  if (!h) return BATS_ERR_INVALID_ARG;
  int32_t init[3] = {0, INT_MAX, 0};
  CK(h, cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  CK(h, launch_debug_wait_timeout(h->errw, h->stream));
  int32_t ew[3];
  CK(h, cudaMemcpyAsync(ew, h->errw, sizeof(ew), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (ew[0] & ERR_TIMEOUT) return fail(h, BATS_ERR_TIMEOUT, "a bounded device wait ran out");
  return BATS_OK;
}

int bats_set_launch(bats_t* h, int persistent, int blocks_per_cta, int ctas_per_sm, int use_graph) {
  if (!h || blocks_per_cta < 1 || ctas_per_sm < 0) return BATS_ERR_INVALID_ARG;
  h->persistent = persistent ? 1 : 0;
  h->bpc = blocks_per_cta;
  h->ctas_per_sm = ctas_per_sm;
  h->use_graph = use_graph ? 1 : 0;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return BATS_OK;
}

int bats_fp64_fma_rate(void* cuda_stream, double* gflops) {
  if (!gflops) return fail(nullptr, BATS_ERR_INVALID_ARG, "gflops is required");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(nullptr, BATS_ERR_CUDA, cudaGetErrorString(e));
  const int ctas = nsm * 8, iters = 4096;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int r = 0; r < 4 && e == cudaSuccess; r++) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_fp64_fma_rate(out, ctas, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * iters * 256.0 * ctas;
    if (e == cudaSuccess && r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e9);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(nullptr, BATS_ERR_CUDA, cudaGetErrorString(e));
  *gflops = best;
  return BATS_OK;
}

int bats_set_staging(bats_t* h, int tma) {
  if (!h) return BATS_ERR_INVALID_ARG;
  if (tma != 0 && tma != 1) return fail(h, BATS_ERR_INVALID_ARG, "staging layout must be 0 or 1");
  h->stage_tma = tma;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return BATS_OK;
}

int bats_get_staging(const bats_t* h) { return h ? h->stage_tma : -1; }

int bats_set_mlp(bats_t* h, const float* params) {
  if (!h) return BATS_ERR_INVALID_ARG;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (!params) {
    h->learned = false;
    h->learned_requested = false;
    return BATS_OK;
  }
  if (h->reflux || h->ph.flux != BATS_FLUX_RUSANOV)
    return fail(h, BATS_ERR_INVALID_ARG,
                "the learned correction needs the Rusanov flux and is not available with refluxing");
  if (!h->mlp_params) {
    int rc;
    const size_t nf = static_cast<size_t>(h->nbt) * 3 * NFACE;
    if ((rc = dev_alloc(h, &h->mlp_params, MLP_NPARAM)) || (rc = dev_alloc(h, &h->Xb, nf * 24)) ||
        (rc = dev_alloc(h, &h->Yb, nf * 8)))
      return rc;
    CK(h, mlp_alloc(&h->mlp));
    CK(h, mlp_setup());
  }
  CK(h, cudaMemcpyAsync(h->mlp_params, params, sizeof(float) * MLP_NPARAM,
                        is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CK(h, launch_mlp_pack(h->mlp_params, h->mlp, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->learned = true;
  return BATS_OK;
}

int bats_debug_face_data(bats_t* h, int grid, int stage_input, double dt, float* X, double* F, size_t n_faces) {
  int rc = grid_check(h, grid);
  if (rc) return rc;
  if (h->ph.flux != BATS_FLUX_RUSANOV)
    return fail(h, BATS_ERR_INVALID_ARG, "face data (the learned correction's inputs and targets) needs the Rusanov flux");
  const GridDev& G = h->grids_h[grid];
  const size_t nf = static_cast<size_t>(G.nb) * 3 * NFACE;
  if (!F || n_faces != nf) return fail(h, BATS_ERR_INVALID_ARG, "face buffer size mismatch");
  if (stage_input && !(dt > 0.0)) return fail(h, BATS_ERR_INVALID_ARG, "stage_input needs dt > 0");
  const size_t all = static_cast<size_t>(h->nbt) * 3 * NFACE;
  float* Xf = nullptr;
  double* Fd = nullptr;
  if ((X && (rc = dev_alloc(h, &Xf, all * 40))) || (rc = dev_alloc(h, &Fd, all * 10))) {
    cudaFree(Xf);
    return rc;
  }
  StageArgs a = base_args(h);
  int32_t init[3] = {0, INT_MAX, 0};
  cudaError_t e = cudaMemcpyAsync(h->errw, init, sizeof(init), cudaMemcpyHostToDevice, h->stream);
  const double* Uin = h->U;
  const float* Win = h->W;
  if (e == cudaSuccess && stage_input) {
    e = launch_dt(h->ngrids, 0, -1.0, dt, h->dt, h->t, h->smax, h->smax_next, h->stream);
    StageArgs s1 = a;
    s1.Uin = h->U;
    s1.Ubase = h->U;
    s1.Uout = h->U1;
    s1.Win = h->W;
    s1.Wout = h->W1;
    s1.kind = 0;
    s1.last = 0;
    s1.beta = 0.5;
    s1.write_u_all = 1;
    if (e == cudaSuccess) {
      rc = launch_stage(h, s1);
      if (rc) {
        cudaFree(Xf);
        cudaFree(Fd);
        return rc;
      }
    }
    Uin = h->U1;
    Win = h->W1;
  }
  if (e == cudaSuccess) {
    a.Uin = Uin;
    a.Win = Win;
    a.kind = 4;
    a.learned = 0;
    a.Xf = Xf;
    a.Fd = Fd;
    rc = launch_stage_one(h, a);
  }
  const size_t off = static_cast<size_t>(G.block0) * 3 * NFACE;
  if (e == cudaSuccess && !rc && X)
    e = cudaMemcpyAsync(X, Xf + off * 40, nf * 40 * sizeof(float),
                        is_device_ptr(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !rc)
    e = cudaMemcpyAsync(F, Fd + off * 10, nf * 10 * sizeof(double),
                        is_device_ptr(F) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(Xf);
  cudaFree(Fd);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(h, e, "bats_debug_face_data");
  return BATS_OK;
}

int bats_get_launch_count(bats_t* h, long long* n) {
  if (!h || !n) return BATS_ERR_INVALID_ARG;
  *n = h->launches;
  return BATS_OK;
}

int bats_get_fallbacks(bats_t* h, long long* n) {
  if (!h || !n) return BATS_ERR_INVALID_ARG;
  *n = h->fallbacks;
  return BATS_OK;
}

// Self-check of the integer-only FP32 <-> FP64 conversions against CUDA's
// conversions (host arrays of n values).
int bats_debug_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out) {
  if (!f || !d || n <= 0 || !f2d_out || !d2f_out) return BATS_ERR_INVALID_ARG;
  float *fd = nullptr, *od2f = nullptr;
  double *dd = nullptr, *of2d = nullptr;
  cudaError_t e = cudaMalloc(&fd, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dd, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&of2d, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&od2f, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(fd, f, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dd, d, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_check_conversions(fd, dd, n, of2d, od2f);
  if (e == cudaSuccess) e = cudaMemcpy(f2d_out, of2d, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(d2f_out, od2f, n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(fd);
  cudaFree(dd);
  cudaFree(of2d);
  cudaFree(od2f);
  return e == cudaSuccess ? BATS_OK : BATS_ERR_CUDA;
}

}  // extern "C"
