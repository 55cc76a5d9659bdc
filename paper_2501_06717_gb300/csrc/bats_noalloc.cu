// bats_noalloc.cu -- bats_step_noalloc: the FP64 time step of one small grid
// for callers that cannot allocate device memory (for example code running
// under an external memory manager or a fixed-budget runtime that forbids
// cudaMalloc after start-up).  Every buffer the step needs beyond the caller's
// state -- the block-major copy of the state, the intermediate stage state
// U*, the block and level tables, the per-grid time-step words and the error
// words -- lives in one file-scope __device__ array of fixed size, reserved
// when the library is loaded and held until the process exits.  Nothing is
// allocated per call, on the device or on the host heap: the grid tables are
// built in fixed-capacity arrays on the caller's stack (about 80 KB).
//
// The kernels are the ones bats_step uses (k_stage FP64 form, k_cfl, k_dt and
// the layout transposes); only where their scratch lives differs.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "bats.h"
#include "bats_internal.h"

namespace batsk {
size_t stage_smem_bytes(bool mixed);
cudaError_t stage_setup(int occ[2]);
cudaError_t launch_stage_kernel(bool mixed, int grid, cudaStream_t st, const StageArgs& a);
cudaError_t launch_to_internal(const double* ext, double* in, int block0, int nb, cudaStream_t st);
cudaError_t launch_to_external(const double* in, double* ext, int block0, int nb, cudaStream_t st);
cudaError_t launch_init_grid_states(GridDev* grids, int ngrids, double inv_gm1, double gm1, cudaStream_t st);
cudaError_t launch_cfl(bool mixed, const double* U, const float* Wt, const GridDev* grids, const BlockDev* blocks,
                       const PhysDev& ph, int b0, int nb, unsigned long long* smax, cudaStream_t st);
cudaError_t launch_dt(int ngrids, int mode, double cfl, double fixed_dt, double* dt, double* t,
                      unsigned long long* smax, unsigned long long* smax_next, cudaStream_t st);
cudaError_t read_index_flag(int32_t* out);
}  // namespace batsk

using namespace batsk;

namespace {

constexpr int kMaxBlocks = BATS_NOALLOC_MAX_BLOCKS;
constexpr int kMaxMap = BATS_NOALLOC_MAX_MAP_ENTRIES;
constexpr int kMaxDevices = 64;

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kStateBytes = size_t(kMaxBlocks) * NV * NCELL * sizeof(double);
constexpr size_t kOffU = 0;
constexpr size_t kOffU1 = align256(kOffU + kStateBytes);
constexpr size_t kOffBlocks = align256(kOffU1 + kStateBytes);
constexpr size_t kOffGrid = align256(kOffBlocks + sizeof(BlockDev) * kMaxBlocks);
constexpr size_t kOffMap = align256(kOffGrid + sizeof(GridDev));
constexpr size_t kOffWords = align256(kOffMap + sizeof(int32_t) * kMaxMap);
// words: dt, t (double), smax, smax_next (u64), err[3] (int32: error bits,
// first bad block, learned-fallback count -- the stage kernel's error block)
constexpr size_t kScratchBytes = align256(kOffWords + 4 * sizeof(double) + 3 * sizeof(int32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

unsigned char* g_scratch_dev[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the
// scratch array (in host code its name is only a host-side stand-in) and the
// stage kernel's shared-memory attribute.  The address is kept only when the
// set-up succeeded; a failed set-up (for example one attempted during a
// stream capture) is tried again by the next call.
cudaError_t setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_dev[dev]) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaSuccess) {
    int occ[2];
    e = stage_setup(occ);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();  // do not leave the failure pending for unrelated code
    return e;
  }
  g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

int report(char* err, size_t len, int code, const char* msg) {
  if (err && len) std::snprintf(err, len, "%s", msg);
  return code;
}

struct Tables {
  GridDev grid;
  BlockDev blocks[kMaxBlocks];
  int32_t map[kMaxMap];
};

// Validate the tree and build the tables (fixed capacity, no heap).
int build_tables(const bats_grid_desc& d, Tables& T, char* err, size_t len) {
  if (d.n_leaves <= 0 || !d.leaves) return report(err, len, BATS_ERR_INVALID_ARG, "no leaves");
  if (d.n_leaves > kMaxBlocks)
    return report(err, len, BATS_ERR_INVALID_ARG,
                  "grid has more blocks than bats_step_noalloc supports (BATS_NOALLOC_MAX_BLOCKS)");
  for (int a = 0; a < 3; a++) {
    if (d.root[a] <= 0 || !(d.hi[a] > d.lo[a])) return report(err, len, BATS_ERR_INVALID_ARG, "bad root or extent");
    for (int s = 0; s < 2; s++)
      if (d.bc[2 * a + s] < 0 || d.bc[2 * a + s] > 2) return report(err, len, BATS_ERR_INVALID_ARG, "bad boundary code");
    if ((d.bc[2 * a] == BATS_BC_PERIODIC) != (d.bc[2 * a + 1] == BATS_BC_PERIODIC))
      return report(err, len, BATS_ERR_INVALID_ARG, "periodic on one side only");
  }
  int maxlev = 0;
  for (int b = 0; b < d.n_leaves; b++) {
    int l = d.leaves[4 * b];
    if (l < 0 || l > MAXLEV) return report(err, len, BATS_ERR_INVALID_ARG, "level out of range");
    maxlev = l > maxlev ? l : maxlev;
  }
  std::memset(&T.grid, 0, sizeof(T.grid));
  GridDev& G = T.grid;
  int64_t off = 0;
  for (int l = 0; l <= MAXLEV; l++) G.map_off[l] = -1;
  for (int l = 0; l <= maxlev; l++) {
    int64_t n = (int64_t(d.root[0]) << l) * (int64_t(d.root[1]) << l) * (int64_t(d.root[2]) << l);
    if (off + n > kMaxMap)
      return report(err, len, BATS_ERR_INVALID_ARG,
                    "level maps exceed BATS_NOALLOC_MAX_MAP_ENTRIES (too many root blocks or levels)");
    G.map_off[l] = off;
    off += n;
  }
  for (int64_t i = 0; i < off; i++) T.map[i] = -1;
  auto nblk = [&](int l, int a) { return int64_t(d.root[a]) << l; };
  auto at = [&](int l, int64_t i, int64_t j, int64_t k) -> int32_t {
    if (l < 0 || l > maxlev) return -1;
    return T.map[G.map_off[l] + (k * nblk(l, 1) + j) * nblk(l, 0) + i];
  };
  long double vol = 0;
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    for (int a = 0; a < 3; a++)
      if (L[1 + a] < 0 || L[1 + a] >= nblk(L[0], a)) return report(err, len, BATS_ERR_INVALID_ARG, "leaf outside the domain");
    int64_t m = G.map_off[L[0]] + (int64_t(L[3]) * nblk(L[0], 1) + L[2]) * nblk(L[0], 0) + L[1];
    if (T.map[m] >= 0) return report(err, len, BATS_ERR_UNBALANCED_TREE, "duplicate leaf");
    T.map[m] = b;
    vol += std::ldexp(1.0L, -3 * L[0]);
  }
  if (vol != static_cast<long double>(d.root[0]) * d.root[1] * d.root[2])
    return report(err, len, BATS_ERR_UNBALANCED_TREE, "leaves do not tile the domain");
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    for (int lc = L[0] - 1; lc >= 0; lc--) {
      int sh = L[0] - lc;
      if (at(lc, L[1] >> sh, L[2] >> sh, L[3] >> sh) >= 0)
        return report(err, len, BATS_ERR_UNBALANCED_TREE, "nested leaves");
    }
  }
  for (int b = 0; b < d.n_leaves; b++) {
    const int32_t* L = d.leaves + 4 * b;
    int l = L[0];
    BlockDev B;
    std::memset(&B, 0, sizeof(B));
    B.grid = 0;
    B.level = l;
    B.bi = L[1];
    B.bj = L[2];
    B.bk = L[3];
    for (int dk = -1; dk <= 1; dk++)
      for (int dj = -1; dj <= 1; dj++)
        for (int di = -1; di <= 1; di++) {
          if (!di && !dj && !dk) continue;
          int dd[3] = {di, dj, dk};
          int64_t p[3] = {L[1] + di, L[2] + dj, L[3] + dk};
          bool off_domain = false;
          int oa = -1, os = 0;
          for (int a = 0; a < 3; a++) {
            int64_t n = nblk(l, a);
            if (p[a] < 0 || p[a] >= n) {
              if (d.bc[2 * a] == BATS_BC_PERIODIC) p[a] = (p[a] % n + n) % n;
              else { off_domain = true; oa = a; os = p[a] < 0 ? 0 : 1; }
            }
          }
          int nz = (di != 0) + (dj != 0) + (dk != 0);
          int face = nz == 1 ? (di ? (di < 0 ? 0 : 1) : dj ? (dj < 0 ? 2 : 3) : (dk < 0 ? 4 : 5)) : -1;
          if (off_domain) {
            if (face >= 0) {
              B.ftype[face] = d.bc[2 * oa + os] == BATS_BC_INFLOW ? FACE_INFLOW : FACE_OUTFLOW;
              B.fnb[face] = -1;
            }
            continue;
          }
          int lc = -1, id = -1;
          for (int c = l; c >= 0; c--) {
            int sh = l - c;
            id = at(c, p[0] >> sh, p[1] >> sh, p[2] >> sh);
            if (id >= 0) { lc = c; break; }
          }
          if (id >= 0) {
            if (lc < l - 1) return report(err, len, BATS_ERR_UNBALANCED_TREE, "neighbours differ by more than one level");
            if (face >= 0) {
              B.ftype[face] = lc == l ? FACE_SAME : FACE_COARSER;
              B.fnb[face] = id;
            }
          } else {
            for (int o = 0; o < 8; o++) {
              int oo[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
              bool ok = true;
              for (int a = 0; a < 3; a++) {
                if (dd[a] < 0 && oo[a] != 1) ok = false;
                if (dd[a] > 0 && oo[a] != 0) ok = false;
              }
              if (ok && at(l + 1, 2 * p[0] + oo[0], 2 * p[1] + oo[1], 2 * p[2] + oo[2]) < 0)
                return report(err, len, BATS_ERR_UNBALANCED_TREE, "neighbours differ by more than one level");
            }
            if (face >= 0) {
              B.ftype[face] = FACE_FINER;
              B.fnb[face] = -1;
            }
          }
        }
    for (int s = 0; s < 6; s++)
      if (B.ftype[s] == FACE_COARSER || B.ftype[s] == FACE_FINER) B.amr = 1;
    T.blocks[b] = B;
  }
  for (int a = 0; a < 3; a++) {
    G.lo[a] = d.lo[a];
    G.hi[a] = d.hi[a];
    G.root[a] = d.root[a];
    G.lof[a] = static_cast<float>(d.lo[a]);
  }
  for (int s = 0; s < 6; s++) G.bc[s] = d.bc[s];
  G.maxlev = maxlev;
  G.block0 = 0;
  G.nb = d.n_leaves;
  G.body_r = d.body_r;
  for (int v = 0; v < 8; v++) {
    G.Winflow[v] = d.inflow[v];
    G.Wbody[v] = d.body[v];
  }
  for (int l = 0; l <= MAXLEV; l++)
    for (int a = 0; a < 3; a++) {
      double ncell = static_cast<double>((int64_t(d.root[a]) << l) * NC);
      G.dx[l][a] = (d.hi[a] - d.lo[a]) / ncell;
      G.idx[l][a] = 1.0 / G.dx[l][a];
      G.dxf[l][a] = static_cast<float>(G.dx[l][a]);
      G.idxf[l][a] = static_cast<float>(G.idx[l][a]);
    }
  if (d.body_r > 0.0) {
    for (int b = 0; b < d.n_leaves; b++) {
      BlockDev& B = T.blocks[b];
      for (int c = 0; c < NCELL && !B.body; c++) {
        int ci = c & 7, cj = (c >> 3) & 7, ck = c >> 6;
        double x = d.lo[0] + ((static_cast<double>(B.bi * NC) + ci) + 0.5) * G.dx[B.level][0];
        double y = d.lo[1] + ((static_cast<double>(B.bj * NC) + cj) + 0.5) * G.dx[B.level][1];
        double z = d.lo[2] + ((static_cast<double>(B.bk * NC) + ck) + 0.5) * G.dx[B.level][2];
        if (x * x + y * y + z * z < d.body_r * d.body_r) B.body = 1;
      }
    }
  }
  return BATS_OK;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int bats_step_noalloc(const bats_grid_desc* grid, const bats_physics* phys, double* U, size_t n, int steps,
                                 double cfl, double dt, double* t_out, void* cuda_stream, char* err, size_t err_len) {
  if (err && err_len) err[0] = '\0';
  if (!grid || !phys || !U) return report(err, err_len, BATS_ERR_INVALID_ARG, "grid, phys and U are required");
  if (steps < 0) return report(err, err_len, BATS_ERR_INVALID_ARG, "negative step count");
  if (!(cfl > 0.0) && !(dt > 0.0)) return report(err, err_len, BATS_ERR_INVALID_ARG, "need cfl > 0 or dt > 0");
  if (!(phys->gamma > 1.0)) return report(err, err_len, BATS_ERR_INVALID_ARG, "gamma must exceed 1");
  if (phys->precision != BATS_FP64 || phys->learned)
    return report(err, err_len, BATS_ERR_INVALID_ARG, "bats_step_noalloc runs the FP64 form only");
  if (phys->limiter < 0 || phys->limiter > 2 || phys->rk < 0 || phys->rk > 2 || phys->b0 < 0 || phys->b0 > 3 ||
      phys->flux < BATS_FLUX_RUSANOV || phys->flux > BATS_FLUX_LINDE)
    return report(err, err_len, BATS_ERR_INVALID_ARG, "bad physics enumeration");
  // options that change the physics and need buffers this entry point does
  // not keep (the flux register, the per-cell time steps): refused, never
  // silently dropped
  if (phys->reflux)
    return report(err, err_len, BATS_ERR_INVALID_ARG, "bats_step_noalloc does not support reflux (use bats_step)");
  if (phys->local_dt)
    return report(err, err_len, BATS_ERR_INVALID_ARG, "bats_step_noalloc does not support local_dt (use bats_step)");
  if (grid->n_leaves > kMaxBlocks)
    return report(err, err_len, BATS_ERR_INVALID_ARG,
                  "grid has more blocks than bats_step_noalloc supports (BATS_NOALLOC_MAX_BLOCKS)");
  if (grid->n_leaves <= 0 || n != static_cast<size_t>(grid->n_leaves) * NV * NCELL)
    return report(err, err_len, BATS_ERR_INVALID_ARG, "state size does not match 8 * 512 * n_leaves");

  Tables T;  // on the caller's stack
  int rc = build_tables(*grid, T, err, err_len);
  if (rc) return rc;

  // an error left pending by unrelated code is not this call's failure
  cudaGetLastError();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(err, err_len, BATS_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(err, err_len, BATS_ERR_CUDA, "device index out of range");
  e = setup_device(dev);
  if (e != cudaSuccess) return report(err, err_len, BATS_ERR_CUDA, cudaGetErrorString(e));
  unsigned char* S = g_scratch_dev[dev];
  double* Ui = reinterpret_cast<double*>(S + kOffU);
  double* U1 = reinterpret_cast<double*>(S + kOffU1);
  BlockDev* blocks = reinterpret_cast<BlockDev*>(S + kOffBlocks);
  GridDev* G = reinterpret_cast<GridDev*>(S + kOffGrid);
  int32_t* levmap = reinterpret_cast<int32_t*>(S + kOffMap);
  double* dtw = reinterpret_cast<double*>(S + kOffWords);
  double* tw = dtw + 1;
  unsigned long long* smax = reinterpret_cast<unsigned long long*>(dtw + 2);
  unsigned long long* smax_next = smax + 1;
  int32_t* errw = reinterpret_cast<int32_t*>(smax + 2);  // [3]

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  PhysDev ph{};
  ph.gamma = phys->gamma;
  ph.gm1 = phys->gamma - 1.0;
  ph.inv_gm1 = 1.0 / (phys->gamma - 1.0);
  ph.gammaf = static_cast<float>(ph.gamma);
  ph.gm1f = static_cast<float>(ph.gm1);
  ph.inv_gm1f = static_cast<float>(ph.inv_gm1);
  ph.limiter = phys->limiter;
  ph.rk = phys->rk;
  ph.precision = BATS_FP64;
  ph.b0 = phys->b0;
  ph.powell = phys->powell ? 1 : 0;
  ph.flux = phys->flux;
  for (int i = 0; i < 12; i++) ph.b0p[i] = phys->b0_param[i];
  const int nb = grid->n_leaves;
  int64_t map_entries = 0;
  for (int l = 0; l <= MAXLEV; l++)
    if (T.grid.map_off[l] >= 0)
      map_entries = T.grid.map_off[l] + (int64_t(grid->root[0]) << l) * (int64_t(grid->root[1]) << l) *
                                            (int64_t(grid->root[2]) << l);

#define NA_CK(call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return report(err, err_len, BATS_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

  // tables and cleared words (the array keeps the previous call's contents)
  NA_CK(cudaMemcpyAsync(G, &T.grid, sizeof(GridDev), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(blocks, T.blocks, sizeof(BlockDev) * nb, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(levmap, T.map, sizeof(int32_t) * map_entries, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemsetAsync(dtw, 0, 4 * sizeof(double), st));
  int32_t init[3] = {0, INT_MAX, 0};
  NA_CK(cudaMemcpyAsync(errw, init, sizeof(init), cudaMemcpyHostToDevice, st));
  NA_CK(launch_init_grid_states(G, 1, ph.inv_gm1, ph.gm1, st));
  // caller state -> block-major copy (host states are staged through U1)
  const bool dev_ptr = device_pointer(U);
  const size_t bytes = n * sizeof(double);
  if (!dev_ptr) NA_CK(cudaMemcpyAsync(U1, U, bytes, cudaMemcpyHostToDevice, st));
  NA_CK(launch_to_internal(dev_ptr ? U : U1, Ui, 0, nb, st));
  NA_CK(launch_cfl(false, Ui, nullptr, G, blocks, ph, 0, nb, smax, st));

  const bool ssp = ph.rk == BATS_RK_SSP2;
  const bool euler = ph.rk == BATS_RK_EULER;
  StageArgs a{};
  a.grids = G;
  a.blocks = blocks;
  a.levmap = levmap;
  a.dt = dtw;
  a.smax_next = smax_next;
  a.err = errw;
  a.nblocks = nb;
  a.blocks_per_item = 1;
  a.ph = ph;
  a.write_u_all = 1;
  const double c = cfl > 0.0 ? cfl : -1.0;
  // the one-stage scheme cannot update in place (other blocks read this
  // block's cells as ghosts): it alternates between Ui and U1
  double* Ucur = Ui;
  double* Uoth = U1;
  for (int s = 0; s < steps; s++) {
    NA_CK(launch_dt(1, 0, c, dt, dtw, tw, smax, smax_next, st));
    if (euler) {
      a.Uin = Ucur;
      a.Ubase = Ucur;
      a.Uout = Uoth;
      a.kind = 0;
      a.last = 1;
      a.beta = 1.0;
      NA_CK(launch_stage_kernel(false, nb, st, a));
      NA_CK(launch_dt(1, 1, c, dt, dtw, tw, smax, smax_next, st));
      double* tmp = Ucur;
      Ucur = Uoth;
      Uoth = tmp;
      continue;
    }
    a.Uin = Ui;
    a.Ubase = Ui;
    a.Uout = U1;
    a.kind = 0;
    a.last = 0;
    a.beta = ssp ? 1.0 : 0.5;
    NA_CK(launch_stage_kernel(false, nb, st, a));
    a.Uin = U1;
    a.Ubase = Ui;
    a.Uout = Ui;
    a.kind = ssp ? 1 : 0;
    a.last = 1;
    a.beta = 1.0;
    NA_CK(launch_stage_kernel(false, nb, st, a));
    NA_CK(launch_dt(1, 1, c, dt, dtw, tw, smax, smax_next, st));
  }
  if (Ucur != Ui) NA_CK(cudaMemcpyAsync(Ui, Ucur, bytes, cudaMemcpyDeviceToDevice, st));
  // block-major -> caller layout (host destinations staged through U1)
  NA_CK(launch_to_external(Ui, dev_ptr ? U : U1, 0, nb, st));
  if (!dev_ptr) NA_CK(cudaMemcpyAsync(U, U1, bytes, cudaMemcpyDeviceToHost, st));
  int32_t ew[3];
  double tt = 0.0;
  NA_CK(cudaMemcpyAsync(ew, errw, sizeof(ew), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaMemcpyAsync(&tt, tw, sizeof(double), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  // checked build: an index that left its range in these launches (always
  // clear in the normal build)
  int32_t bad_index = 0;
  NA_CK(read_index_flag(&bad_index));
#undef NA_CK
  if (t_out) *t_out = tt;
  if (bad_index) return report(err, err_len, BATS_ERR_CUDA, "index check failed (checked build): an index left its range");
  if (ew[0] & ERR_TIMEOUT) return report(err, err_len, BATS_ERR_TIMEOUT, "a bounded device wait ran out");
  if (ew[0] & ERR_BOUNDS) return report(err, err_len, BATS_ERR_CUDA, "ghost fill met a source two levels away");
  if (ew[0] & ERR_NONPHYSICAL) return report(err, err_len, BATS_ERR_NONPHYSICAL, "non-physical state after an update");
  return BATS_OK;
}
