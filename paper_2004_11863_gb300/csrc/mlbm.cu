// Host side of the library: level layout, interface descriptors, the
// recursive level schedule of Sec. 4.3, CUDA-graph capture of a coarse step
// and the C ABI declared in include/mlbm.h.
//
// Schedule of one step of level l (parent of level l+1), issued as kernels:
//   [l >= 1] K3 inject level l's TF/IE nodes from its parent's history;
//   [child]  K2 record level l's pre-collision state at t+1 on the child box
//            surface (the fine sub-steps interpolate from it);
//            advance(l+1) with the temporal weights of eq. TempInt (t+1/2);
//            K4 restrict the child's pre-collision state at its t+1 into
//            level l's TN nodes (the restriction) -- it only needs the child's state
//            after its first sub-step, which already determines it;
//            advance(l+1) with the direct transfer (t+1);
//   K1 stream + collide level l (the coarse streaming of the asynchronous
//      iteration and the coarse collision of the synchronous one).
// The coarse level therefore streams and collides in one fused pass after
// the fine sub-steps: nothing it streams is changed by the fine sub-steps
// except its TN nodes, which the restriction rebuilds anyway.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/mlbm.h"
#include "desc.h"
#include "lattice.cuh"
#include "ops.cuh"

using namespace mlbm;

namespace {

thread_local char g_errmsg[256] = "";

#define CK(expr)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf(g_errmsg, sizeof(g_errmsg), "%s: %s (%s:%d)", #expr,                 \
               cudaGetErrorString(e_), __FILE__, __LINE__);                         \
      return LBM_ECUDA;                                                             \
    }                                                                               \
  } while (0)

struct Level {
  int n[3] = {1, 1, 1};
  int per[3] = {1, 1, 1};
  int boxed[3] = {0, 0, 0};
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // box in parent units (l >= 1)
  double tau = 1.0;
  LevelView view{};
  void* mem = nullptr;
  size_t bytes = 0;
  int last = 0;  // parity of the last update (0 after init)
  long long nsteps = 0;
  long long n_nodes = 0, n_active = 0;
  // interface with the parent (l >= 1)
  RingDesc ring{};
  BndDesc bnd{};
  TnDesc tn{};  // TN nodes of the parent
  void* hist_mem = nullptr;
  double origin[3] = {0, 0, 0}, h = 1.0;  // node positions in level-0 units
  int head = 1;  // history slot holding the newest parent state (t+1)
  // hybrid collision only: velocity-deviation planes [run][D][plane] and
  // (l >= 1) the parent strain-rate history [run][3][6][K]
  void* du_mem = nullptr;
  void* sh_mem = nullptr;
  // (l >= 1, x bounded by the box, not the hybrid collision) face buffer of
  // the nodes on the two faces normal to x: the rebuild writes their
  // populations there and the level update reads them from there
  void* xf_mem = nullptr;
  // block shape of the level update (lbm_autotune)
  int k1_bx = 32, k1_by = 4;
  // non-hydrodynamic mode sensors (lbm_sensors_enable)
  bool sens_on = false;
  void* sens_mem = nullptr;
  SensorState sens{};
};

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Nodes per chunk of the host <-> device staging (lbm_init, lbm_macros):
// two buffers of 4 doubles per node, 256 MB in all.
constexpr long long kStageNodes = 1LL << 22;

// Analytic initial fields (FP64) at the nodes of a level, the same
// definitions as the host-side input generator: uniform flow; convected
// vortex (Sec. 10.1, linearised density); Gaussian pulse (Sec. 9.2).
__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

__global__ void k_ic_fields(LevelView v, Placement pl, ICDesc ic, double rho0, int dim,
                            double* rho, double* u) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  if (t >= N) return;
  const int x = (int)(t % v.n[0]), y = (int)((t / v.n[0]) % v.n[1]),
            z = (int)(t / ((long long)v.n[0] * v.n[1]));
  double X[3] = {pl.origin[0] + pl.h * x, pl.origin[1] + pl.h * y, pl.origin[2] + pl.h * z};
  for (int a = 0; a < dim; ++a) X[a] = fmod(X[a], (double)pl.dom[a]);
  double r = rho0, ux = ic.u0[0], uy = ic.u0[1], uz = dim == 3 ? ic.u0[2] : 0.0;
  const double cs2 = 1.0 / 3.0;
  if (ic.kind == 0) {
    r = rho0 + ic.drho;
  } else if (ic.kind == 1) {
    const double dx = min_image(X[0] - ic.center[0], pl.dom[0]);
    const double dy = min_image(X[1] - ic.center[1], pl.dom[1]);
    const double R = ic.radius;
    const double gg = exp(-(dx * dx + dy * dy) / (2.0 * R * R));
    r = rho0 * (1.0 - ic.eps * ic.eps / (2.0 * cs2) * gg * gg);
    ux += -ic.eps * (dy / R) * gg;
    uy += ic.eps * (dx / R) * gg;
  } else {
    double r2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double d = min_image(X[a] - ic.center[a], pl.dom[a]);
      r2 += d * d;
    }
    r = rho0 * (1.0 + ic.amplitude * exp(-r2 / (2.0 * ic.radius * ic.radius)));
  }
  rho[t] = r;
  u[t] = ux;
  u[N + t] = uy;
  u[2 * N + t] = uz;
}

}  // namespace

struct lbm_ctx {
  lbm_config cfg{};
  RefState ref{};  // reference state of the shifted storage
  int q = 0, D = 0, nlev = 0, batch = 1;
  Ops ops{};
  int device = -1;  // the device current at lbm_create (the stream's device)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t cur = nullptr;
  // side stream per level: a parent's update runs there, beside its child's
  // second sub-step (they touch disjoint memory)
  cudaStream_t side[LBM_MAX_LEVELS] = {};
  cudaEvent_t ev_fork[LBM_MAX_LEVELS] = {}, ev_join[LBM_MAX_LEVELS] = {},
              ev_restrict[LBM_MAX_LEVELS] = {};
  bool has_alloc = false;
  lbm_allocator alloc{};
  Level lev[LBM_MAX_LEVELS];
  std::vector<char> inited;  // [level][run]
  bool ready = false;
  bool seeded = false;
  long long coarse_steps = 0;
  bool use_graphs = true;
  bool use_xf = true;  // face buffers (lbm_set_face_buffer)
  // One graph per phase of a coarse step: level-0 parity (period 2) times
  // the history-slot rotation of every interface (period 3).
  static constexpr int kPhases = 6;
  cudaGraphExec_t exec[kPhases] = {};
  long long exec_nodes[kPhases] = {};
  long long launches = 0;
  // per-kernel CUDA-event timing (lbm_profile)
  struct Rec {
    int kind, level;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;
  size_t pool_used = 0;
  cudaEvent_t next_event() {
    if (pool_used == event_pool.size()) {
      cudaEvent_t e = nullptr;
      cudaEventCreate(&e);
      event_pool.push_back(e);
    }
    return event_pool[pool_used++];
  }
  // persistent fused step (lbm_set_fused): the programs of six coarse steps
  // (recorded from the scheduler with launch = false), their device copies,
  // the tables they read, the grid barrier words and the error words
  int fused = 0;                      // 0 off, 1 on, 2 test: barrier that cannot complete
  bool fused_valid = false;           // programs and tables match the current set-up
  std::vector<Phase>* recording = nullptr;
  std::vector<Phase> prog[kPhases];
  void* fused_tab = nullptr;
  Phase* fused_prog = nullptr;
  int* fused_start = nullptr;
  unsigned* fused_bar = nullptr;
  int* fused_err = nullptr;
  int* fused_err_host = nullptr;      // mapped pinned host memory
  int* fused_err_dev = nullptr;       // its device alias
  int fused_blocks = 0;
  bool fused_cluster = false;  // the fused grid is one cluster
  // probes
  int probe_level = -1, probe_n = 0, probe_cap = 0;
  long long probe_pending = 0;  // coarse steps recorded since the last read-out
  int* probe_ijk = nullptr;
  double* probe_rec = nullptr;
  unsigned long long* probe_counter = nullptr;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (has_alloc) return alloc.alloc(bytes, alloc.user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    if (has_alloc)
      alloc.free(p, alloc.user);
    else
      cudaFree(p);
  }

  // Host <-> device staging of lbm_init and lbm_macros: fields move in
  // chunks through two device buffers, copied on their own stream while the
  // other buffer's chunk is converted on the handle's stream.
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_stage[2] = {}, ev_used[2] = {};
  bool staging_ready() {
    if (copy_stream) return true;
    if (cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      copy_stream = nullptr;
      return false;
    }
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&ev_stage[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_used[b], cudaEventDisableTiming) != cudaSuccess)
        return false;
    return true;
  }
  void staging_release() {
    for (int b = 0; b < 2; ++b) {
      if (ev_stage[b]) cudaEventDestroy(ev_stage[b]);
      if (ev_used[b]) cudaEventDestroy(ev_used[b]);
      ev_stage[b] = ev_used[b] = nullptr;
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
  }
  // Device scratch of the synchronising set-up and read-out calls
  // (lbm_init, lbm_macros: the two staging buffers, at most 256 MB, kept
  // until lbm_destroy so that set-up and read-out never allocate again;
  // lbm_populations: one level's q FP64 planes, released after the call).
  // Grows by
  // freeing before allocating, so it never holds more than the largest
  // single request.  Every user synchronises before returning, so the
  // buffer is idle whenever it is released.
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* scratch_get(size_t bytes) {
    if (scratch && bytes <= scratch_bytes) return scratch;
    scratch_drop();
    scratch = dalloc(bytes);
    scratch_bytes = scratch ? bytes : 0;
    return scratch;
  }
  void scratch_drop() {
    dfree(scratch);
    scratch = nullptr;
    scratch_bytes = 0;
  }
};

namespace {

Ops ops_for(int lattice) {
  switch (lattice) {
    case LBM_D2Q9: return make_ops<D2Q9>();
    case LBM_D3Q19: return make_ops<D3Q19>();
    default: return make_ops<D3Q27>();
  }
}

void drop_graphs(lbm_ctx* h) {
  h->fused_valid = false;
  for (int k = 0; k < lbm_ctx::kPhases; ++k)
    if (h->exec[k]) {
      cudaGraphExecDestroy(h->exec[k]);
      h->exec[k] = nullptr;
      h->exec_nodes[k] = 0;
    }
}

void release(lbm_ctx* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (int l = 0; l < h->nlev; ++l) {
    h->dfree(h->lev[l].mem);
    h->dfree(h->lev[l].hist_mem);
    h->dfree(h->lev[l].du_mem);
    h->dfree(h->lev[l].sh_mem);
    h->dfree(h->lev[l].sens_mem);
    h->dfree(h->lev[l].xf_mem);
    h->lev[l].xf_mem = nullptr;
    h->lev[l].mem = h->lev[l].hist_mem = h->lev[l].du_mem = h->lev[l].sh_mem = nullptr;
    h->lev[l].sens_mem = nullptr;
  }
  h->dfree(h->probe_ijk);
  h->dfree(h->probe_rec);
  h->dfree(h->probe_counter);
  h->scratch_drop();
  h->staging_release();
  h->dfree(h->fused_tab);
  h->dfree(h->fused_prog);
  h->dfree(h->fused_start);
  h->dfree(h->fused_bar);
  h->dfree(h->fused_err);
  h->fused_tab = h->fused_prog = nullptr;
  h->fused_start = nullptr;
  h->fused_bar = nullptr;
  h->fused_err = nullptr;
  if (h->fused_err_host) cudaFreeHost(h->fused_err_host);
  h->fused_err_host = h->fused_err_dev = nullptr;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int l = 0; l < LBM_MAX_LEVELS; ++l) {
    if (h->side[l]) cudaStreamDestroy(h->side[l]);
    if (h->ev_fork[l]) cudaEventDestroy(h->ev_fork[l]);
    if (h->ev_join[l]) cudaEventDestroy(h->ev_join[l]);
    if (h->ev_restrict[l]) cudaEventDestroy(h->ev_restrict[l]);
  }
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  h->event_pool.clear();
}

// Node counts and axis kinds of every level; checks the layout rules.
int build_layout(lbm_ctx* h) {
  const lbm_config& c = h->cfg;
  const int D = h->D;
  Level& L0 = h->lev[0];
  for (int a = 0; a < 3; ++a) {
    L0.n[a] = a < D ? c.dims[a] : 1;
    L0.per[a] = 1;
    L0.boxed[a] = 0;
    if (L0.n[a] < 1) return LBM_EINVAL;
  }
  if (D == 2 && c.dims[2] != 1) return LBM_EINVAL;
  for (int a = 0; a < D; ++a)
    if (L0.n[a] < 4) return LBM_EINVAL;
  L0.tau = c.tau0;
  for (int l = 1; l < h->nlev; ++l) {
    Level& p = h->lev[l - 1];
    Level& v = h->lev[l];
    int any = 0;
    for (int a = 0; a < 3; ++a) {
      v.lo[a] = c.box[l - 1].lo[a];
      v.hi[a] = c.box[l - 1].hi[a];
      if (a >= D) {
        v.n[a] = 1;
        v.per[a] = 1;
        v.boxed[a] = 0;
        continue;
      }
      const int E = v.hi[a] - v.lo[a];
      if (p.per[a] && v.lo[a] == 0 && E == p.n[a]) {
        v.boxed[a] = 0;
        v.per[a] = 1;
        v.n[a] = 2 * p.n[a];
      } else {
        if (E < 4) return LBM_EINVAL;
        if (p.per[a]) {
          if (v.lo[a] < 0 || v.hi[a] > p.n[a] || p.n[a] - E < 4) return LBM_EINVAL;
        } else {
          if (v.lo[a] < 4 || v.hi[a] > p.n[a] - 5) return LBM_EINVAL;
        }
        v.boxed[a] = 1;
        v.per[a] = 0;
        v.n[a] = 2 * E + 1;
        any = 1;
      }
    }
    if (!any) return LBM_EINVAL;
    v.tau = 2.0 * p.tau - 0.5;  // eq. rescTau
    v.h = p.h / 2.0;
    for (int a = 0; a < 3; ++a) v.origin[a] = v.boxed[a] ? p.origin[a] + v.lo[a] * p.h : p.origin[a];
  }
  return LBM_OK;
}

// Storage geometry (ghost skin on bounded axes, row pitch a multiple of
// MLBM_ROW_ALIGN elements).
#ifndef MLBM_ROW_ALIGN
#define MLBM_ROW_ALIGN 32
#endif
void build_view(lbm_ctx* h, int l) {
  Level& v = h->lev[l];
  LevelView& w = v.view;
  int g[3];
  for (int a = 0; a < 3; ++a) g[a] = v.per[a] ? 0 : 1;
  w.SX = round_up(v.n[0] + 2 * g[0], MLBM_ROW_ALIGN);
  w.SY = v.n[1] + 2 * g[1];
  const long long SZ = v.n[2] + 2 * g[2];
  w.off = 32 + ((long long)g[2] * w.SY + g[1]) * w.SX;
  long long need = w.off + SZ * w.SY * (long long)w.SX + 32;
  // binary16 with two or more runs: runs interleaved in pairs (es = 2)
  w.es = (h->cfg.storage == LBM_FP16_SHIFTED && h->batch >= 2) ? 2 : 1;
  w.plane = (need + 63) / 64 * 64 * w.es;
  w.run_stride = w.plane * h->q;
  for (int a = 0; a < 3; ++a) {
    w.n[a] = v.n[a];
    w.per[a] = v.per[a];
  }
  w.batch = h->batch;
  w.has_ina = 0;
  w.has_tn = 0;
  w.hrr = h->cfg.collision == LBM_HRR ? 1 : 0;
  v.n_nodes = (long long)v.n[0] * v.n[1] * v.n[2];
  v.n_active = v.n_nodes;
  if (l + 1 < h->nlev) {
    const Level& c = h->lev[l + 1];
    w.has_ina = 1;
    long long ina = 1;
    for (int a = 0; a < 3; ++a) {
      if (c.boxed[a]) {
        w.ina_lo[a] = c.lo[a] + 2;
        w.ina_hi[a] = c.hi[a] - 2;
      } else {
        w.ina_lo[a] = 0;
        w.ina_hi[a] = v.n[a] - 1;
      }
      ina *= (w.ina_hi[a] - w.ina_lo[a] + 1);
    }
    w.has_tn = 1;
    for (int a = 0; a < 3; ++a) {
      w.tn_lo[a] = c.boxed[a] ? c.lo[a] + 1 : 0;
      w.tn_hi[a] = c.boxed[a] ? c.hi[a] - 1 : v.n[a] - 1;
    }
    v.n_active = v.n_nodes - ina;
  }
  v.bytes = (size_t)w.run_stride * ((h->batch + w.es - 1) / w.es) *
            (h->cfg.storage == LBM_FP16_SHIFTED ? 2 : 4);
}

// Interface descriptors of level l (l >= 1) against its parent.
void build_interface(lbm_ctx* h, int l) {
  Level& c = h->lev[l];
  const Level& p = h->lev[l - 1];
  const int D = h->D;
  RingDesc& R = c.ring;
  BndDesc& B = c.bnd;
  TnDesc& T = c.tn;
  R.nf = B.nf = T.nf = 0;
  R.start[0] = B.start[0] = T.start[0] = 0;
  for (int a = 0; a < 3; ++a) {
    R.pn[a] = p.n[a];
    R.pper[a] = p.per[a];
    R.boxed[a] = c.boxed[a];
    T.lo[a] = c.lo[a];
    T.boxed[a] = c.boxed[a];
  }
  for (int a = 0; a < D; ++a) {
    if (!c.boxed[a]) continue;
    for (int side = 0; side < 2; ++side) {
      int f = R.nf;
      R.axis[f] = B.axis[f] = T.axis[f] = a;
      R.side[f] = B.side[f] = T.side[f] = side;
      long long rs = 1, bs = 1, ts = 1;
      for (int b = 0; b < 3; ++b) {
        const int E = c.hi[b] - c.lo[b];
        // history ring (parent nodes), extended one parent cell past edges
        if (b == a) {
          R.ext[f][b] = 1;
          R.base[f][b] = side ? c.hi[b] : c.lo[b];
        } else if (b >= D) {
          R.ext[f][b] = 1;
          R.base[f][b] = 0;
        } else if (c.boxed[b]) {
          R.ext[f][b] = E + 3;
          R.base[f][b] = c.lo[b] - 1;
        } else {
          R.ext[f][b] = p.n[b];
          R.base[f][b] = 0;
        }
        // child boundary nodes, each on its first face only
        if (b == a) {
          B.lo[f][b] = side ? c.n[b] - 1 : 0;
          B.ext[f][b] = 1;
        } else if (b >= D || !c.boxed[b]) {
          B.lo[f][b] = 0;
          B.ext[f][b] = c.n[b];
        } else if (b < a) {
          B.lo[f][b] = 1;
          B.ext[f][b] = c.n[b] - 2;
        } else {
          B.lo[f][b] = 0;
          B.ext[f][b] = c.n[b];
        }
        // parent TN nodes (box-relative on bounded axes), first face only
        if (b == a) {
          T.rlo[f][b] = side ? E - 1 : 1;
          T.rext[f][b] = 1;
        } else if (b >= D) {
          T.rlo[f][b] = 0;
          T.rext[f][b] = 1;
        } else if (!c.boxed[b]) {
          T.rlo[f][b] = 0;
          T.rext[f][b] = p.n[b];
        } else if (b < a) {
          T.rlo[f][b] = 2;
          T.rext[f][b] = E - 3;
        } else {
          T.rlo[f][b] = 1;
          T.rext[f][b] = E - 1;
        }
        rs *= R.ext[f][b];
        bs *= B.ext[f][b];
        ts *= T.rext[f][b];
      }
      R.start[f + 1] = R.start[f] + rs;
      B.start[f + 1] = B.start[f] + bs;
      T.start[f + 1] = T.start[f] + ts;
      R.nf = B.nf = T.nf = f + 1;
    }
  }
  R.K = R.start[R.nf];
  R.nv = 4 + h->q;
  B.count = B.start[B.nf];
  T.count = T.start[T.nf];
}

// Device bytes of the velocity planes of level l, and of the hybrid
// collision's extra arrays.
size_t du_bytes(const lbm_ctx* h, int l) {
  return sizeof(float) * (size_t)h->D * (size_t)h->lev[l].view.plane * h->batch;
}
size_t hrr_du_bytes(const lbm_ctx* h, int l) {
  return h->cfg.collision == LBM_HRR ? du_bytes(h, l) : 0;
}
size_t hrr_sh_bytes(const lbm_ctx* h, int l) {
  if (h->cfg.collision != LBM_HRR || l < 1) return 0;
  return sizeof(float) * 3 * 6 * (size_t)h->lev[l].ring.K * h->batch;
}

// Device bytes of level l's face buffer (3D levels, faces normal to a
// bounded x axis; the hybrid collision, whose velocity pass reads the
// rebuilt nodes from the planes, has none): two faces of n[1] n[2] nodes, q
// populations, every run (binary16 run pairs: the batch rounded up to whole
// pairs).
size_t xf_bytes(const lbm_ctx* h, int l) {
  const Level& v = h->lev[l];
  if (l < 1 || h->D != 3 || !v.boxed[0] || h->cfg.collision == LBM_HRR) return 0;
  const size_t es = v.view.es > 0 ? (size_t)v.view.es : 1;
  const size_t runs = (h->batch + es - 1) / es * es;
  const size_t s = h->cfg.storage == LBM_FP16_SHIFTED ? 2 : 4;
  return s * runs * 2 * (size_t)h->q * (size_t)v.n[1] * (size_t)v.n[2];
}

// The face buffer level l's rebuild and update use now: none while the
// level's sensors are on (they read the rebuilt nodes from the planes).
void* xf_of(const lbm_ctx* h, int l) {
  const Level& v = h->lev[l];
  return (v.sens_on || !h->use_xf) ? nullptr : v.xf_mem;
}


const float kTimeQuad[3] = {-1.0f / 8.0f, 3.0f / 4.0f, 3.0f / 8.0f};  // eq. TempInt
const float kTimeLin[3] = {0.0f, 0.5f, 0.5f};   // first step: no t-1 yet
const float kTimeDirect[3] = {0.0f, 0.0f, 1.0f};  // synchronous sub-step

inline float omega_of(double tau) { return (float)(1.0 - 1.0 / tau); }

// Issue one kernel (when `launch`), bracketed by timing events when the
// handle is profiling (kind: 0 level update, 1 capture, 2 inject,
// 3 restrict, 4 probe).
#define LAUNCH_K(kind_, level_, expr)                                    \
  do {                                                                   \
    if (launch) {                                                        \
      cudaEvent_t ea_ = nullptr, eb_ = nullptr;                          \
      if (h->profiling) {                                                \
        ea_ = h->next_event();                                           \
        eb_ = h->next_event();                                           \
        CK(cudaEventRecord(ea_, h->cur));                                \
      }                                                                  \
      CK(expr);                                                          \
      ++h->launches;                                                     \
      if (h->profiling) {                                                \
        CK(cudaEventRecord(eb_, h->cur));                                \
        h->recs.push_back({kind_, level_, ea_, eb_});                    \
      }                                                                  \
    }                                                                    \
  } while (0)
#define LAUNCH(expr) LAUNCH_K(-1, -1, expr)

// Sensors of level l for the update of parity par, once its pre-collision
// state is final (kind 8; with_velocity: issue the velocity pass first,
// which the hybrid schedule has already done).
int sensor_pass(lbm_ctx* h, int l, int par, bool launch, bool with_velocity) {
  Level& v = h->lev[l];
  if (!v.sens_on) return LBM_OK;
  float* du = (float*)v.du_mem;
  if (with_velocity) LAUNCH_K(5, l, h->ops.velocity(v.view, h->cfg.storage, par, du, h->ref, h->cur));
  LAUNCH_K(8, l, h->ops.sensors(v.view, h->cfg.storage, du, par, v.sens, h->ref, h->cur));
  return LBM_OK;
}

// One step of level l with its finer levels (see the file comment).
int advance(lbm_ctx* h, int l, const float* wt, bool launch, cudaEvent_t wait_before_update) {
  Level& v = h->lev[l];
  const int st = h->cfg.storage;
  const RefState& ref = h->ref;
  const int par = 1 - v.last;
  if (l >= 1) {
    const Level& p = h->lev[l - 1];
    const float resc = (float)(v.tau / (2.0 * p.tau));  // eq. rescff
    const int slots[3] = {(v.head + 1) % 3, (v.head + 2) % 3, v.head};  // t-1, t, t+1
    if (h->recording)
      h->recording->push_back(Phase{2, l, par, 0, {slots[0], slots[1], slots[2]},
                                    {wt[0], wt[1], wt[2]}, resc, 0.0f});
    LAUNCH_K(2, l, h->ops.inject(v.view, v.bnd, v.ring, st, wt, slots, resc, par, ref,
                                 xf_of(h, l), h->cur));
  }
  if (l + 1 < h->nlev) {
    Level& c = h->lev[l + 1];
    c.head = (c.head + 1) % 3;
    if (h->recording)
      h->recording->push_back(Phase{1, l, par, 0, {c.head, c.head, c.head}, {}, 0.0f, 0.0f});
    LAUNCH_K(1, l, h->ops.capture(v.view, c.ring, st, par, 0, c.head, c.head, ref, h->cur));
    int rc = advance(h, l + 1, v.nsteps == 0 ? kTimeLin : kTimeQuad, launch, nullptr);
    if (rc) return rc;
    // The restriction and level l's own update need nothing the child's
    // second sub-step produces and touch none of the memory it writes,
    // except that the child's second update overwrites the cells the
    // restriction reads: run restriction + level-l update on the side
    // stream, and let the child's update wait for the restriction only
    // (serialised while profiling, so each kernel is timed alone).
    cudaStream_t main = h->cur;
    const bool fork = launch && !h->profiling;
    if (fork) {
      CK(cudaEventRecord(h->ev_fork[l], main));
      CK(cudaStreamWaitEvent(h->side[l], h->ev_fork[l], 0));
      h->cur = h->side[l];
    }
    const float resc = (float)(2.0 * v.tau / c.tau);  // eq. rescfc
    // (recorded for the fused step with no barrier after it: the child's
    // second rebuild, next in the program, touches other cells -- the
    // streams above run the two side by side)
    if (h->recording)
      h->recording->push_back(Phase{3, l, par, 1 - c.last, {}, {}, resc, 0.0f, 1});
    LAUNCH_K(3, l, h->ops.restrict_tn(v.view, c.view, c.tn, st, resc, par, 1 - c.last, ref,
                                      h->cur));
    if (fork) CK(cudaEventRecord(h->ev_restrict[l], h->side[l]));
    int rs = sensor_pass(h, l, par, launch, true);
    if (rs) return rs;
    // (this level may itself be a second sub-step whose update must wait
    // for its parent's restriction)
    if (launch && wait_before_update) CK(cudaStreamWaitEvent(h->cur, wait_before_update, 0));
    // (recorded for the fused step after the child's second rebuild, with
    // no barrier before the child's next phase: nothing there reads or
    // writes this level's populations)
    const Phase upd{0, l, par, 0, {}, {}, 0.0f, omega_of(v.tau), 1};
    LAUNCH_K(0, l, h->ops.stream_collide(v.view, h->cfg.collision, st, par, omega_of(v.tau), ref,
                                         v.k1_bx, v.k1_by, xf_of(h, l), h->cur));
    if (fork) {
      CK(cudaEventRecord(h->ev_join[l], h->side[l]));
      h->cur = main;
    }
    v.last = par;
    v.nsteps++;
    const size_t at = h->recording ? h->recording->size() : 0;
    rc = advance(h, l + 1, kTimeDirect, launch, fork ? h->ev_restrict[l] : nullptr);
    if (rc) return rc;
    if (h->recording) h->recording->insert(h->recording->begin() + at + 1, upd);
    if (fork) CK(cudaStreamWaitEvent(main, h->ev_join[l], 0));
    return LBM_OK;
  }
  int rs = sensor_pass(h, l, par, launch, true);
  if (rs) return rs;
  if (launch && wait_before_update) CK(cudaStreamWaitEvent(h->cur, wait_before_update, 0));
  if (h->recording) h->recording->push_back(Phase{0, l, par, 0, {}, {}, 0.0f, omega_of(v.tau)});
  LAUNCH_K(0, l, h->ops.stream_collide(v.view, h->cfg.collision, st, par, omega_of(v.tau), ref,
                                       v.k1_bx, v.k1_by, xf_of(h, l), h->cur));
  v.last = par;
  v.nsteps++;
  return LBM_OK;
}

inline float hrr_ks(const lbm_ctx* h, double tau) {
  return (float)(-2.0 * tau / 3.0 * (1.0 - h->cfg.sigma));  // -2 tau cs^2 (1 - sigma)
}

// One step of level l with its finer levels for the hybrid collision
// (Sec. 4.4).  Differences from advance(): each update is preceded by the
// velocity pass; the restriction collides the TN nodes itself; a refined
// level's outer node layer collides after its update, with the parent's
// strain rate interpolated from the strain history -- which, on the first
// sub-step, first receives the parent's S at t+1 (that needs this level's
// post-collision middle nodes for the TN velocities).
// (kinds: 5 velocity, 6 parent strain, 7 outer-layer collision)
int advance_hrr(lbm_ctx* h, int l, const float* wt, bool launch, cudaEvent_t wait_before_update,
                bool first_substep) {
  Level& v = h->lev[l];
  const int st = h->cfg.storage;
  const RefState& ref = h->ref;
  const int par = 1 - v.last;
  const float sig = (float)h->cfg.sigma;
  float* du = (float*)v.du_mem;
  int slots[3] = {0, 0, 0};
  if (l >= 1) {
    const Level& p = h->lev[l - 1];
    const float resc = (float)(v.tau / (2.0 * p.tau));  // eq. rescff
    slots[0] = (v.head + 1) % 3;
    slots[1] = (v.head + 2) % 3;
    slots[2] = v.head;
    LAUNCH_K(2, l, h->ops.inject(v.view, v.bnd, v.ring, st, wt, slots, resc, par, ref, nullptr,
                                 h->cur));
  }
  if (l + 1 < h->nlev) {
    Level& c = h->lev[l + 1];
    c.head = (c.head + 1) % 3;
    LAUNCH_K(1, l, h->ops.capture(v.view, c.ring, st, par, 0, c.head, c.head, ref, h->cur));
    int rc = advance_hrr(h, l + 1, v.nsteps == 0 ? kTimeLin : kTimeQuad, launch, nullptr, true);
    if (rc) return rc;
    cudaStream_t main = h->cur;
    const bool fork = launch && !h->profiling;
    if (fork) {
      CK(cudaEventRecord(h->ev_fork[l], main));
      CK(cudaStreamWaitEvent(h->side[l], h->ev_fork[l], 0));
      h->cur = h->side[l];
    }
    const float resc = (float)(2.0 * v.tau / c.tau);  // eq. rescfc
    LAUNCH_K(3, l, h->ops.restrict_hrr(v.view, c.view, c.tn, st, resc, par, 1 - c.last, du,
                                       omega_of(v.tau), sig, hrr_ks(h, v.tau), ref, h->cur));
    if (fork) CK(cudaEventRecord(h->ev_restrict[l], h->side[l]));
    LAUNCH_K(5, l, h->ops.velocity(v.view, st, par, du, ref, h->cur));
    rc = sensor_pass(h, l, par, launch, false);
    if (rc) return rc;
    if (launch && wait_before_update) CK(cudaStreamWaitEvent(h->cur, wait_before_update, 0));
    LAUNCH_K(0, l, h->ops.stream_collide_hrr(v.view, st, par, omega_of(v.tau), du, sig,
                                             hrr_ks(h, v.tau), ref, h->cur));
    if (fork) {
      CK(cudaEventRecord(h->ev_join[l], h->side[l]));
      h->cur = main;
    }
    v.last = par;
    v.nsteps++;
    rc = advance_hrr(h, l + 1, kTimeDirect, launch, fork ? h->ev_restrict[l] : nullptr, false);
    if (rc) return rc;
    if (fork) CK(cudaStreamWaitEvent(main, h->ev_join[l], 0));
  } else {
    LAUNCH_K(5, l, h->ops.velocity(v.view, st, par, du, ref, h->cur));
    int rs = sensor_pass(h, l, par, launch, false);
    if (rs) return rs;
    if (launch && wait_before_update) CK(cudaStreamWaitEvent(h->cur, wait_before_update, 0));
    LAUNCH_K(0, l, h->ops.stream_collide_hrr(v.view, st, par, omega_of(v.tau), du, sig,
                                             hrr_ks(h, v.tau), ref, h->cur));
    v.last = par;
    v.nsteps++;
  }
  if (l >= 1) {
    Level& p = h->lev[l - 1];
    float* sh = (float*)v.sh_mem;
    if (first_substep)
      LAUNCH_K(6, l - 1, h->ops.parent_strain(p.view, v.view, v.ring, v.tn, st, sh, v.head, v.head,
                                              1 - p.last, 1 - v.last, 0, ref, h->cur));
    LAUNCH_K(7, l, h->ops.collide_bnd(v.view, v.bnd, v.ring, st, sh, wt, slots, omega_of(v.tau),
                                      sig, hrr_ks(h, v.tau), par, ref, h->cur));
  }
  return LBM_OK;
}

int probe_launch(lbm_ctx* h, bool launch) {
  if (h->probe_n <= 0) return LBM_OK;
  const Level& v = h->lev[h->probe_level];
  // (for the fused step: with two or more levels the next coarse step
  // starts with a capture, which writes only the history)
  if (h->recording)
    h->recording->push_back(Phase{4, h->probe_level, v.last, 0, {}, {}, 0.0f, 0.0f,
                                  h->nlev > 1 ? 1 : 0});
  LAUNCH_K(4, h->probe_level, h->ops.probe(v.view, h->cfg.storage, v.last, h->probe_ijk, h->probe_n, h->probe_rec,
                      h->probe_cap, h->probe_counter, h->ref, h->cur));
  return LBM_OK;
}

int coarse_step(lbm_ctx* h, bool launch) {
  int rc = h->cfg.collision == LBM_HRR ? advance_hrr(h, 0, nullptr, launch, nullptr, false)
                                       : advance(h, 0, nullptr, launch, nullptr);
  if (rc) return rc;
  return probe_launch(h, launch);
}

// History set-up after initialisation: slots 0 (t) and 1 (t+1, the
// newest) <- (drho, u, 0) of the initial state.
int seed_history(lbm_ctx* h) {
  const bool launch = true;
  h->cur = h->stream;
  for (int l = 1; l < h->nlev; ++l) {
    Level& p = h->lev[l - 1];
    h->lev[l].head = 1;
    LAUNCH(h->ops.capture(p.view, h->lev[l].ring, h->cfg.storage, p.last, 1, 1, 0, h->ref,
                          h->cur));
    if (h->cfg.collision == LBM_HRR)
      LAUNCH(h->ops.parent_strain(p.view, h->lev[l].view, h->lev[l].ring, h->lev[l].tn,
                                  h->cfg.storage, (float*)h->lev[l].sh_mem, 1, 0, p.last,
                                  h->lev[l].last, 1, h->ref, h->cur));
  }
  h->seeded = true;
  return LBM_OK;
}

}  // namespace

// =============================================================== C ABI
extern "C" {

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument or level layout";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return g_errmsg[0] ? g_errmsg : "CUDA error";
    case LBM_EUNSTABLE: return "non-finite mass: the run is unstable";
    case LBM_ESTATE: return "call out of order (initialise every level and run first)";
    case LBM_ETIMEOUT: return "a grid barrier wait of the fused step ran out; the run's state is lost";
    default: return "unknown error";
  }
}

int lbm_lattice(int lattice, int* xi, double* w) {
  if (!xi || !w) return LBM_EINVAL;
  auto fill = [&](auto L) {
    using LT = decltype(L);
    for (int i = 0; i < LT::Q; ++i) {
      for (int a = 0; a < 3; ++a) xi[3 * i + a] = LT::c(i, a);
      w[i] = LT::w(i);
    }
    return LT::Q;
  };
  switch (lattice) {
    case LBM_D2Q9: return fill(D2Q9{});
    case LBM_D3Q19: return fill(D3Q19{});
    case LBM_D3Q27: return fill(D3Q27{});
    default: return LBM_EINVAL;
  }
}

int lbm_create(const lbm_config* cfg, void* stream, const lbm_allocator* alloc,
               lbm_handle* out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!cfg) return LBM_EINVAL;
  if (cfg->lattice < 0 || cfg->lattice > 2 || cfg->collision < 0 || cfg->collision > 3 ||
      cfg->storage < 0 || cfg->storage > 1 || cfg->nlevels < 1 ||
      cfg->nlevels > LBM_MAX_LEVELS || cfg->batch < 1 || !(cfg->tau0 > 0.5) ||
      !(cfg->rho0 > 0.0) || !std::isfinite(cfg->tau0))
    return LBM_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(cfg->u_ref[a]) || std::fabs(cfg->u_ref[a]) > 0.5) return LBM_EINVAL;
  if (cfg->lattice == LBM_D2Q9 && cfg->u_ref[2] != 0.0) return LBM_EINVAL;
  if (cfg->collision == LBM_HRR && !(cfg->sigma >= 0.0 && cfg->sigma <= 1.0)) return LBM_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return LBM_EINVAL;
  lbm_ctx* h = new (std::nothrow) lbm_ctx();
  if (!h) return LBM_ENOMEM;
  h->cfg = *cfg;
  h->ref.rho0 = cfg->rho0;
  for (int a = 0; a < 3; ++a) h->ref.U[a] = cfg->u_ref[a];
  h->ops = ops_for(cfg->lattice);
  h->q = h->ops.q;
  h->D = h->ops.d;
  h->nlev = cfg->nlevels;
  h->batch = cfg->batch;
  h->stream = (cudaStream_t)stream;
  h->cur = h->stream;
  if (alloc) {
    h->has_alloc = true;
    h->alloc = *alloc;
  }
  int rc = build_layout(h);
  if (rc) {
    delete h;
    return rc;
  }
  for (int l = 0; l < h->nlev; ++l) {
    const Level& v = h->lev[l];
    // launch-grid limits of the level update (grid.y, grid.z)
    if ((long long)v.n[2] * h->batch > 65535 || (v.n[1] + 3) / 4 > 65535 || h->batch > 65535) {
      delete h;
      return LBM_EINVAL;
    }
  }
  for (int l = 0; l < h->nlev; ++l) {
    build_view(h, l);
    if (h->lev[l].view.plane > 2147483647LL) {  // kernels index planes in 32 bits
      delete h;
      return LBM_EINVAL;
    }
  }
  for (int l = 1; l < h->nlev; ++l) build_interface(h, l);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return LBM_ECUDA;
  }
  // device memory
  for (int l = 0; l < h->nlev; ++l) {
    Level& v = h->lev[l];
    v.mem = h->dalloc(v.bytes);
    if (!v.mem) {
      release(h);
      delete h;
      return LBM_ENOMEM;
    }
    v.view.f = v.mem;
    if (cudaMemsetAsync(v.mem, 0, v.bytes, h->stream) != cudaSuccess) {
      release(h);
      delete h;
      return LBM_ECUDA;
    }
    if (l >= 1) {
      size_t hb = sizeof(float) * 3 * (size_t)v.ring.nv * (size_t)v.ring.K * h->batch;
      v.hist_mem = h->dalloc(hb);
      if (!v.hist_mem) {
        release(h);
        delete h;
        return LBM_ENOMEM;
      }
      v.ring.hist = (float*)v.hist_mem;
      cudaMemsetAsync(v.hist_mem, 0, hb, h->stream);
    }
    if (const size_t xb = xf_bytes(h, l)) {
      v.xf_mem = h->dalloc(xb);
      if (!v.xf_mem) {
        release(h);
        delete h;
        return LBM_ENOMEM;
      }
      cudaMemsetAsync(v.xf_mem, 0, xb, h->stream);

    }
    const size_t db = hrr_du_bytes(h, l), sb = hrr_sh_bytes(h, l);
    if (db) {
      v.du_mem = h->dalloc(db);
      if (!v.du_mem) {
        release(h);
        delete h;
        return LBM_ENOMEM;
      }
      cudaMemsetAsync(v.du_mem, 0, db, h->stream);
    }
    if (sb) {
      v.sh_mem = h->dalloc(sb);
      if (!v.sh_mem) {
        release(h);
        delete h;
        return LBM_ENOMEM;
      }
      cudaMemsetAsync(v.sh_mem, 0, sb, h->stream);
    }
  }
  bool ok = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int l = 0; l < h->nlev && ok; ++l)
    ok = cudaStreamCreateWithFlags(&h->side[l], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_fork[l], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_join[l], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_restrict[l], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    release(h);
    delete h;
    return LBM_ECUDA;
  }
  h->inited.assign((size_t)h->nlev * h->batch, 0);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    release(h);
    delete h;
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

int lbm_bytes(const lbm_config* cfg, unsigned long long* bytes) {
  if (!cfg || !bytes) return LBM_EINVAL;
  if (cfg->lattice < 0 || cfg->lattice > 2 || cfg->nlevels < 1 ||
      cfg->nlevels > LBM_MAX_LEVELS || cfg->batch < 1 || cfg->storage < 0 || cfg->storage > 1 ||
      cfg->collision < 0 || cfg->collision > 3)
    return LBM_EINVAL;
  lbm_ctx* h = new (std::nothrow) lbm_ctx();
  if (!h) return LBM_ENOMEM;
  h->cfg = *cfg;
  h->ops = ops_for(cfg->lattice);
  h->q = h->ops.q;
  h->D = h->ops.d;
  h->nlev = cfg->nlevels;
  h->batch = cfg->batch;
  int rc = build_layout(h);
  unsigned long long total = 0;
  if (rc == LBM_OK) {
    for (int l = 0; l < h->nlev; ++l) build_view(h, l);
    for (int l = 1; l < h->nlev; ++l) build_interface(h, l);
    for (int l = 0; l < h->nlev; ++l) {
      total += h->lev[l].bytes + hrr_du_bytes(h, l) + hrr_sh_bytes(h, l) + xf_bytes(h, l);
      if (l >= 1)
        total += sizeof(float) * 3ull * h->lev[l].ring.nv * h->lev[l].ring.K * h->batch;
    }
    *bytes = total;
  }
  delete h;
  return rc;
}

int lbm_level_info(lbm_handle h, int level, int* n, double* tau, long long* n_active) {
  if (!h || level < 0 || level >= h->nlev) return LBM_EINVAL;
  const Level& v = h->lev[level];
  if (n)
    for (int a = 0; a < 3; ++a) n[a] = v.n[a];
  if (tau) *tau = v.tau;
  if (n_active) *n_active = v.n_active;
  return LBM_OK;
}

int lbm_init(lbm_handle h, int level, int run, const double* rho, const double* u) {
  if (!h || level < 0 || level >= h->nlev || run < 0 || run >= h->batch || !rho || !u)
    return LBM_EINVAL;
  if (h->ready) {
    // a new initial state: every level of every run must be set again
    std::fill(h->inited.begin(), h->inited.end(), 0);
    h->ready = false;
  }
  Level& v = h->lev[level];
  const long long N = v.n_nodes;
  // chunks of at most kStageNodes nodes through two staging buffers
  const long long C = std::min(N, kStageNodes);
  double* d = (double*)h->scratch_get(sizeof(double) * 4 * C * 2);
  if (!d) return LBM_ENOMEM;
  if (!h->staging_ready()) return LBM_ECUDA;
  int rc = LBM_OK;
  do {
    cudaError_t e = cudaSuccess;
    // the staging buffers' last users (an earlier set-up or read-out) are
    // ordered on the handle's stream
    if ((e = cudaEventRecord(h->ev_used[0], h->stream)) != cudaSuccess ||
        (e = cudaEventRecord(h->ev_used[1], h->stream)) != cudaSuccess)
      break;
    long long k = 0;
    for (long long c0 = 0; c0 < N && e == cudaSuccess; c0 += C, ++k) {
      const int b = (int)(k & 1);
      const long long cnt = std::min(C, N - c0);
      double* buf = d + (long long)b * 4 * C;
      e = cudaStreamWaitEvent(h->copy_stream, h->ev_used[b], 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf, rho + c0, sizeof(double) * cnt, cudaMemcpyHostToDevice,
                            h->copy_stream);
      for (int a = 0; a < 3 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(buf + (1 + a) * C, u + a * N + c0, sizeof(double) * cnt,
                            cudaMemcpyHostToDevice, h->copy_stream);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_stage[b], h->copy_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_stage[b], 0);
      if (e == cudaSuccess)
        e = h->ops.init(v.view, h->cfg.storage, run, buf, buf + C, C, c0, cnt, h->ref,
                        h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_used[b], h->stream);
      ++h->launches;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      snprintf(g_errmsg, sizeof(g_errmsg), "init: %s", cudaGetErrorString(e));
      rc = LBM_ECUDA;
    }
  } while (0);
  if (rc) return rc;
  h->inited[(size_t)level * h->batch + run] = 1;
  if (std::all_of(h->inited.begin(), h->inited.end(), [](char c) { return c != 0; })) {
    for (int l = 0; l < h->nlev; ++l) {
      h->lev[l].last = 0;
      h->lev[l].nsteps = 0;
    }
    h->coarse_steps = 0;
    h->seeded = false;
    h->ready = true;
  }
  return LBM_OK;
}

int lbm_init_analytic(lbm_handle h, int run, const lbm_ic* ic) {
  if (!h || !ic || run < 0 || run >= h->batch || ic->kind < 0 || ic->kind > 2) return LBM_EINVAL;
  if (ic->kind != LBM_IC_UNIFORM && !(ic->radius > 0.0)) return LBM_EINVAL;
  if (h->ready) {
    std::fill(h->inited.begin(), h->inited.end(), 0);
    h->ready = false;
  }
  ICDesc d{};
  d.kind = ic->kind;
  for (int a = 0; a < 3; ++a) {
    d.u0[a] = ic->u0[a];
    d.center[a] = ic->center[a];
  }
  d.radius = ic->radius;
  d.amplitude = ic->amplitude;
  d.eps = ic->eps;
  d.drho = ic->drho;
  for (int l = 0; l < h->nlev; ++l) {
    Level& v = h->lev[l];
    const long long N = v.n_nodes;
    double* buf = (double*)h->dalloc(sizeof(double) * 4 * N);
    if (!buf) return LBM_ENOMEM;
    Placement pl{};
    for (int a = 0; a < 3; ++a) {
      pl.origin[a] = v.origin[a];
      pl.dom[a] = h->lev[0].n[a];
    }
    pl.h = v.h;
    k_ic_fields<<<(unsigned)((N + 127) / 128), 128, 0, h->stream>>>(v.view, pl, d, h->cfg.rho0,
                                                                    h->D, buf, buf + N);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = h->ops.init(v.view, h->cfg.storage, run, buf, buf + N, N, 0, N, h->ref, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 2;
    h->dfree(buf);
    if (e != cudaSuccess) {
      snprintf(g_errmsg, sizeof(g_errmsg), "init_analytic: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
    h->inited[(size_t)l * h->batch + run] = 1;
  }
  if (std::all_of(h->inited.begin(), h->inited.end(), [](char c) { return c != 0; })) {
    for (int l = 0; l < h->nlev; ++l) {
      h->lev[l].last = 0;
      h->lev[l].nsteps = 0;
    }
    h->coarse_steps = 0;
    h->seeded = false;
    h->ready = true;
  }
  return LBM_OK;
}

int lbm_noise(lbm_handle refined, lbm_handle single, int run, int margin, double* max_abs,
              double* rms, long long* count) {
  if (!refined || !single || !max_abs || !rms || run < 0 || run >= refined->batch ||
      run >= single->batch || margin < 0)
    return LBM_EINVAL;
  if (refined->nlev < 2 || refined->cfg.lattice != single->cfg.lattice ||
      refined->cfg.storage != single->cfg.storage)
    return LBM_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (refined->lev[0].n[a] != single->lev[0].n[a]) return LBM_EINVAL;
  if (!refined->ready || !single->ready) return LBM_ESTATE;
  CK(cudaStreamSynchronize(single->stream));
  const Level& va = refined->lev[0];
  const Level& vb = single->lev[0];
  const Level& c = refined->lev[1];
  NoiseRegion reg{};
  for (int a = 0; a < 3; ++a) {
    reg.boxed[a] = c.boxed[a];
    reg.lo[a] = c.lo[a];
    reg.E[a] = c.hi[a] - c.lo[a];
    reg.n[a] = va.n[a];
  }
  reg.margin = margin;
  const int nb = (int)((va.n_nodes + kDiagThreads - 1) / kDiagThreads);
  double* part = (double*)refined->dalloc(sizeof(double) * 3 * nb);
  if (!part) return LBM_ENOMEM;
  std::vector<double> hp((size_t)3 * nb);
  cudaError_t e = refined->ops.noise_partial(va.view, va.last, refined->ref, vb.view, vb.last,
                                             single->ref, refined->cfg.storage, run, reg, part,
                                             nb, refined->stream);
  ++refined->launches;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost,
                        refined->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(refined->stream);
  refined->dfree(part);
  if (e != cudaSuccess) {
    snprintf(g_errmsg, sizeof(g_errmsg), "noise: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  double mx = 0.0, ss = 0.0, cnt = 0.0;
  for (int b = 0; b < nb; ++b) {
    mx = std::max(mx, hp[b]);
    ss += hp[(size_t)nb + b];
    cnt += hp[(size_t)2 * nb + b];
  }
  *max_abs = mx;
  *rms = cnt > 0 ? std::sqrt(ss / cnt) : 0.0;
  if (count) *count = (long long)cnt;
  return std::isfinite(mx) ? LBM_OK : LBM_EUNSTABLE;
}

int lbm_set_graphs(lbm_handle h, int enable) {
  if (!h) return LBM_EINVAL;
  h->use_graphs = enable != 0;
  return LBM_OK;
}

namespace {

// The fused step covers the plain, regularized and recursive regularized
// collisions without sensors, outside the per-kernel profiling mode.
bool fused_usable(const lbm_ctx* h) {
  if (!h->fused || h->profiling || h->cfg.collision == LBM_HRR) return false;
  for (int l = 0; l < h->nlev; ++l)
    if (h->lev[l].sens_on) return false;
  return true;
}

// Record the programs of the six coarse steps that follow the current state
// (the scheduler with launch = false: host bookkeeping only, undone after),
// upload them and the tables they read, and size the grid: one thread per
// item of the largest phase, at most the co-resident grid.
int fused_prepare(lbm_ctx* h) {
  int head[LBM_MAX_LEVELS], last[LBM_MAX_LEVELS];
  long long nsteps[LBM_MAX_LEVELS];
  for (int l = 0; l < h->nlev; ++l) {
    head[l] = h->lev[l].head;
    last[l] = h->lev[l].last;
    nsteps[l] = h->lev[l].nsteps;
  }
  int rc = LBM_OK;
  for (int k = 0; k < lbm_ctx::kPhases; ++k) h->prog[k].clear();
  for (int s = 0; s < lbm_ctx::kPhases && rc == LBM_OK; ++s) {
    h->recording = &h->prog[(h->coarse_steps + s) % lbm_ctx::kPhases];
    rc = coarse_step(h, false);
  }
  h->recording = nullptr;
  for (int l = 0; l < h->nlev; ++l) {
    h->lev[l].head = head[l];
    h->lev[l].last = last[l];
    h->lev[l].nsteps = nsteps[l];
  }
  if (rc) return rc;
  size_t total = 0;
  for (int k = 0; k < lbm_ctx::kPhases; ++k) total += h->prog[k].size();
  if (total > (size_t)kFusedMaxPhases) return LBM_EINVAL;
  std::vector<Phase> all;
  int start[lbm_ctx::kPhases + 1];
  start[0] = 0;
  for (int k = 0; k < lbm_ctx::kPhases; ++k) {
    all.insert(all.end(), h->prog[k].begin(), h->prog[k].end());
    start[k + 1] = (int)all.size();
  }
  CK(cudaStreamSynchronize(h->stream));  // no fused launch still reads the old copies
  h->dfree(h->fused_prog);
  h->fused_prog = (Phase*)h->dalloc(sizeof(Phase) * all.size());
  if (!h->fused_tab) h->fused_tab = h->dalloc(h->ops.fused_tab_bytes());
  if (!h->fused_start) h->fused_start = (int*)h->dalloc(sizeof(start));
  if (!h->fused_bar) h->fused_bar = (unsigned*)h->dalloc(2 * sizeof(unsigned));
  if (!h->fused_err) h->fused_err = (int*)h->dalloc(sizeof(int));
  if (!h->fused_prog || !h->fused_tab || !h->fused_start || !h->fused_bar || !h->fused_err)
    return LBM_ENOMEM;
  CK(cudaMemcpy(h->fused_prog, all.data(), sizeof(Phase) * all.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->fused_start, start, sizeof(start), cudaMemcpyHostToDevice));
  FusedHost hst{};
  long long items = 1;
  for (int l = 0; l < h->nlev; ++l) {
    const Level& v = h->lev[l];
    hst.v[l] = v.view;
    hst.ring[l] = v.ring;
    hst.bnd[l] = v.bnd;
    hst.tn[l] = v.tn;
    items = std::max(items, v.n_nodes * h->batch);
  }
  hst.refd = h->ref;
  hst.coll = h->cfg.collision;
  hst.probe_n = h->probe_n;
  hst.probe_cap = h->probe_cap;
  hst.probe_ijk = h->probe_ijk;
  hst.probe_rec = h->probe_rec;
  hst.probe_counter = h->probe_counter;
  CK(h->ops.fused_setup(hst, h->fused_tab));
  const int maxb = h->ops.fused_max_blocks(h->cfg.storage);
  if (maxb <= 0) {
    snprintf(g_errmsg, sizeof(g_errmsg), "fused step: no co-resident grid");
    return LBM_ECUDA;
  }
  const long long need = (items + 255) / 256;
  h->fused_blocks = (int)std::min<long long>(maxb, need);
  // a run that fits one cluster at four items a thread or fewer runs as one
  // cluster with the hardware barrier (not the timeout test's mode 2: its
  // barrier must be the bounded one)
  h->fused_cluster = false;
  const int maxc = h->fused == 1 ? h->ops.fused_max_cluster(h->cfg.storage) : 0;
  if (maxc >= 2 && need <= 4LL * maxc) {
    h->fused_blocks = (int)std::min<long long>(maxc, need);
    h->fused_cluster = h->fused_blocks >= 2;
  }
  h->fused_valid = true;
  return LBM_OK;
}

// n coarse steps in cooperative launches of at most 1024 steps each; the
// host-side bookkeeping of every step follows as for graph replays.
int fused_steps(lbm_ctx* h, int n) {
  if (h->fused_err_host && *(volatile int*)h->fused_err_host) return LBM_ETIMEOUT;
  if (!h->fused_valid) {
    int rc = fused_prepare(h);
    if (rc) return rc;
  }
  while (n > 0) {
    const int chunk = std::min(n, 1024);
    CK(cudaMemsetAsync(h->fused_bar, 0, 2 * sizeof(unsigned), h->stream));
    CK(cudaMemsetAsync(h->fused_err, 0, sizeof(int), h->stream));
    FusedArgs A{};
    A.tab = (const FusedTables*)h->fused_tab;
    A.prog = h->fused_prog;
    A.prog_start = h->fused_start;
    A.first_key = (int)(h->coarse_steps % lbm_ctx::kPhases);
    A.nsteps = chunk;
    A.bar = h->fused_bar;
    A.err = h->fused_err;
    A.err_host = h->fused_err_dev;
    // a bounded wait: 2^21 probes of the barrier word, the first 256 without
    // sleeping and then 64 ns of __nanosleep each, about 0.13 s plus the
    // read latency of every probe; the barrier test needs milliseconds
    A.spin_limit = h->fused == 2 ? (1LL << 12) : (1LL << 21);
    A.expect_extra = h->fused == 2 ? 1 : 0;
    A.cluster = h->fused_cluster ? 1 : 0;
    CK(h->ops.fused(A, h->cfg.storage, h->fused_blocks, h->stream));
    ++h->launches;
    for (int s = 0; s < chunk; ++s) {
      int rc = coarse_step(h, false);
      if (rc) return rc;
      ++h->coarse_steps;
      if (h->probe_n > 0) ++h->probe_pending;
    }
    n -= chunk;
  }
  return LBM_OK;
}

}  // namespace

int lbm_set_fused(lbm_handle h, int mode) {
  if (!h || mode < 0 || mode > 2) return LBM_EINVAL;
  if (mode != 0 && h->cfg.collision == LBM_HRR) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  if (mode != 0 && !h->fused_err_host) {
    int* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return LBM_ENOMEM;
    }
    int* d = nullptr;
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(p);
      return LBM_ECUDA;
    }
    h->fused_err_host = p;
    h->fused_err_dev = d;
  }
  if (h->fused_err_host) *(volatile int*)h->fused_err_host = 0;
  h->fused = mode;
  h->fused_valid = false;
  return LBM_OK;
}

int lbm_step(lbm_handle h, int n_coarse) {
  if (!h || n_coarse < 0) return LBM_EINVAL;
  if (!h->ready) return LBM_ESTATE;
  if (!h->seeded) {
    int rc = seed_history(h);
    if (rc) return rc;
  }
  for (int s = 0; s < n_coarse; ++s) {
    // the first coarse step (first sub-steps with one history slot) stays
    // on the per-phase kernels; the fused programs start after it
    if (h->coarse_steps > 0 && fused_usable(h)) return fused_steps(h, n_coarse - s);
    if (h->coarse_steps == 0 || !h->use_graphs || h->profiling) {
      h->cur = h->stream;
      int rc = coarse_step(h, true);
      if (rc) return rc;
    } else {
      // every level's parity and every history rotation restart with the
      // initial state, so the phase of a coarse step is its index mod 6
      const int key = (int)(h->coarse_steps % lbm_ctx::kPhases);
      if (!h->exec[key]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        h->cur = h->cap_stream;
        const long long before = h->launches;
        int rc = coarse_step(h, true);
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        h->cur = h->stream;
        h->launches = before;  // counted when the graph runs
        if (rc) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        CK(e);
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        e = cudaGraphInstantiate(&h->exec[key], g, 0);
        cudaGraphDestroy(g);
        CK(e);
        h->exec_nodes[key] = (long long)nn;
      } else {
        int rc = coarse_step(h, false);
        if (rc) return rc;
      }
      CK(cudaGraphLaunch(h->exec[key], h->stream));
      h->launches += h->exec_nodes[key];
    }
    ++h->coarse_steps;
    if (h->probe_n > 0) ++h->probe_pending;
  }
  return LBM_OK;
}

int lbm_macros(lbm_handle h, int level, int run, double* rho, double* u) {
  if (!h || level < 0 || level >= h->nlev || run < 0 || run >= h->batch || !rho || !u)
    return LBM_EINVAL;
  if (!h->ready) return LBM_ESTATE;
  const Level& v = h->lev[level];
  const long long N = v.n_nodes;
  // chunks through two staging buffers: the read-out of one chunk (on the
  // copy stream) overlaps the next chunk's moments (on the handle's stream)
  const long long C = std::min(N, kStageNodes);
  double* d = (double*)h->scratch_get(sizeof(double) * 4 * C * 2);
  if (!d) return LBM_ENOMEM;
  if (!h->staging_ready()) return LBM_ECUDA;
  cudaError_t e = cudaSuccess;
  long long k = 0;
  for (long long c0 = 0; c0 < N && e == cudaSuccess; c0 += C, ++k) {
    const int b = (int)(k & 1);
    const long long cnt = std::min(C, N - c0);
    double* buf = d + (long long)b * 4 * C;
    // chunk k - 2's copies out of this buffer are done
    if (k >= 2) e = cudaStreamWaitEvent(h->stream, h->ev_used[b], 0);
    if (e == cudaSuccess)
      e = h->ops.macros_d(v.view, h->cfg.storage, run, v.last, buf, buf + C, C, c0, cnt, h->ref,
                          h->stream);
    ++h->launches;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_stage[b], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->ev_stage[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rho + c0, buf, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                          h->copy_stream);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a)
      e = cudaMemcpyAsync(u + a * N + c0, buf + (1 + a) * C, sizeof(double) * cnt,
                          cudaMemcpyDeviceToHost, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_used[b], h->copy_stream);
  }
  // the next user of the staging buffers runs on the handle's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_used[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_used[1], 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    snprintf(g_errmsg, sizeof(g_errmsg), "macros: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

// Candidate block shapes of the level update (threads along x, rows).
static const int kShapes[][2] = {{32, 4}, {32, 2}, {32, 1}, {64, 2}, {64, 1}, {128, 1}, {32, 3}};

int lbm_set_block_shape(lbm_handle h, int level, int bx, int by) {
  if (!h || level < 0 || level >= h->nlev || bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 128)
    return LBM_EINVAL;
  Level& v = h->lev[level];
  if ((v.n[1] + by - 1) / by > 65535) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  v.k1_bx = bx;
  v.k1_by = by;
  drop_graphs(h);
  return LBM_OK;
}

int lbm_set_face_buffer(lbm_handle h, int enable) {
  if (!h || enable < 0 || enable > 1) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  h->use_xf = enable != 0;
  drop_graphs(h);
  return LBM_OK;
}

int lbm_autotune(lbm_handle h, int reps, int* shapes) {
  if (!h || reps < 1) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  const int nc = (int)(sizeof(kShapes) / sizeof(kShapes[0]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = LBM_OK;
  for (int l = 0; l < h->nlev && rc == LBM_OK; ++l) {
    Level& v = h->lev[l];
    if (h->cfg.collision == LBM_HRR) continue;  // the hybrid update has its own kernel
    // time the update on a scratch copy of the level at rest (g = 0): the
    // arithmetic does not depend on the values, and the run is untouched
    void* scratch = h->dalloc(v.bytes);
    if (!scratch) {
      rc = LBM_ENOMEM;
      break;
    }
    LevelView w = v.view;
    w.f = scratch;
    cudaError_t e = cudaMemsetAsync(scratch, 0, v.bytes, h->stream);
    float best = 1e30f;
    int bx = v.k1_bx, by = v.k1_by;
    const float om = omega_of(v.tau);
    for (int k = 0; k < nc && e == cudaSuccess; ++k) {
      const int cx = kShapes[k][0], cy = kShapes[k][1];
      if ((v.n[1] + cy - 1) / cy > 65535) continue;
      for (int r = 0; r < 1 + reps && e == cudaSuccess; ++r) {
        if (r == 1) e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess)
          e = h->ops.stream_collide(w, h->cfg.collision, h->cfg.storage, 0, om, h->ref, cx, cy,
                                    xf_of(h, l), h->stream);
        if (e == cudaSuccess)
          e = h->ops.stream_collide(w, h->cfg.collision, h->cfg.storage, 1, om, h->ref, cx, cy,
                                    xf_of(h, l), h->stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        bx = cx;
        by = cy;
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->dfree(scratch);
    if (e != cudaSuccess) {
      snprintf(g_errmsg, sizeof(g_errmsg), "autotune: %s", cudaGetErrorString(e));
      rc = LBM_ECUDA;
      break;
    }
    v.k1_bx = bx;
    v.k1_by = by;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graphs(h);
  if (shapes)
    for (int l = 0; l < h->nlev; ++l) {
      shapes[2 * l] = h->lev[l].k1_bx;
      shapes[2 * l + 1] = h->lev[l].k1_by;
    }
  return rc;
}

int lbm_sensors_enable(lbm_handle h, int level, double eps, double g_threshold) {
  if (!h || level < 0 || level >= h->nlev || !(eps >= 0.0) || !(g_threshold >= 0.0) ||
      !std::isfinite(eps) || !std::isfinite(g_threshold))
    return LBM_EINVAL;
  Level& v = h->lev[level];
  CK(cudaStreamSynchronize(h->stream));
  if (!v.du_mem) {
    v.du_mem = h->dalloc(du_bytes(h, level));
    if (!v.du_mem) return LBM_ENOMEM;
    CK(cudaMemsetAsync(v.du_mem, 0, du_bytes(h, level), h->stream));
  }
  const int nc = h->D == 3 ? 3 : 1;
  const size_t plane = (size_t)v.view.plane * h->batch;
  if (!v.sens_mem) {
    const size_t bytes = sizeof(float) * (2 + nc) * plane + plane;
    v.sens_mem = h->dalloc(bytes);
    if (!v.sens_mem) return LBM_ENOMEM;
    CK(cudaMemsetAsync(v.sens_mem, 0, bytes, h->stream));
    v.sens.div = (float*)v.sens_mem;
    v.sens.curl = v.sens.div + plane;
    v.sens.gn = v.sens.curl + nc * plane;
    v.sens.flag = (unsigned char*)(v.sens.gn + plane);
    v.sens.nc = nc;
  }
  v.sens.eps = (float)eps;
  v.sens.g2 = (float)(g_threshold * g_threshold);
  v.sens_on = true;
  drop_graphs(h);  // the next coarse step captures the sensor pass
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_sensors(lbm_handle h, int level, int run, unsigned char* flags, double* div,
                double* curl, double* gnorm) {
  if (!h || level < 0 || level >= h->nlev || run < 0 || run >= h->batch) return LBM_EINVAL;
  const Level& v = h->lev[level];
  if (!v.sens_on) return LBM_ESTATE;
  const long long N = v.n_nodes;
  char* d = (char*)h->dalloc(sizeof(double) * 5 * N + N);
  if (!d) return LBM_ENOMEM;
  double* dd = (double*)d;
  unsigned char* df = (unsigned char*)(dd + 5 * N);
  cudaError_t e = h->ops.sensor_read(v.view, run, v.sens, df, dd, dd + N, dd + 4 * N, h->stream);
  ++h->launches;
  if (e == cudaSuccess && flags) e = cudaMemcpyAsync(flags, df, N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && div)
    e = cudaMemcpyAsync(div, dd, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && curl)
    e = cudaMemcpyAsync(curl, dd + N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && gnorm)
    e = cudaMemcpyAsync(gnorm, dd + 4 * N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->dfree(d);
  if (e != cudaSuccess) {
    snprintf(g_errmsg, sizeof(g_errmsg), "sensors: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int lbm_macros_device(lbm_handle h, int level, int run, float* rho_dev, float* u_dev) {
  if (!h || level < 0 || level >= h->nlev || run < 0 || run >= h->batch || !rho_dev || !u_dev)
    return LBM_EINVAL;
  if (!h->ready) return LBM_ESTATE;
  const Level& v = h->lev[level];
  CK(h->ops.macros_f(v.view, h->cfg.storage, run, v.last, rho_dev, u_dev, h->ref, h->stream));
  ++h->launches;
  return LBM_OK;
}

int lbm_populations(lbm_handle h, int level, int run, double* g) {
  if (!h || level < 0 || level >= h->nlev || run < 0 || run >= h->batch || !g)
    return LBM_EINVAL;
  if (!h->ready) return LBM_ESTATE;
  const Level& v = h->lev[level];
  const size_t bytes = sizeof(double) * h->q * (size_t)v.n_nodes;
  double* d = (double*)h->scratch_get(bytes);
  if (!d) return LBM_ENOMEM;
  cudaError_t e = h->ops.populations(v.view, h->cfg.storage, run, v.last, d, h->ref, h->stream);
  ++h->launches;
  if (e == cudaSuccess) e = cudaMemcpyAsync(g, d, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  h->scratch_drop();  // (a level's q FP64 planes: not kept)
  if (e != cudaSuccess) {
    snprintf(g_errmsg, sizeof(g_errmsg), "populations: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int lbm_probe_add(lbm_handle h, int level, int n, const int* ijk) {
  if (!h || level < 0 || level >= h->nlev || n < 0 || (n > 0 && !ijk) || n > 4096)
    return LBM_EINVAL;
  const Level& v = h->lev[level];
  for (int k = 0; k < n; ++k)
    for (int a = 0; a < 3; ++a)
      if (ijk[3 * k + a] < 0 || ijk[3 * k + a] >= v.n[a]) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  h->dfree(h->probe_ijk);
  h->dfree(h->probe_rec);
  h->dfree(h->probe_counter);
  h->probe_ijk = nullptr;
  h->probe_rec = nullptr;
  h->probe_counter = nullptr;
  h->probe_n = 0;
  h->probe_pending = 0;
  if (n == 0) return LBM_OK;
  long long per_step = (long long)h->batch * n * 4;
  long long cap = std::min<long long>(65536, std::max<long long>(16, (1LL << 26) / per_step));
  h->probe_ijk = (int*)h->dalloc(sizeof(int) * 3 * n);
  h->probe_rec = (double*)h->dalloc(sizeof(double) * per_step * cap);
  h->probe_counter = (unsigned long long*)h->dalloc(sizeof(unsigned long long));
  if (!h->probe_ijk || !h->probe_rec || !h->probe_counter) return LBM_ENOMEM;
  CK(cudaMemcpyAsync(h->probe_ijk, ijk, sizeof(int) * 3 * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->probe_counter, 0, sizeof(unsigned long long), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->probe_level = level;
  h->probe_n = n;
  h->probe_cap = (int)cap;
  return LBM_OK;
}

int lbm_probe(lbm_handle h, double* out, int max_steps, int* n_steps) {
  if (!h || !n_steps || max_steps < 0 || (max_steps > 0 && !out)) return LBM_EINVAL;
  *n_steps = 0;
  if (h->probe_n <= 0) return LBM_OK;
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, h->probe_counter, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const long long kept = std::min<long long>((long long)cnt, h->probe_cap);
  const long long take = std::min<long long>(kept, max_steps);
  const long long per_step = (long long)h->batch * h->probe_n * 4;
  for (long long s = 0; s < take; ++s) {
    const unsigned long long step = cnt - take + s;
    const long long slot = (long long)(step % (unsigned long long)h->probe_cap);
    CK(cudaMemcpyAsync(out + s * per_step, h->probe_rec + slot * per_step,
                       sizeof(double) * per_step, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemsetAsync(h->probe_counter, 0, sizeof(unsigned long long), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->probe_pending = 0;
  *n_steps = (int)take;
  return LBM_OK;
}

int lbm_probe_async(lbm_handle h, double* out, int max_steps, int* n_steps) {
  if (!h || !n_steps || max_steps < 0 || (max_steps > 0 && !out)) return LBM_EINVAL;
  *n_steps = 0;
  if (h->probe_n <= 0) return LBM_OK;
  // the device counter advanced once per coarse step since its last reset,
  // so the host count gives the slots without reading it back
  const long long kept = std::min<long long>(h->probe_pending, h->probe_cap);
  const long long take = std::min<long long>(kept, max_steps);
  const long long per_step = (long long)h->batch * h->probe_n * 4;
  long long s = 0;
  while (s < take) {  // at most two copies: the ring may wrap once
    const long long step = h->probe_pending - take + s;
    const long long slot = step % h->probe_cap;
    const long long run = std::min<long long>(take - s, h->probe_cap - slot);
    CK(cudaMemcpyAsync(out + s * per_step, h->probe_rec + slot * per_step,
                       sizeof(double) * per_step * run, cudaMemcpyDeviceToHost, h->stream));
    s += run;
  }
  CK(cudaMemsetAsync(h->probe_counter, 0, sizeof(unsigned long long), h->stream));
  h->probe_pending = 0;
  *n_steps = (int)take;
  return LBM_OK;
}

int lbm_diag(lbm_handle h, int run, double* mass, double* mom) {
  if (!h || run < 0 || run >= h->batch || !mass || !mom) return LBM_EINVAL;
  if (!h->ready) return LBM_ESTATE;
  int rc = LBM_OK;
  for (int l = 0; l < h->nlev && rc == LBM_OK; ++l) {
    const Level& v = h->lev[l];
    const int nb = (int)((v.n_nodes + kDiagThreads - 1) / kDiagThreads);
    double* part = (double*)h->dalloc(sizeof(double) * 4 * nb);
    if (!part) return LBM_ENOMEM;
    std::vector<double> hp((size_t)4 * nb);
    cudaError_t e =
        h->ops.diag_partial(v.view, h->cfg.storage, run, v.last, part, nb, h->ref, h->stream);
    ++h->launches;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->dfree(part);
    if (e != cudaSuccess) {
      snprintf(g_errmsg, sizeof(g_errmsg), "diag: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
    // block partials summed in a fixed order on the host
    double s[4] = {0, 0, 0, 0};
    for (int j = 0; j < 4; ++j)
      for (int b = 0; b < nb; ++b) s[j] += hp[(size_t)j * nb + b];
    mass[l] = s[0];
    for (int a = 0; a < 3; ++a) mom[3 * l + a] = s[1 + a];
    for (int j = 0; j < 4; ++j)
      if (!std::isfinite(s[j])) rc = LBM_EUNSTABLE;
  }
  return rc;
}

int lbm_sync(lbm_handle h) {
  if (!h) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  if (h->fused_err_host && *(volatile int*)h->fused_err_host) return LBM_ETIMEOUT;
  return LBM_OK;
}

long long lbm_kernel_launches(lbm_handle h) { return h ? h->launches : -1; }

int lbm_profile(lbm_handle h, int enable) {
  if (!h) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  h->recs.clear();
  h->pool_used = 0;
  h->profiling = enable != 0;
  return LBM_OK;
}

int lbm_profile_read(lbm_handle h, int kind, int level, double* total_ms, long long* count) {
  if (!h || !total_ms || !count) return LBM_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  double t = 0.0;
  long long n = 0;
  for (const auto& r : h->recs) {
    if (r.kind != kind || (level >= 0 && r.level != level)) continue;
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    ++n;
  }
  *total_ms = t;
  *count = n;
  return LBM_OK;
}

void lbm_destroy(lbm_handle h) {
  if (!h) return;
  release(h);
  delete h;
}

}  // extern "C"

// ======================================================================
// lbm_diag_noalloc: the conservation diagnostic without any allocation.
//
// lbm_diag obtains a temporary device buffer for its per-block partial sums
// on every call.  Some callers cannot let the library allocate: a serving
// loop that admits runs against a fixed device-memory budget and must not
// grow after admission, a host whose device memory is entirely handed to
// another framework's caching pool, or a monitor that cannot afford the
// device-wide synchronisation that cudaFree implies.  This variant keeps the
// partial sums in one fixed array that lives in the library's device image
// for as long as the library is loaded (every GPU that loads the library
// holds it until the process exits).
// ======================================================================
namespace {

// Room for the per-block partials of a level of up to this many nodes
// (kDiagThreads nodes per block, 4 sums per block) plus the final sums.
constexpr long long kNoAllocMaxNodes = 16777216LL;  // 2^24
constexpr int kNoAllocMaxBlocks = (int)(kNoAllocMaxNodes / kDiagThreads);
constexpr int kNoAllocSlots = 4 * kNoAllocMaxBlocks + 4;

static __device__ __align__(256) double g_diag_scratch[kNoAllocSlots];

// Final sums of the block partials, one thread per quantity, in block order
// (the same order lbm_diag uses on the host, so both give the same bits).
__global__ void k_diag_final(const double* partial, int nblocks, double* out) {
  const int j = threadIdx.x;
  if (j >= 4) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)j * nblocks + b];
  out[j] = s;
}

std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};

// Address of the scratch array on device `dev` (which must be current),
// looked up once per device.
int scratch_on_device(int dev, double** out) {
  if (dev < 0 || dev >= 64) return LBM_EINVAL;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_diag_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_ptr[dev]);
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_diag_noalloc(lbm_handle h, int run, double* mass, double* mom) {
  if (!h || run < 0 || run >= h->batch || !mass || !mom) return LBM_EINVAL;
  for (int l = 0; l < h->nlev; ++l)
    if (h->lev[l].n_nodes > kNoAllocMaxNodes) return LBM_EINVAL;  // beyond the fixed scratch
  if (!h->ready) return LBM_ESTATE;
  // the scratch address is per device: the handle's device must be current
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != h->device) return LBM_EINVAL;
  double* scratch = nullptr;
  int rc = scratch_on_device(dev, &scratch);
  if (rc) return rc;
  double* partial = scratch;
  double* result = scratch + 4 * (long long)kNoAllocMaxBlocks;
  rc = LBM_OK;
  for (int l = 0; l < h->nlev; ++l) {
    const Level& v = h->lev[l];
    const int nb = (int)((v.n_nodes + kDiagThreads - 1) / kDiagThreads);
    // every partial the final sum reads is written first, so nothing needs
    // clearing between calls
    CK(h->ops.diag_partial(v.view, h->cfg.storage, run, v.last, partial, nb, h->ref, h->stream));
    k_diag_final<<<1, 32, 0, h->stream>>>(partial, nb, result);
    CK(cudaGetLastError());
    h->launches += 2;
    double s[4];
    CK(cudaMemcpyAsync(s, result, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    mass[l] = s[0];
    for (int a = 0; a < 3; ++a) mom[3 * l + a] = s[1 + a];
    for (int j = 0; j < 4; ++j)
      if (!std::isfinite(s[j])) rc = LBM_EUNSTABLE;
  }
  return rc;
}
