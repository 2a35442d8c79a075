// Kernels of one multi-level step (Sec. 4.3, cell-vertex coupling):
//
//   k_stream_collide  fused stream + collide of every active node of a level
//                     (eq. LBMequation), in place with the AA pattern;
//   k_capture         parent pre-collision (drho, u, f^(1)) at t+1 on a child
//                     box surface -> three-slot history (steps 2a/2b, 2g);
//   k_inject          child TF / IE nodes: temporal (eq. TempInt) and spatial
//                     (eq. spaceInt) interpolation, rescaling (eq. rescff),
//                     written where the child's next update reads them;
//   k_restrict        parent TN nodes: filtered child f^(1) (eq. filterFneq),
//                     rescaling (eq. rescfc), written where the parent's next
//                     update reads them (step 3d);
//   k_init / k_macros / k_diag_* / k_probe   set-up and read-out.
//
// AA pattern.  A step of parity 0 reads g_i of node n from plane i at n and
// writes the post-collision g_i* to plane opp(i) at n; a step of parity 1
// reads g_i from plane opp(i) at n - xi_i and writes g_i* to plane i at
// n + xi_i.  Every memory cell is read and then written by the same node, so
// one array suffices.  The "read location" of (i, n) for parity p is where
// the update of parity p fetches the pre-collision g_i(n); the interface
// kernels overwrite exactly those cells for the nodes they rebuild, so the
// level update itself has no special cases.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "desc.h"
#include "lattice.cuh"

namespace mlbm {

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Element offsets of a node and of its 3^D neighbours inside a plane.
struct NodeAddr {
  long long zo[3];
  int yo[3];
  int xo[3];
  long long off;
  __device__ __forceinline__ long long at(int dx, int dy, int dz) const {
    return off + zo[dz + 1] + yo[dy + 1] + xo[dx + 1];
  }
};

template <class L>
__device__ __forceinline__ NodeAddr node_addr(const LevelView& v, int x, int y, int z) {
  NodeAddr a;
  a.off = v.off;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int xx = x + d, yy = y + d;
    if (v.per[0]) xx = wrapi(xx, v.n[0]);
    if (v.per[1]) yy = wrapi(yy, v.n[1]);
    a.xo[d + 1] = xx;
    a.yo[d + 1] = yy * v.SX;
    if constexpr (L::D == 3) {
      int zz = z + d;
      if (v.per[2]) zz = wrapi(zz, v.n[2]);
      a.zo[d + 1] = (long long)zz * v.SY * v.SX;
    } else {
      a.zo[d + 1] = 0;
    }
  }
  return a;
}

__device__ __forceinline__ bool inactive(const LevelView& v, int x, int y, int z) {
  return v.has_ina && x >= v.ina_lo[0] && x <= v.ina_hi[0] && y >= v.ina_lo[1] &&
         y <= v.ina_hi[1] && z >= v.ina_lo[2] && z <= v.ina_hi[2];
}

// Pre-collision populations of node a for an update of parity PAR.
template <class L, class S>
__device__ __forceinline__ void load_pre(const S* f, long long plane, const NodeAddr& a, int par,
                                         float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (par == 0)
      g[i] = Store<S>::ld(f + (long long)i * plane + a.at(0, 0, 0));
    else
      g[i] = Store<S>::ld(f + (long long)opp<L>(i) * plane +
                          a.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)));
  });
}

// Write populations into the cells an update of parity `par` reads.
template <class L, class S>
__device__ __forceinline__ void store_pre(S* f, long long plane, const NodeAddr& a, int par,
                                          const float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (par == 0)
      Store<S>::st(f + (long long)i * plane + a.at(0, 0, 0), g[i]);
    else
      Store<S>::st(f + (long long)opp<L>(i) * plane + a.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)),
                   g[i]);
  });
}

// Post-collision populations of node a after an update of parity `last`
// (initial states are written like a parity-0 update).
template <class L, class S>
__device__ __forceinline__ void load_post(const S* f, long long plane, const NodeAddr& a,
                                          int last, float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (last == 0)
      g[i] = Store<S>::ld(f + (long long)opp<L>(i) * plane + a.at(0, 0, 0));
    else
      g[i] = Store<S>::ld(f + (long long)i * plane + a.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)));
  });
}

// ------------------------------------------------------- K1: level update
// One thread per node; a warp covers 32 consecutive x of one row.
template <class L, int COLL, class S, int PAR>
__global__ void __launch_bounds__(128) k_stream_collide(LevelView v, float omega, float rho0) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  int z = blockIdx.z, run = 0;
  if (v.batch > 1) {
    run = z / v.n[2];
    z -= run * v.n[2];
  }
  if (x >= v.n[0] || y >= v.n[1]) return;
  if (inactive(v, x, y, z)) return;
  S* f = static_cast<S*>(v.f) + run * v.run_stride;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_pre<L, S>(f, v.plane, a, PAR, g);
  collide<L, COLL>(g, omega, rho0);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (PAR == 0)
      Store<S>::st(f + (long long)opp<L>(i) * v.plane + a.at(0, 0, 0), g[i]);
    else
      Store<S>::st(f + (long long)i * v.plane + a.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)), g[i]);
  });
}

// (drho, u, f^(1)) of a population set.
template <class L>
__device__ __forceinline__ void split_neq(const float (&g)[L::Q], float rho0, float& drho,
                                          float& ux, float& uy, float& uz, float (&f1)[L::Q]) {
  float jx, jy, jz;
  moments<L>(g, drho, jx, jy, jz);
  const float inv = 1.0f / (rho0 + drho);
  ux = jx * inv;
  uy = jy * inv;
  uz = (L::D == 3) ? jz * inv : 0.0f;
  float g0[L::Q];
  equilibrium<L>(drho, rho0 + drho, ux, uy, uz, g0);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f1[i] = g[i] - g0[i];
  });
}

__device__ __forceinline__ int ring_face(const long long* start, int nf, long long k) {
  int f = 0;
  while (f + 1 < nf && k >= start[f + 1]) ++f;
  return f;
}

// ------------------------------------------------------------ K2: capture
// mode 0: shift the slots (t-1 <- t, t <- t+1) and store the parent's
// pre-collision state for an update of parity `par` into slot t+1.
// mode 1 (set-up): store (drho, u, 0) of the parent's current state (laid
// out after an update of parity `par`) into slots t and t+1.
template <class L, class S>
__global__ void k_capture(LevelView p, RingDesc R, int par, int mode, float rho0) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  if (k >= R.K) return;
  const int fc = ring_face(R.start, R.nf, k);
  long long loc = k - R.start[fc];
  int P[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = R.ext[fc][a];
    int i = (int)(loc % e);
    loc /= e;
    int c = R.base[fc][a] + i;
    if (R.pper[a]) c = ((c % R.pn[a]) + R.pn[a]) % R.pn[a];
    P[a] = c;
  }
  const S* f = static_cast<const S*>(p.f) + run * p.run_stride;
  const NodeAddr a = node_addr<L>(p, P[0], P[1], P[2]);
  float g[L::Q];
  if (mode == 0)
    load_pre<L, S>(f, p.plane, a, par, g);
  else
    load_post<L, S>(f, p.plane, a, par, g);
  float drho, ux, uy, uz, f1[L::Q];
  split_neq<L>(g, rho0, drho, ux, uy, uz, f1);
  const int nv = R.nv;
  float* h = R.hist + (long long)run * 3 * nv * R.K;
  auto slot = [&](int s, int vv) -> float& { return h[((long long)s * nv + vv) * R.K + k]; };
  if (mode == 0) {
    for (int vv = 0; vv < nv; ++vv) {
      slot(0, vv) = slot(1, vv);
      slot(1, vv) = slot(2, vv);
    }
  }
  float nvv[4] = {drho, ux, uy, uz};
  for (int s = (mode == 0 ? 2 : 1); s <= 2; ++s) {
#pragma unroll
    for (int vv = 0; vv < 4; ++vv) slot(s, vv) = nvv[vv];
    sfor<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      slot(s, 4 + i) = (mode == 0) ? f1[i] : 0.0f;
    });
  }
}

// ------------------------------------------------------------- K3: inject
// Child boundary nodes.  wt: temporal weights on slots (t-1, t, t+1);
// resc = tau_f / (2 tau_c) (eq. rescff); par: the child's next update.
template <class L, class S>
__global__ void k_inject(LevelView c, BndDesc B, RingDesc R, float w0, float w1, float w2,
                         float resc, int par, float rho0) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  if (k >= B.count) return;
  const int fc = ring_face(B.start, B.nf, k);
  long long loc = k - B.start[fc];
  int X[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = B.ext[fc][a];
    X[a] = B.lo[fc][a] + (int)(loc % e);
    loc /= e;
  }
  // odd child coordinates (at most two, never the face axis)
  int odd0 = -1, odd1 = -1;
#pragma unroll
  for (int a = 0; a < L::D; ++a)
    if (X[a] & 1) {
      if (odd0 < 0) odd0 = a;
      else odd1 = a;
    }
  const int n0 = odd0 >= 0 ? 4 : 1, n1 = odd1 >= 0 ? 4 : 1;
  const float sw[4] = {-1.0f / 16.0f, 9.0f / 16.0f, 9.0f / 16.0f, -1.0f / 16.0f};
  // ring face of the same (axis, side): strides of its local index
  const int rf = fc;
  long long stride[3];
  stride[0] = 1;
  stride[1] = R.ext[rf][0];
  stride[2] = stride[1] * R.ext[rf][1];
  const int nv = R.nv;
  const float* h = R.hist + (long long)run * 3 * nv * R.K;
  float acc[4 + L::Q];
#pragma unroll
  for (int j = 0; j < 4 + L::Q; ++j) acc[j] = 0.0f;
  for (int s0 = 0; s0 < n0; ++s0)
    for (int s1 = 0; s1 < n1; ++s1) {
      long long idx = R.start[rf];
      float w = 1.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a == R.axis[rf] || a >= L::D) continue;
        int xc = X[a];
        if (a == odd0) {
          xc += 2 * s0 - 3;
          w *= sw[s0];
        } else if (a == odd1) {
          xc += 2 * s1 - 3;
          w *= sw[s1];
        }
        const int half = (xc >= 0) ? xc / 2 : -((-xc) / 2);  // xc is even
        int li;
        if (R.boxed[a])
          li = half + 1;
        else
          li = wrapi(half, R.pn[a]);
        idx += (long long)li * stride[a];
      }
#pragma unroll
      for (int j = 0; j < 4 + L::Q; ++j) {
        const float v0 = h[((long long)0 * nv + j) * R.K + idx];
        const float v1 = h[((long long)1 * nv + j) * R.K + idx];
        const float v2 = h[((long long)2 * nv + j) * R.K + idx];
        acc[j] += w * (w0 * v0 + w1 * v1 + w2 * v2);
      }
    }
  float g[L::Q];
  equilibrium<L>(acc[0], rho0 + acc[0], acc[1], acc[2], acc[3], g);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    g[i] += resc * acc[4 + i];
  });
  S* f = static_cast<S*>(c.f) + run * c.run_stride;
  const NodeAddr a = node_addr<L>(c, X[0], X[1], X[2]);
  store_pre<L, S>(f, c.plane, a, par, g);
}

// ----------------------------------------------------------- K4: restrict
// Parent TN nodes.  resc = 2 tau_c / tau_f (eq. rescfc); ppar / cpar: the
// parent's and the child's next updates.
template <class L, class S>
__global__ void k_restrict(LevelView p, LevelView c, TnDesc T, float resc, int ppar, int cpar,
                           float rho0) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  if (k >= T.count) return;
  const int fc = ring_face(T.start, T.nf, k);
  long long loc = k - T.start[fc];
  int P[3], X[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = T.rext[fc][a];
    const int r = T.rlo[fc][a] + (int)(loc % e);
    loc /= e;
    if (T.boxed[a]) {
      int pc = T.lo[a] + r;
      if (p.per[a]) pc = wrapi(pc, p.n[a]);
      P[a] = pc;
      X[a] = 2 * r;
    } else {
      P[a] = r;
      X[a] = 2 * r;
    }
  }
  const S* fc_ = static_cast<const S*>(c.f) + run * c.run_stride;
  float f1s[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) f1s[i] = 0.0f;
  float drho_c = 0.0f, ux_c = 0.0f, uy_c = 0.0f, uz_c = 0.0f;
  const int dzr = (L::D == 3) ? 1 : 0;
  for (int dz = -dzr; dz <= dzr; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int xx = X[0] + dx, yy = X[1] + dy, zz = X[2] + dz;
        if (c.per[0]) xx = wrapi(xx, c.n[0]);
        if (c.per[1]) yy = wrapi(yy, c.n[1]);
        if (L::D == 3 && c.per[2]) zz = wrapi(zz, c.n[2]);
        const NodeAddr a = node_addr<L>(c, xx, yy, zz);
        float g[L::Q], f1[L::Q], drho, ux, uy, uz;
        load_pre<L, S>(fc_, c.plane, a, cpar, g);
        split_neq<L>(g, rho0, drho, ux, uy, uz, f1);
        const float w = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) *
                        (L::D == 3 ? (dz == 0 ? 0.5f : 0.25f) : 1.0f);
        sfor<L::Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          f1s[i] += w * f1[i];
        });
        if (dx == 0 && dy == 0 && dz == 0) {
          drho_c = drho;
          ux_c = ux;
          uy_c = uy;
          uz_c = uz;
        }
      }
  float g[L::Q];
  equilibrium<L>(drho_c, rho0 + drho_c, ux_c, uy_c, uz_c, g);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    g[i] += resc * f1s[i];
  });
  S* fp = static_cast<S*>(p.f) + run * p.run_stride;
  const NodeAddr a = node_addr<L>(p, P[0], P[1], P[2]);
  store_pre<L, S>(fp, p.plane, a, ppar, g);
}

// ------------------------------------------------------ set-up / read-out
__device__ __forceinline__ bool node_of(const LevelView& v, long long t, int& x, int& y, int& z) {
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  if (t >= N) return false;
  x = (int)(t % v.n[0]);
  t /= v.n[0];
  y = (int)(t % v.n[1]);
  z = (int)(t / v.n[1]);
  return true;
}

// Equilibrium initial state from FP64 fields, laid out as after a parity-0
// update (post-collision g_i at plane opp(i) of the node).
template <class L, class S>
__global__ void k_init(LevelView v, int run, const double* rho, const double* u, double rho0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  const double r = rho[t];
  double g0[L::Q];
  equilibrium<L, double>(r - rho0, r, u[t], u[N + t], u[2 * N + t], g0);
  S* f = static_cast<S*>(v.f) + run * v.run_stride;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Store<S>::st(f + (long long)opp<L>(i) * v.plane + a.at(0, 0, 0), (float)g0[i]);
  });
}

// rho and u (FP64 or FP32 outputs) of the post-collision state; NaN at
// inactive nodes.
template <class L, class S, class T>
__global__ void k_macros(LevelView v, int run, int last, T* rho, T* u, double rho0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  if (inactive(v, x, y, z)) {
    const T nan = T(__longlong_as_double(0x7ff8000000000000ULL));
    rho[t] = nan;
    u[t] = u[N + t] = u[2 * N + t] = nan;
    return;
  }
  const S* f = static_cast<const S*>(v.f) + run * v.run_stride;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_post<L, S>(f, v.plane, a, last, g);
  float drho, jx, jy, jz;
  moments<L>(g, drho, jx, jy, jz);
  const double r = rho0 + (double)drho;
  rho[t] = T(r);
  u[t] = T((double)jx / r);
  u[N + t] = T((double)jy / r);
  u[2 * N + t] = T(L::D == 3 ? (double)jz / r : 0.0);
}

// Shifted populations of the post-collision state, [q][N] FP64.
template <class L, class S>
__global__ void k_populations(LevelView v, int run, int last, double* out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  const S* f = static_cast<const S*>(v.f) + run * v.run_stride;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_post<L, S>(f, v.plane, a, last, g);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) out[(long long)i * N + t] = (double)g[i];
}

// FP64 per-block partial sums of (drho, rho u) over active nodes; a fixed
// shared-memory tree order makes the result deterministic.
template <class L, class S>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(LevelView v, int run, int last,
                                                               double* partial) {
  __shared__ double sh[4][kDiagThreads];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s[4] = {0, 0, 0, 0};
  int x, y, z;
  if (node_of(v, t, x, y, z) && !inactive(v, x, y, z)) {
    const S* f = static_cast<const S*>(v.f) + run * v.run_stride;
    const NodeAddr a = node_addr<L>(v, x, y, z);
    float g[L::Q];
    load_post<L, S>(f, v.plane, a, last, g);
    sfor<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double gi = (double)g[i];
      s[0] += gi;
      s[1] += L::c(i, 0) * gi;
      s[2] += L::c(i, 1) * gi;
      s[3] += L::c(i, 2) * gi;
    });
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] = s[j];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) partial[(long long)j * gridDim.x + blockIdx.x] = sh[j][0];
}

// Probe sampling: rho, u of registered nodes of one level for every run,
// into slot (*counter % cap) of the record.  One block; thread 0 advances
// the counter after all threads have read it.
template <class L, class S>
__global__ void k_probe(LevelView v, int last, const int* ijk, int n, double* rec, int cap,
                        unsigned long long* counter, double rho0) {
  __shared__ unsigned long long slot;
  if (threadIdx.x == 0) slot = *counter;
  __syncthreads();
  const long long base = (long long)(slot % (unsigned long long)cap) * v.batch * n;
  for (int t = threadIdx.x; t < n * v.batch; t += blockDim.x) {
    const int run = t / n, k = t - run * n;
    const S* f = static_cast<const S*>(v.f) + run * v.run_stride;
    const NodeAddr a = node_addr<L>(v, ijk[3 * k], ijk[3 * k + 1], ijk[3 * k + 2]);
    float g[L::Q];
    load_post<L, S>(f, v.plane, a, last, g);
    float drho, jx, jy, jz;
    moments<L>(g, drho, jx, jy, jz);
    const double r = rho0 + (double)drho;
    double* o = rec + (base + (long long)run * n + k) * 4;
    o[0] = r;
    o[1] = jx / r;
    o[2] = jy / r;
    o[3] = (L::D == 3) ? jz / r : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = slot + 1;
}

}  // namespace mlbm
