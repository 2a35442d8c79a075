// Kernels of the hybrid recursive regularized collision (H-RR, Sec. 3.3,
// eq. a1ij_HRR) and of its strain-rate transfers at refinement interfaces
// (Sec. 4.4).  The collision needs S = (grad u + grad u^T) / 2 from
// second-order central differences of the pre-collision velocity, so a level
// step becomes
//
//   k_velocity            pre-collision velocity deviation du = u - U of every
//                         updated node into D planes laid out like the
//                         population planes;
//   k_stream_collide_hrr  the level update with S from those planes (middle
//                         nodes; TN nodes and, on refined levels, the outer
//                         node layer are left to the kernels below);
//   k_parent_strain       after a child's first sub-step: the parent's S at
//                         t+1 on the child box surface, with the velocity of
//                         the parent's TN nodes at t+1 from a fictitious
//                         streaming of the child's post-collision state; kept
//                         in a three-slot history like the populations';
//   k_collide_bnd         the child's outer node layer: S of the parent
//                         interpolated in time (eq. TempInt) and space
//                         (eq. spaceInt), halved (eq. PijResc), then the
//                         collision;
//   k_restrict_tile<HRR>  (kernels.cuh) collides each rebuilt TN node at once
//                         with S = 2 S^f of its co-located child node.
//
// Strain-rate history layout: sh[((run * 3 + slot) * 6 + j) * K + k],
// j = (xx, yy, zz, xy, xz, yz), k a history-ring entry.
#pragma once
#include "kernels.cuh"

namespace mlbm {

__device__ __forceinline__ bool tn_node(const LevelView& v, int x, int y, int z) {
  return v.has_tn && x >= v.tn_lo[0] && x <= v.tn_hi[0] && y >= v.tn_lo[1] &&
         y <= v.tn_hi[1] && z >= v.tn_lo[2] && z <= v.tn_hi[2] && !inactive(v, x, y, z);
}

template <class L>
__device__ __forceinline__ bool outer_geom(const LevelView& v, int x, int y, int z) {
  bool b = (!v.per[0] && (x == 0 || x == v.n[0] - 1)) ||
           (!v.per[1] && (y == 0 || y == v.n[1] - 1));
  if constexpr (L::D == 3) b = b || (!v.per[2] && (z == 0 || z == v.n[2] - 1));
  return b;
}

template <class L>
__device__ __forceinline__ bool outer_layer(const LevelView& v, int x, int y, int z) {
  if (!v.hrr) return false;
  bool b = (!v.per[0] && (x == 0 || x == v.n[0] - 1)) ||
           (!v.per[1] && (y == 0 || y == v.n[1] - 1));
  if constexpr (L::D == 3) b = b || (!v.per[2] && (z == 0 || z == v.n[2] - 1));
  return b;
}

// Post-collision store of an update of parity PAR (the level update's).
template <class L, class S, int I>
__device__ __forceinline__ void store_post_i(S* f, long long plane, const NodeAddr& a, int par,
                                             int es, float val) {
  if (par == 0)
    Store<S>::st(f + (long long)opp<L>(I) * plane + es * a.at(0, 0, 0), val);
  else
    Store<S>::st(f + (long long)I * plane + es * a.at(L::c(I, 0), L::c(I, 1), L::c(I, 2)), val);
}

// --------------------------------------------------------------- velocity
// (hybrid collision: TN nodes are left to the restriction, which writes
// their velocity; otherwise every active node)
template <class L, class S>
__global__ void k_velocity(LevelView v, float* du, int par, RefF ref) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  if (inactive(v, x, y, z) || (v.hrr && tn_node(v, x, y, z))) return;
  const S* f = run_cptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q], drho, u[3];
  load_pre<L, S>(f, v.plane, a, par, v.es, g);
  deviations<L>(g, ref, drho, u[0], u[1], u[2]);
  float* d = du + (long long)run * L::D * v.plane + a.at(0, 0, 0);
#pragma unroll
  for (int b = 0; b < L::D; ++b) d[(long long)b * v.plane] = u[b];
}

// ------------------------------------------------------ level update, H-RR
// One thread per node, 32 x 4 blocks like the plain update.  ks = -2 tau
// cs^2 (1 - sig) of this level.
template <class L, class S, int PAR, bool MOV>
__global__ void __launch_bounds__(128)
    k_stream_collide_hrr(LevelView v, float omega, RefF R, const float* du, float sig, float ks) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  int z = blockIdx.z, run = 0;
  if (v.batch > 1) {
    run = z / v.n[2];
    z -= run * v.n[2];
  }
  if (x >= v.n[0] || y >= v.n[1]) return;
  if (inactive(v, x, y, z) || tn_node(v, x, y, z) || outer_layer<L>(v, x, y, z)) return;
  S* f = run_ptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_pre<L, S>(f, v.plane, a, PAR, v.es, g);
  const float* d = du + (long long)run * L::D * v.plane;
  float up[3][3] = {}, um[3][3] = {};
#pragma unroll
  for (int ax = 0; ax < L::D; ++ax) {
    const int ep = a.at(ax == 0, ax == 1, ax == 2), em = a.at(-(ax == 0), -(ax == 1), -(ax == 2));
#pragma unroll
    for (int b = 0; b < L::D; ++b) {
      up[ax][b] = __ldg(d + (long long)b * v.plane + ep);
      um[ax][b] = __ldg(d + (long long)b * v.plane + em);
    }
  }
  HrrIn hy;
  hy.sig = sig;
  hy.ks = ks;
  strain_from<L>(up, um, hy.s);
  collide_emit<L, 3, MOV>(
      g, omega, R,
      [&](auto I, float val) {
        constexpr int i = decltype(I)::value;
        store_post_i<L, S, i>(f, v.plane, a, PAR, v.es, val);
      },
      &hy);
}

// ------------------------------------------------- parent strain history
// One thread per history-ring entry k (a parent node on the child box
// surface or one cell past its edges).  Central differences of the parent
// velocity at t+1 along each axis; a neighbour inside the restriction ring
// (a TN node) takes the velocity of the co-located child node after a
// fictitious streaming of the child's post-collision state (the child's
// pre-collision state for its next update, parity cpar); any other
// neighbour takes the parent's streamed state (pre-collision for the
// parent's next update, parity ppar).  mode 1 (set-up): every neighbour
// from the parent's current state (laid out after an update of parity ppar)
// into slots s_new and s_also.
template <class L, class S>
__global__ void k_parent_strain(LevelView p, LevelView c, RingDesc R, TnDesc T, float* sh,
                                int s_new, int s_also, int ppar, int cpar, int mode, RefF ref) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  if (k >= R.K) return;
  const int fc = ring_face(R.start, R.nf, k);
  long long loc = k - R.start[fc];
  int P[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = R.ext[fc][a];
    const int i = (int)(loc % e);
    loc /= e;
    int cc = R.base[fc][a] + i;
    if (R.pper[a]) cc = ((cc % R.pn[a]) + R.pn[a]) % R.pn[a];
    P[a] = cc;
  }
  const S* fp = run_cptr<S>(p, run);
  const S* fcb = run_cptr<S>(c, run);
  float up[3][3] = {}, um[3][3] = {};
  for (int ax = 0; ax < L::D; ++ax)
    for (int sg = 0; sg < 2; ++sg) {
      int Q[3] = {P[0], P[1], P[2]};
      Q[ax] += sg ? -1 : 1;
      if (p.per[ax]) Q[ax] = wrapi(Q[ax], p.n[ax]);
      float g[L::Q], drho, u[3];
      if (mode == 0 && p.has_tn && Q[0] >= p.tn_lo[0] && Q[0] <= p.tn_hi[0] &&
          Q[1] >= p.tn_lo[1] && Q[1] <= p.tn_hi[1] && Q[2] >= p.tn_lo[2] && Q[2] <= p.tn_hi[2]) {
        int X[3] = {0, 0, 0};
        for (int b = 0; b < L::D; ++b) X[b] = T.boxed[b] ? 2 * (Q[b] - T.lo[b]) : 2 * Q[b];
        load_pre<L, S>(fcb, c.plane, node_addr<L>(c, X[0], X[1], X[2]), cpar, c.es, g);
      } else if (mode == 0) {
        load_pre<L, S>(fp, p.plane, node_addr<L>(p, Q[0], Q[1], Q[2]), ppar, p.es, g);
      } else {
        load_post<L, S>(fp, p.plane, node_addr<L>(p, Q[0], Q[1], Q[2]), ppar, p.es, g);
      }
      deviations<L>(g, ref, drho, u[0], u[1], u[2]);
      for (int b = 0; b < 3; ++b) (sg ? um : up)[ax][b] = u[b];
    }
  float Sv[6];
  strain_from<L>(up, um, Sv);
  float* h = sh + (long long)run * 3 * 6 * R.K;
  for (int rep = 0; rep < (mode == 0 ? 1 : 2); ++rep) {
    float* hs = h + (long long)(rep == 0 ? s_new : s_also) * 6 * R.K + k;
#pragma unroll
    for (int j = 0; j < 6; ++j) hs[(long long)j * R.K] = Sv[j];
  }
}

// --------------------------------------------- child outer layer collision
// One thread per child boundary node (TF / IE).  The parent strain rate is
// interpolated in time with weights (w0, w1, w2) on slots (s_m1, s_0, s_p1)
// and in space with the eq. spaceInt stencil along the face's odd
// coordinates, halved (eq. PijResc); the node's pre-collision state (written
// by the rebuild for the update of parity par) is collided with it.
template <class L, class S, bool MOV>
__global__ void k_collide_bnd(LevelView c, BndDesc B, RingDesc R, const float* sh, float w0,
                              float w1, float w2, int s_m1, int s_0, int s_p1, float omega,
                              float sig, float ks, int par, RefF ref) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  if (k >= B.count) return;
  const int f = ring_face(B.start, B.nf, k);
  long long loc = k - B.start[f];
  int X[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = B.ext[f][a];
    X[a] = B.lo[f][a] + (int)(loc % e);
    loc /= e;
  }
  const int fa = B.axis[f];
  long long stride[3];
  stride[0] = 1;
  stride[1] = R.ext[f][0];
  stride[2] = stride[1] * R.ext[f][1];
  // stencil along (up to) two tangent axes
  int tax[2] = {-1, -1}, nt = 0;
  for (int b = 0; b < L::D; ++b)
    if (b != fa) tax[nt++] = b;
  int n_s[2] = {1, 1}, p0[2] = {0, 0};
  for (int t = 0; t < nt; ++t) {
    const int b = tax[t];
    if (X[b] & 1) {
      n_s[t] = 4;
      p0[t] = (X[b] - 3) / 2;
    } else {
      p0[t] = X[b] / 2;
    }
  }
  auto sw = [](int s) { return (s == 0 || s == 3) ? -1.0f / 16.0f : 9.0f / 16.0f; };
  const float* h = sh + (long long)run * 3 * 6 * R.K;
  float Sv[6] = {0, 0, 0, 0, 0, 0};
  for (int s0 = 0; s0 < n_s[0]; ++s0)
    for (int s1 = 0; s1 < n_s[1]; ++s1) {
      float w = 1.0f;
      long long idx = R.start[f];
      for (int t = 0; t < nt; ++t) {
        const int b = tax[t], s = t == 0 ? s0 : s1;
        if (n_s[t] == 4) w *= sw(s);
        int pc = p0[t] + s;  // parent coordinate (box-relative on bounded axes)
        if (R.boxed[b])
          pc += 1;  // ring entries start one parent cell before the box
        else
          pc = ((pc % R.pn[b]) + R.pn[b]) % R.pn[b];
        idx += (long long)pc * stride[b];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float vt = w0 * h[((long long)s_m1 * 6 + j) * R.K + idx] +
                         w1 * h[((long long)s_0 * 6 + j) * R.K + idx] +
                         w2 * h[((long long)s_p1 * 6 + j) * R.K + idx];
        Sv[j] += w * vt;
      }
    }
  HrrIn hy;
  hy.sig = sig;
  hy.ks = ks;
#pragma unroll
  for (int j = 0; j < 6; ++j) hy.s[j] = 0.5f * Sv[j];  // eq. PijResc
  S* fb = run_ptr<S>(c, run);
  const NodeAddr a = node_addr<L>(c, X[0], X[1], X[2]);
  float g[L::Q];
  load_pre<L, S>(fb, c.plane, a, par, c.es, g);
  collide_emit<L, 3, MOV>(
      g, omega, ref,
      [&](auto I, float val) {
        constexpr int i = decltype(I)::value;
        store_post_i<L, S, i>(fb, c.plane, a, par, c.es, val);
      },
      &hy);
}

}  // namespace mlbm
