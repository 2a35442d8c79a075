// Kernels of one multi-level step (Sec. 4.3, cell-vertex coupling):
//
//   k_stream_collide  fused stream + collide of every active node of a level
//                     (eq. LBMequation), in place with the AA pattern;
//   k_capture         parent pre-collision (drho, u, f^(1)) at t+1 on a child
//                     box surface -> three-slot history;
//   k_inject          child TF / IE nodes: temporal (eq. TempInt) and spatial
//                     (eq. spaceInt) interpolation staged per face tile in
//                     shared memory, rescaling (eq. rescff), written where
//                     the child's next update reads them (2D; k_inject_sep,
//                     the same with the stencil applied one axis at a time,
//                     in 3D);
//   k_restrict_tile   parent TN nodes: filtered child f^(1) (eq. filterFneq),
//                     rescaling (eq. rescfc), written where the parent's next
//                     update reads them (the restriction), per face tile; with
//                     the hybrid collision it also collides the TN nodes;
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
#include "lattice_x2.cuh"

namespace mlbm {

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// binary32 reference with its per-direction constants (formed on the host
// by make_ref_f in the launch wrappers)

// Element offsets of a node and of its 3^D neighbours inside a plane
// (32-bit: the host keeps every plane below 2^31 elements; plane bases are
// formed in 64 bits from warp-uniform values).
struct NodeAddr {
  int zo[3];
  int yo[3];
  int xo[3];
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return zo[dz + 1] + yo[dy + 1] + xo[dx + 1];
  }
};

template <class L>
__device__ __forceinline__ NodeAddr node_addr(const LevelView& v, int x, int y, int z) {
  NodeAddr a;
  const int off = (int)v.off;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int xx = x + d, yy = y + d;
    if (v.per[0]) xx = wrapi(xx, v.n[0]);
    if (v.per[1]) yy = wrapi(yy, v.n[1]);
    a.xo[d + 1] = xx + off;
    a.yo[d + 1] = yy * v.SX;
    if constexpr (L::D == 3) {
      int zz = z + d;
      if (v.per[2]) zz = wrapi(zz, v.n[2]);
      a.zo[d + 1] = zz * v.SY * v.SX;
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

// First element of run `run` (see LevelView for the layout).
template <class S>
__device__ __forceinline__ S* run_ptr(const LevelView& v, int run) {
  return static_cast<S*>(v.f) + (long long)(run / v.es) * v.run_stride + (run % v.es);
}
template <class S>
__device__ __forceinline__ const S* run_cptr(const LevelView& v, int run) {
  return static_cast<const S*>(v.f) + (long long)(run / v.es) * v.run_stride + (run % v.es);
}

// Pre-collision populations of node a for an update of parity PAR (es: the
// layout's element stride).
template <class L, class S>
__device__ __forceinline__ void load_pre(const S* f, long long plane, const NodeAddr& a, int par,
                                         int es, float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (par == 0)
      g[i] = Store<S>::ld(f + (long long)i * plane + es * a.at(0, 0, 0));
    else
      g[i] = Store<S>::ld(f + (long long)opp<L>(i) * plane +
                          es * a.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)));
  });
}

// Write populations into the cells an update of parity `par` reads.
template <class L, class S>
__device__ __forceinline__ void store_pre(S* f, long long plane, const NodeAddr& a, int par,
                                          int es, const float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (par == 0)
      Store<S>::st(f + (long long)i * plane + es * a.at(0, 0, 0), g[i]);
    else
      Store<S>::st(
          f + (long long)opp<L>(i) * plane + es * a.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)),
          g[i]);
  });
}

// Post-collision populations of node a after an update of parity `last`
// (initial states are written like a parity-0 update).
template <class L, class S>
__device__ __forceinline__ void load_post(const S* f, long long plane, const NodeAddr& a,
                                          int last, int es, float (&g)[L::Q]) {
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (last == 0)
      g[i] = Store<S>::ld(f + (long long)opp<L>(i) * plane + es * a.at(0, 0, 0));
    else
      g[i] = Store<S>::ld(f + (long long)i * plane +
                          es * a.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)));
  });
}

// ------------------------------------------------------- K1: level update
// One thread per node; a warp covers 32 consecutive x of one row.
// Launch shape of the level update per lattice and storage type: NPT nodes
// per thread (consecutive rows, so a thread keeps NPT x q loads in flight)
// and the resident blocks per SM its register budget is compiled for
// (MINB; MINB_EVEN for the even step, whose accesses share one address;
// MINB_MOV with a moving reference, whose deviation terms need more
// registers).  Chosen by measurement (the shape sweep in the benchmarks).
template <class L, class S>
struct K1Tune;
// (each value may be overridden at compile time, e.g. -DK1_NPT_D2Q9_F=1)
#ifndef K1_NPT_D2Q9_F
#define K1_NPT_D2Q9_F 1
#endif
#ifndef K1_MINB_D2Q9_F
#define K1_MINB_D2Q9_F 12
#endif
#ifndef K1_MINBE_D2Q9_F
#define K1_MINBE_D2Q9_F K1_MINB_D2Q9_F
#endif
#ifndef K1_MINBM_D2Q9_F
#define K1_MINBM_D2Q9_F 10
#endif
#ifndef K1_NPT_D2Q9_H
#define K1_NPT_D2Q9_H 2
#endif
#ifndef K1_MINB_D2Q9_H
#define K1_MINB_D2Q9_H 6
#endif
#ifndef K1_MINBE_D2Q9_H
#define K1_MINBE_D2Q9_H K1_MINB_D2Q9_H
#endif
#ifndef K1_MINBM_D2Q9_H
#define K1_MINBM_D2Q9_H 6
#endif
#ifndef K1_NPT_D3Q19_F
#define K1_NPT_D3Q19_F 1
#endif
#ifndef K1_MINB_D3Q19_F
#define K1_MINB_D3Q19_F 6
#endif
#ifndef K1_MINBE_D3Q19_F
#define K1_MINBE_D3Q19_F 7
#endif
#ifndef K1_MINBM_D3Q19_F
#define K1_MINBM_D3Q19_F 5
#endif
#ifndef K1_NPT_D3Q19_H
#define K1_NPT_D3Q19_H 1
#endif
#ifndef K1_MINB_D3Q19_H
#define K1_MINB_D3Q19_H 6
#endif
#ifndef K1_MINBE_D3Q19_H
#define K1_MINBE_D3Q19_H K1_MINB_D3Q19_H
#endif
#ifndef K1_MINBM_D3Q19_H
#define K1_MINBM_D3Q19_H 5
#endif
#ifndef K1_NPT_D3Q27_F
#define K1_NPT_D3Q27_F 1
#endif
#ifndef K1_MINB_D3Q27_F
#define K1_MINB_D3Q27_F 5
#endif
#ifndef K1_MINBE_D3Q27_F
#define K1_MINBE_D3Q27_F 6
#endif
#ifndef K1_MINBM_D3Q27_F
#define K1_MINBM_D3Q27_F 4
#endif
#ifndef K1_NPT_D3Q27_H
#define K1_NPT_D3Q27_H 1
#endif
#ifndef K1_MINB_D3Q27_H
#define K1_MINB_D3Q27_H 5
#endif
#ifndef K1_MINBE_D3Q27_H
#define K1_MINBE_D3Q27_H K1_MINB_D3Q27_H
#endif
#ifndef K1_MINBM_D3Q27_H
#define K1_MINBM_D3Q27_H 4
#endif
template <>
struct K1Tune<D2Q9, float> {
  static constexpr int NPT = K1_NPT_D2Q9_F, MINB = K1_MINB_D2Q9_F,
                       MINB_EVEN = K1_MINBE_D2Q9_F, MINB_MOV = K1_MINBM_D2Q9_F;
};
template <>
struct K1Tune<D2Q9, __half> {
  static constexpr int NPT = K1_NPT_D2Q9_H, MINB = K1_MINB_D2Q9_H,
                       MINB_EVEN = K1_MINBE_D2Q9_H, MINB_MOV = K1_MINBM_D2Q9_H;
};
template <>
struct K1Tune<D3Q19, float> {
  static constexpr int NPT = K1_NPT_D3Q19_F, MINB = K1_MINB_D3Q19_F,
                       MINB_EVEN = K1_MINBE_D3Q19_F, MINB_MOV = K1_MINBM_D3Q19_F;
};
template <>
struct K1Tune<D3Q19, __half> {
  static constexpr int NPT = K1_NPT_D3Q19_H, MINB = K1_MINB_D3Q19_H,
                       MINB_EVEN = K1_MINBE_D3Q19_H, MINB_MOV = K1_MINBM_D3Q19_H;
};
template <>
struct K1Tune<D3Q27, float> {
  static constexpr int NPT = K1_NPT_D3Q27_F, MINB = K1_MINB_D3Q27_F,
                       MINB_EVEN = K1_MINBE_D3Q27_F, MINB_MOV = K1_MINBM_D3Q27_F;
};
template <>
struct K1Tune<D3Q27, __half> {
  static constexpr int NPT = K1_NPT_D3Q27_H, MINB = K1_MINB_D3Q27_H,
                       MINB_EVEN = K1_MINBE_D3Q27_H, MINB_MOV = K1_MINBM_D3Q27_H;
};

// Addresses of a strip of NPT consecutive rows (same x and z): node k's
// neighbour (dx, dy, dz) sits at zo[dz+1] + yo[k+dy+1] + xo[dx+1].
template <int NPT>
struct StripAddr {
  int zo[3];
  int yo[NPT + 2];
  int xo[3];
  __device__ __forceinline__ int at(int k, int dx, int dy, int dz) const {
    return zo[dz + 1] + yo[k + dy + 1] + xo[dx + 1];
  }
};

// Face buffer of a level whose x axis is bounded by its box: the rebuilt
// pre-collision populations of the nodes on the two faces normal to x
// (x = 0: side 0, x = n[0] - 1: side 1), written there by the coarse ->
// fine rebuild instead of into the level's planes.  On those faces x is
// the fastest axis of the planes, so each rebuilt population would land in
// its own 32-byte sector; in the face buffer a face is a plane of its own
// (y fastest), written and read in whole sectors.  Element of run r,
// side s, direction i, face node (y, z):
//   ((((r / es) * 2 + s) * q + i) * F + z * n[1] + y) * es + r % es,
// F = n[1] * n[2].  (3D levels only: a 2D face holds n[1] nodes of q = 9
// populations, where the scattered stores cost little.)  The level update
// reads a face node's populations from
// here; a warp holds such a node only if it covers x = 0 or x = n[0] - 1,
// and only those warps load from the face buffer (a warp-uniform branch
// after the loads every lane issues from the planes, so that the other
// warps run the same code as without face buffers).
__device__ __forceinline__ bool warp_has_xface(const LevelView& v, const void* xf) {
  const int xw = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  return xf != nullptr && (xw == 0 || (xw <= v.n[0] - 1 && v.n[0] - 1 < xw + 32));
}

// One thread updates NPT nodes (x, y0 .. y0+NPT-1, z); a warp covers 32
// consecutive x of NPT rows.  All loads of the thread's nodes are issued
// before the first collision.  The block shape (blockDim.x a multiple of 32,
// blockDim.x * blockDim.y <= 128) is chosen at run time (lbm_autotune); it
// changes which nodes share a block, not any node's arithmetic.
template <class L, int COLL, class S, int PAR, bool MOV>
__global__ void __launch_bounds__(128, MOV ? K1Tune<L, S>::MINB_MOV
                                           : (PAR == 0 ? K1Tune<L, S>::MINB_EVEN
                                                       : K1Tune<L, S>::MINB))
    k_stream_collide(LevelView v, float omega, RefF R, const S* __restrict__ xf) {
  constexpr int NPT = K1Tune<L, S>::NPT;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * NPT;
  int z = blockIdx.z, run = 0;
  if (v.batch > 1) {
    run = z / v.n[2];
    z -= run * v.n[2];
  }
  if (x >= v.n[0] || y0 >= v.n[1]) return;
  S* f = static_cast<S*>(v.f) + run * v.run_stride;  // es = 1 for this kernel
  StripAddr<NPT> a;
  const int off = (int)v.off;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int xx = x + d;
    if (v.per[0]) xx = wrapi(xx, v.n[0]);
    a.xo[d + 1] = xx + off;
    if constexpr (L::D == 3) {
      int zz = z + d;
      if (v.per[2]) zz = wrapi(zz, v.n[2]);
      a.zo[d + 1] = zz * v.SY * v.SX;
    } else {
      a.zo[d + 1] = 0;
    }
  }
#pragma unroll
  for (int r = 0; r < NPT + 2; ++r) {
    int yy = y0 - 1 + r;
    if (v.per[1]) yy = wrapi(yy, v.n[1]);
    a.yo[r] = yy * v.SX;
  }
  // a lane on a face normal to x takes its populations from the face buffer:
  // every lane loads from the planes, then only warps holding such a lane
  // (a warp-uniform branch) replace that lane's values by the face buffer's
  const bool fw = warp_has_xface(v, xf);
  const bool fx = fw && (x == 0 || x == v.n[0] - 1);
  bool ok[NPT];
  float g[NPT][L::Q];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    ok[k] = (y0 + k < v.n[1]) && !inactive(v, x, y0 + k, z);
    if (ok[k]) {
      sfor<L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (PAR == 0)
          g[k][i] = Store<S>::ld(f + (long long)i * v.plane + a.at(k, 0, 0, 0));
        else
          g[k][i] = Store<S>::ld(f + (long long)opp<L>(i) * v.plane +
                                 a.at(k, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2)));
      });
    }
  }
  if constexpr (L::D == 3) {  // (2D levels have no face buffer)
    if (fw && fx) {
      const long long F = (long long)v.n[1] * v.n[2];
      const S* xb =
          xf + ((long long)run * 2 + (x != 0)) * L::Q * F + (long long)z * v.n[1] + y0;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        if (!ok[k]) continue;
        sfor<L::Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          g[k][i] = Store<S>::ld(xb + i * F + k);
        });
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    if (!ok[k]) continue;
    collide_emit<L, COLL, MOV>(g[k], omega, R, [&](auto I, float val) {
      constexpr int i = decltype(I)::value;
      if constexpr (PAR == 0)
        Store<S>::st(f + (long long)opp<L>(i) * v.plane + a.at(k, 0, 0, 0), val);
      else
        Store<S>::st(f + (long long)i * v.plane + a.at(k, L::c(i, 0), L::c(i, 1), L::c(i, 2)),
                     val);
    });
  }
}

// Level update, two nodes per thread in one two-lane collision: the nodes
// (x, y0) and (x, y0 + 1) take the two lanes of the packed FP32 arithmetic
// (lattice_x2.cuh), so their collisions issue about half the floating-point
// instructions of two scalar collisions.  A lane whose node is outside the
// level or inactive computes on its partner's populations and stores
// nothing.  Per lattice, K1X2_<lattice> selects this kernel over
// k_stream_collide for binary32, K1X2H_<lattice> for binary16 with one run
// per element (es = 1), and K1X2_MINB_<lattice> / K1X2H_MINB_<lattice> set
// the resident blocks per SM each is compiled for.
#ifndef K1X2H_D2Q9
#define K1X2H_D2Q9 1
#endif
#ifndef K1X2H_D3Q19
#define K1X2H_D3Q19 1
#endif
#ifndef K1X2H_D3Q27
#define K1X2H_D3Q27 1
#endif
#ifndef K1X2_D2Q9
#define K1X2_D2Q9 0
#endif
#ifndef K1X2H_MINB_D2Q9
#define K1X2H_MINB_D2Q9 K1X2_MINB_D2Q9
#endif
#ifndef K1X2H_MINB_D3Q19
#define K1X2H_MINB_D3Q19 K1X2_MINB_D3Q19
#endif
#ifndef K1X2H_MINB_D3Q27
#define K1X2H_MINB_D3Q27 K1X2_MINB_D3Q27
#endif
#ifndef K1X2_D3Q19
#define K1X2_D3Q19 1
#endif
#ifndef K1X2_D3Q27
#define K1X2_D3Q27 1
#endif
#ifndef K1X2_MINB_D2Q9
#define K1X2_MINB_D2Q9 8
#endif
#ifndef K1X2_MINB_D3Q19
#define K1X2_MINB_D3Q19 4
#endif
#ifndef K1X2_MINB_D3Q27
#define K1X2_MINB_D3Q27 3
#endif
// MINB1: resident blocks of the binary32 odd-parity update, whose shifted
// addresses need more registers: at the even update's bound it spilled
// (D3Q19: 104 bytes at 128 registers); one block fewer holds it in
// registers (D3Q19 168, D3Q27 252), +3 % on the D3Q19 slab's step and +2 %
// on the nested D3Q27 case (GB300); both parities at the lower bound were
// slower.
#ifndef K1X2H_MINB1_D2Q9
#define K1X2H_MINB1_D2Q9 K1X2H_MINB_D2Q9
#endif
#ifndef K1X2H_MINB1_D3Q19
#define K1X2H_MINB1_D3Q19 K1X2H_MINB_D3Q19
#endif
#ifndef K1X2H_MINB1_D3Q27
#define K1X2H_MINB1_D3Q27 K1X2H_MINB_D3Q27
#endif
#ifndef K1X2_MINB1_D2Q9
#define K1X2_MINB1_D2Q9 K1X2_MINB_D2Q9
#endif
#ifndef K1X2_MINB1_D3Q19
#define K1X2_MINB1_D3Q19 3
#endif
#ifndef K1X2_MINB1_D3Q27
#define K1X2_MINB1_D3Q27 2
#endif
template <class L>
struct K1X2Tune;
template <>
struct K1X2Tune<D2Q9> {
  static constexpr bool ON = K1X2_D2Q9;
  static constexpr bool ON_H = K1X2H_D2Q9;
  static constexpr int MINB = K1X2_MINB_D2Q9;
  static constexpr int MINB1 = K1X2_MINB1_D2Q9;
  static constexpr int MINB_H = K1X2H_MINB_D2Q9;
  static constexpr int MINB1_H = K1X2H_MINB1_D2Q9;
};
template <>
struct K1X2Tune<D3Q19> {
  static constexpr bool ON = K1X2_D3Q19;
  static constexpr bool ON_H = K1X2H_D3Q19;
  static constexpr int MINB = K1X2_MINB_D3Q19;
  static constexpr int MINB1 = K1X2_MINB1_D3Q19;
  static constexpr int MINB_H = K1X2H_MINB_D3Q19;
  static constexpr int MINB1_H = K1X2H_MINB1_D3Q19;
};
template <>
struct K1X2Tune<D3Q27> {
  static constexpr bool ON = K1X2_D3Q27;
  static constexpr bool ON_H = K1X2H_D3Q27;
  static constexpr int MINB = K1X2_MINB_D3Q27;
  static constexpr int MINB1 = K1X2_MINB1_D3Q27;
  static constexpr int MINB_H = K1X2H_MINB_D3Q27;
  static constexpr int MINB1_H = K1X2H_MINB1_D3Q27;
};

// z-planes per thread of the two-node update (1: one node pair per thread;
// more: the thread walks that many consecutive planes and prefetches the
// next plane's populations into L2 before colliding the current one, which
// keeps DRAM reads in flight during the collision without holding
// registers).  Binary32: 8 planes (against one: +9 % on the D3Q19 slab;
// against four: +1.3 % there and +1 % on the nested D3Q27 case; sixteen
// measured no better); binary16: 1 (its update is nearer the instruction
// limit: the prefetches cost it 5-7 %).  Measured on GB300.
#ifndef K1X2_PFZ_F
#define K1X2_PFZ_F 8
#endif
#ifndef K1X2_PFZ_H
#define K1X2_PFZ_H 1
#endif
template <class S>
struct K1X2Pfz {
  static constexpr int PZ = std::is_same<S, float>::value ? K1X2_PFZ_F : K1X2_PFZ_H;
};

// Element offsets of the two-node update within a run are 32-bit (the
// launcher takes it only for runs below 2^31 elements; larger runs take the
// one-node update): 2 % faster on the D3Q19 slab than 64-bit offsets.
using X2Idx = int;

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <class L, class S, int COLL, int PAR, bool MOV>
__device__ __forceinline__ void stream_collide_x2_pair(const LevelView& v, float omega,
                                                       const RefF& R, const S* __restrict__ xf,
                                                       int x, int y0, int z, int run) {
  const bool ok0 = y0 < v.n[1] && !inactive(v, x, y0, z);
  const bool ok1 = y0 + 1 < v.n[1] && !inactive(v, x, y0 + 1, z);
  if (!ok0 && !ok1) return;
  S* f = static_cast<S*>(v.f) + run * v.run_stride;  // es = 1 for this kernel
  // each lane's node; an idle lane reads its partner's
  const NodeAddr a0 = node_addr<L>(v, x, ok0 ? y0 : y0 + 1, z);
  const NodeAddr a1 = node_addr<L>(v, x, ok1 ? y0 + 1 : y0, z);
  // a lane on a face normal to x takes its populations from the face buffer:
  // every lane loads from the planes, then only warps holding such a lane
  // (a warp-uniform branch) replace that lane's values by the face buffer's
  const bool fw = warp_has_xface(v, xf);
  const bool fx = fw && (x == 0 || x == v.n[0] - 1);
  // element offsets are formed whole before indexing (f[i * plane + at]):
  // per-direction base pointers would cost 64-bit registers per direction
  F2 g[L::Q];
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (PAR == 0) {
      g[i].v.x = Store<S>::ld(&f[(X2Idx)i * (X2Idx)v.plane + a0.at(0, 0, 0)]);
      g[i].v.y = Store<S>::ld(&f[(X2Idx)i * (X2Idx)v.plane + a1.at(0, 0, 0)]);
    } else {
      g[i].v.x = Store<S>::ld(
          &f[(X2Idx)opp<L>(i) * (X2Idx)v.plane + a0.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2))]);
      g[i].v.y = Store<S>::ld(
          &f[(X2Idx)opp<L>(i) * (X2Idx)v.plane + a1.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2))]);
    }
  });
  if constexpr (L::D == 3) {  // (2D levels have no face buffer)
    if (fw && fx) {
      const long long F = (long long)v.n[1] * v.n[2];
      const S* xb = xf + ((long long)run * 2 + (x != 0)) * L::Q * F + (long long)z * v.n[1];
      const S* xb0 = xb + (ok0 ? y0 : y0 + 1);
      const S* xb1 = xb + (ok1 ? y0 + 1 : y0);
      sfor<L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        g[i].v.x = Store<S>::ld(xb0 + i * F);
        g[i].v.y = Store<S>::ld(xb1 + i * F);
      });
    }
  }
  collide_emit_x2<L, COLL, MOV>(g, omega, R, [&](auto I, F2 val) {
    constexpr int i = decltype(I)::value;
    if constexpr (PAR == 0) {
      if (ok0) Store<S>::st(&f[(X2Idx)opp<L>(i) * (X2Idx)v.plane + a0.at(0, 0, 0)], val.v.x);
      if (ok1) Store<S>::st(&f[(X2Idx)opp<L>(i) * (X2Idx)v.plane + a1.at(0, 0, 0)], val.v.y);
    } else {
      if (ok0)
        Store<S>::st(&f[(X2Idx)i * (X2Idx)v.plane + a0.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))],
                     val.v.x);
      if (ok1)
        Store<S>::st(&f[(X2Idx)i * (X2Idx)v.plane + a1.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))],
                     val.v.y);
    }
  });
}

template <class L, class S, int COLL, int PAR, bool MOV>
__global__ void __launch_bounds__(128, std::is_same<S, float>::value
                                           ? (PAR ? K1X2Tune<L>::MINB1 : K1X2Tune<L>::MINB)
                                           : (PAR ? K1X2Tune<L>::MINB1_H : K1X2Tune<L>::MINB_H))
    k_stream_collide_x2(LevelView v, float omega, RefF R, const S* __restrict__ xf) {
  constexpr int PZ = K1X2Pfz<S>::PZ;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * 2;
  const int nzb = (v.n[2] + PZ - 1) / PZ;  // z blocks per run
  int zc = blockIdx.z, run = 0;
  if (v.batch > 1) {
    run = zc / nzb;
    zc -= run * nzb;
  }
  if (x >= v.n[0]) return;
  if constexpr (PZ == 1) {
    stream_collide_x2_pair<L, S, COLL, PAR, MOV>(v, omega, R, xf, x, y0, zc, run);
  } else {
    const S* f = static_cast<const S*>(v.f) + run * v.run_stride;
    const int ya = y0 < v.n[1] ? y0 : v.n[1] - 1, yb = y0 + 1 < v.n[1] ? y0 + 1 : ya;
#pragma unroll 1
    for (int k = 0; k < PZ; ++k) {
      const int z = zc * PZ + k;
      if (z >= v.n[2]) break;
      // the next plane's populations into L2 (not for nodes a parent level
      // leaves to its child: they are not updated)
      if (k + 1 < PZ && z + 1 < v.n[2] &&
          !(inactive(v, x, ya, z + 1) && inactive(v, x, yb, z + 1))) {
        const NodeAddr p0 = node_addr<L>(v, x, ya, z + 1), p1 = node_addr<L>(v, x, yb, z + 1);
        sfor<L::Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          if constexpr (PAR == 0) {
            prefetch_l2(&f[(X2Idx)i * (X2Idx)v.plane + p0.at(0, 0, 0)]);
            prefetch_l2(&f[(X2Idx)i * (X2Idx)v.plane + p1.at(0, 0, 0)]);
          } else {
            prefetch_l2(&f[(X2Idx)opp<L>(i) * (X2Idx)v.plane +
                           p0.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2))]);
            prefetch_l2(&f[(X2Idx)opp<L>(i) * (X2Idx)v.plane +
                           p1.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2))]);
          }
        });
      }
      stream_collide_x2_pair<L, S, COLL, PAR, MOV>(v, omega, R, xf, x, y0, z, run);
    }
  }
}

// Level update of binary16 storage with runs interleaved in pairs (es = 2):
// one thread updates one node of runs 2p and 2p+1, moving each direction of
// both runs with one 4-byte access (a half2 of the two runs' values), and
// computes the two collisions as one two-lane collision on the packed FP32
// instructions (lattice_x2.cuh).  The last
// pair of an odd batch carries an unused run that stays at rest (zero
// deviations collide to zero; no interface kernel touches it).
template <class L>
struct K1PairTune;
#ifndef K1P_MINB_D2Q9
#define K1P_MINB_D2Q9 10
#endif
#ifndef K1P_MINB_D3Q19
#define K1P_MINB_D3Q19 4
#endif
#ifndef K1P_MINB_D3Q27
#define K1P_MINB_D3Q27 3
#endif
template <>
struct K1PairTune<D2Q9> {
  static constexpr int MINB = K1P_MINB_D2Q9;
};
template <>
struct K1PairTune<D3Q19> {
  static constexpr int MINB = K1P_MINB_D3Q19;
};
template <>
struct K1PairTune<D3Q27> {
  static constexpr int MINB = K1P_MINB_D3Q27;
};

template <class L, int COLL, int PAR, bool MOV>
__global__ void __launch_bounds__(128, K1PairTune<L>::MINB)
    k_stream_collide_pair(LevelView v, float omega, RefF R, const __half* __restrict__ xf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int npairs = (v.batch + 1) / 2;
  int z = blockIdx.z, pair = 0;
  if (npairs > 1) {
    pair = z / v.n[2];
    z -= pair * v.n[2];
  }
  if (x >= v.n[0] || y >= v.n[1] || inactive(v, x, y, z)) return;
  // half2 units: a plane is plane / 2 of them, node e sits at e
  __half2* f = reinterpret_cast<__half2*>(static_cast<__half*>(v.f) + pair * v.run_stride);
  const long long ph = v.plane / 2;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  // a lane on a face normal to x takes its populations from the face buffer
  // (after the loads from the planes, in warps holding such a lane only)
  const bool fw = warp_has_xface(v, xf);
  const bool fx = fw && (x == 0 || x == v.n[0] - 1);
  F2 g[L::Q];  // lane x: run 2p, lane y: run 2p+1
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    __half2 h;
    if constexpr (PAR == 0)
      h = f[i * ph + a.at(0, 0, 0)];
    else
      h = f[opp<L>(i) * ph + a.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2))];
    g[i].v = __half22float2(h);
  });
  if constexpr (L::D == 3) {  // (2D levels have no face buffer)
    if (fw && fx) {
      const long long F = (long long)v.n[1] * v.n[2];
      const __half2* xb = reinterpret_cast<const __half2*>(xf) +
                          ((long long)pair * 2 + (x != 0)) * L::Q * F + (long long)z * v.n[1] + y;
      sfor<L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        g[i].v = __half22float2(xb[i * F]);
      });
    }
  }
  collide_emit_x2<L, COLL, MOV>(g, omega, R, [&](auto I, F2 val) {
    constexpr int i = decltype(I)::value;
    const __half2 h = __float22half2_rn(val.v);
    if constexpr (PAR == 0)
      f[opp<L>(i) * ph + a.at(0, 0, 0)] = h;
    else
      f[i * ph + a.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))] = h;
  });
}

// (drho, du, f^(1)) of a population set (deviations from the reference).
template <class L>
__device__ __forceinline__ void split_neq(const float (&g)[L::Q], const RefF& R, float& drho,
                                          float& dux, float& duy, float& duz,
                                          float (&f1)[L::Q]) {
  deviations<L>(g, R, drho, dux, duy, duz);
  float g0[L::Q];
  equilibrium_f<L>(drho, dux, duy, duz, R, g0);
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
// The history keeps three slots that rotate: the host passes the slot that
// receives the newest state.  mode 0: store the parent's pre-collision state
// for an update of parity `par` into slot `s_new`.  mode 1 (set-up): store
// (drho, du, 0) of the parent's current state (laid out after an update of
// parity `par`) into slots `s_new` and `s_also`.
template <class L, class S>
__device__ __forceinline__ void capture_item(const LevelView& p, const RingDesc& R, int par,
                                             int mode, int s_new, int s_also, const RefF& ref,
                                             long long k, int run) {
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
  const S* f = run_cptr<S>(p, run);
  const NodeAddr a = node_addr<L>(p, P[0], P[1], P[2]);
  float g[L::Q];
  if (mode == 0)
    load_pre<L, S>(f, p.plane, a, par, p.es, g);
  else
    load_post<L, S>(f, p.plane, a, par, p.es, g);
  float drho, dux, duy, duz, f1[L::Q];
  split_neq<L>(g, ref, drho, dux, duy, duz, f1);
  const int nv = R.nv;
  float* h = R.hist + (long long)run * 3 * nv * R.K;
  const float m4[4] = {drho, dux, duy, duz};
  for (int rep = 0; rep < (mode == 0 ? 1 : 2); ++rep) {
    float* hs = h + (long long)(rep == 0 ? s_new : s_also) * nv * R.K + k;
#pragma unroll
    for (int vv = 0; vv < 4; ++vv) hs[(long long)vv * R.K] = m4[vv];
    sfor<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      hs[(long long)(4 + i) * R.K] = (mode == 0) ? f1[i] : 0.0f;
    });
  }
}

template <class L, class S>
__global__ void k_capture(LevelView p, RingDesc R, int par, int mode, int s_new, int s_also,
                          RefF ref) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R.K) return;
  capture_item<L, S>(p, R, par, mode, s_new, s_also, ref, k, blockIdx.y);
}

// ------------------------------------------------------------- K3: inject
// Child TF / IE nodes (the outer node layer of the child box).  wt: temporal
// weights on the history slots s_m1, s_0, s_p1 holding t-1, t, t+1;
// resc = tau_f / (2 tau_c) (eq. rescff); par: the child's next update.
// Organised by face tiles: a block covers TI x TJ child nodes of one face of
// the child box with G thread groups.  It first stages the temporally
// interpolated parent history (eq. TempInt) of the parent nodes the tile's
// stencils reach in shared memory (all threads); then the G threads of a
// node share its spatial stencil (eq. spaceInt, tensor product on face
// centres), each for every G-th interpolated value; then they share its
// rebuild (eq. rescff) and stores, each for every G-th direction.  Each
// history value is read once per tile instead of once per stencil use, and
// a node's serial work is split G ways (the kernel is latency-bound: a
// surface's worth of nodes does not fill the GPU).
#ifndef INJ_TJ_3D
#define INJ_TJ_3D 8
#endif
#ifndef INJ_G_3D
#define INJ_G_3D 1
#endif
#ifndef INJ_G_2D
#define INJ_G_2D 4
#endif
template <class L>
struct InjTile {
  static constexpr int TI = 32;                           // along the first tangent axis
  static constexpr int TJ = (L::D == 3) ? INJ_TJ_3D : 1;  // along the second
  static constexpr int G = (L::D == 3) ? INJ_G_3D : INJ_G_2D;  // thread groups per node
  static constexpr int WI = TI / 2 + 5;           // parent window (stencil reach)
  static constexpr int WJ = (L::D == 3) ? TJ / 2 + 5 : 1;
  static constexpr int NV = 4 + L::Q;
  static constexpr int NT = TI * TJ * G;
};

// Write direction I into the cell an update of parity `par` reads.
template <class L, class S, int I>
__device__ __forceinline__ void store_pre_i(S* f, long long plane, const NodeAddr& a, int par,
                                            int es, float v) {
  if (par == 0)
    Store<S>::st(f + (long long)I * plane + es * a.at(0, 0, 0), v);
  else
    Store<S>::st(
        f + (long long)opp<L>(I) * plane + es * a.at(-L::c(I, 0), -L::c(I, 1), -L::c(I, 2)), v);
}

// Rebuild f = f0(rho, u) + resc f^(1) (eq. rescff) of child node (x, y, z)
// from its interpolated values val(j) = (drho, du, f^(1)) and store, from
// thread group grp of G, every G-th direction where the child's update of
// parity par reads it -- or, for a node on a face normal to x when the
// level has a face buffer (xs = its side, 0 or 1; -1 otherwise), into the
// face buffer xf (its layout: see warp_has_xface).
template <class L, class S, int G, class V>
__device__ __forceinline__ void inject_rebuild(const LevelView& c, int run, int x, int y, int z,
                                               int par, float resc, const RefF& ref, int grp,
                                               V val, S* xf, int xs) {
  const float drho = val(0), dux = val(1), duy = val(2);
  const float duz = (L::D == 3) ? val(3) : 0.0f;
  const float Ux = ref.Ux, Uy = ref.Uy, Uz = (L::D == 3) ? ref.Uz : 0.0f;
  const float ux = Ux + dux, uy = Uy + duy, uz = Uz + duz;
  float A[7], dA[7];
  third_coeffs(ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, A, dA);
  const float dusq = 1.5f * (dux * (ux + Ux) + duy * (uy + Uy) + duz * (uz + Uz));
  const float rho = ref.rho0 + drho;
  S* fb = run_ptr<S>(c, run);
  const NodeAddr ad = node_addr<L>(c, x, y, z);
  const long long F = (long long)c.n[1] * c.n[2];
  S* xb = nullptr;
  if (xs >= 0)
    xb = xf + ((((long long)(run / c.es) * 2 + xs) * L::Q * F + (long long)z * c.n[1] + y) * c.es +
               run % c.es);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (i % G == grp) {
      const float g = eq_i<L, i, true>(drho, rho, dux, duy, duz, dusq, dA, ref) +
                      resc * val(4 + i);
      if (xs >= 0)
        Store<S>::st(xb + (long long)i * F * c.es, g);
      else
        store_pre_i<L, S, i>(fb, c.plane, ad, par, c.es, g);
    }
  });
}

template <class L, class S>
__global__ void __launch_bounds__(InjTile<L>::NT)
    k_inject(LevelView c, InjDesc J, RingDesc R, float w0, float w1, float w2, int s_m1,
             int s_0, int s_p1, float resc, int par, RefF ref, S* xf) {
  using T = InjTile<L>;
  constexpr bool SPLIT = T::G > 1;  // a node's values shared through shared memory
  __shared__ float sv[T::NV][T::WJ][T::WI];
  __shared__ float res[SPLIT ? T::NV : 1][SPLIT ? T::TJ : 1][SPLIT ? T::TI : 1];
  const int run = blockIdx.y;
  // tile -> face, tile coordinates
  int f = 0;
  while (f + 1 < J.nf && (long long)blockIdx.x >= J.tstart[f + 1]) ++f;
  const int tile = (int)(blockIdx.x - J.tstart[f]);
  const int a = J.axis[f], t1 = J.t1[f], t2 = J.t2[f];
  const int X0 = (tile % J.ntile1[f]) * T::TI;
  const int Y0 = (tile / J.ntile1[f]) * T::TJ;
  const int p0i = (X0 >> 1) - 2, p0j = (L::D == 3) ? (Y0 >> 1) - 2 : 0;
  // per-face scalars picked without indexing local arrays
  auto pick = [](const int (&v)[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); };
  const long long ext0 = R.ext[f][0], ext01 = ext0 * R.ext[f][1];
  const long long st1 = t1 == 0 ? 1 : (t1 == 1 ? ext0 : ext01);
  const long long st2 = t2 == 0 ? 1 : (t2 == 1 ? ext0 : ext01);
  const int bx1 = pick(R.boxed, t1), bx2 = pick(R.boxed, t2);
  const int e1 = pick(R.ext[f], t1), e2 = pick(R.ext[f], t2);
  const int pn1 = pick(R.pn, t1), pn2 = pick(R.pn, t2);
  const float* h = R.hist + (long long)run * 3 * R.nv * R.K;
  const long long K = R.K, nv = R.nv;
  const bool one_slot = w0 == 0.0f && w1 == 0.0f;  // uniform over the grid
  // stage: parent window x values, interpolated in time
  const int tid = (threadIdx.z * T::TJ + threadIdx.y) * T::TI + threadIdx.x;
#pragma unroll 4
  for (int e = tid; e < T::NV * T::WJ * T::WI; e += T::NT) {
    const int pi = e % T::WI, pj = (e / T::WI) % T::WJ, vv = e / (T::WI * T::WJ);
    int ri = p0i + pi, rj = p0j + pj;  // parent coordinates relative to the box / absolute
    bool ok = true;
    long long idx = R.start[f];
    // first tangent axis
    if (bx1) {
      ok = ok && ri >= -1 && ri <= e1 - 2;
      idx += (long long)(ri + 1) * st1;
    } else {
      ri = ((ri % pn1) + pn1) % pn1;
      idx += (long long)ri * st1;
    }
    if (L::D == 3) {
      if (bx2) {
        ok = ok && rj >= -1 && rj <= e2 - 2;
        idx += (long long)(rj + 1) * st2;
      } else {
        rj = ((rj % pn2) + pn2) % pn2;
        idx += (long long)rj * st2;
      }
    }
    float val = 0.0f;
    if (ok) {
      if (one_slot)  // the synchronous sub-step: t+1 only
        val = w2 * h[((long long)s_p1 * nv + vv) * K + idx];
      else
        val = w0 * h[((long long)s_m1 * nv + vv) * K + idx] +
              w1 * h[((long long)s_0 * nv + vv) * K + idx] +
              w2 * h[((long long)s_p1 * nv + vv) * K + idx];
    }
    sv[vv][pj][pi] = val;
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int xi = X0 + tx, xj = Y0 + ty;
  const int xa = J.side[f] ? pick(c.n, a) - 1 : 0;
  // node coordinates: xa on the face axis, xi on t1, xj on t2 (0 in 2D)
  const int Xn[3] = {a == 0 ? xa : (t1 == 0 ? xi : xj), a == 1 ? xa : (t1 == 1 ? xi : xj),
                     a == 2 ? xa : (L::D == 3 ? (t1 == 2 ? xi : xj) : 0)};
  bool live = xi < pick(c.n, t1) && (L::D == 2 || xj < pick(c.n, t2));
  // each boundary node is written by the first face (lowest axis) holding it
#pragma unroll
  for (int b = 0; b < 3; ++b)
    if (b < a && J.boxed[b] && (Xn[b] == 0 || Xn[b] == c.n[b] - 1)) live = false;
  // eq. spaceInt weights: -1/16 on the outer, 9/16 on the inner points
  auto sw = [](int k) { return (k == 0 || k == 3) ? -1.0f / 16.0f : 9.0f / 16.0f; };
  const bool oi = xi & 1, oj = (L::D == 3) && (xj & 1);
  const int ni = oi ? 4 : 1, nj = oj ? 4 : 1;
  // window index of the stencil's first point along each tangent axis
  const int bi = (oi ? (xi - 3) / 2 : xi / 2) - p0i;
  const int bj = (L::D == 3) ? ((oj ? (xj - 3) / 2 : xj / 2) - p0j) : 0;
  auto interp = [&](int j) {
    float acc = 0.0f;
    for (int sj = 0; sj < nj; ++sj)
      for (int si = 0; si < ni; ++si) {
        const float w = (oi ? sw(si) : 1.0f) * (oj ? sw(sj) : 1.0f);
        acc += w * sv[j][bj + sj][bi + si];
      }
    return acc;
  };
  // value j of this node: from the shared split (G > 1) or interpolated here
  float own[SPLIT ? 1 : T::NV];
  if constexpr (SPLIT) {
    if (live)
      for (int j = tz; j < T::NV; j += T::G) res[j][ty][tx] = interp(j);
    __syncthreads();
  } else {
    if (live)
#pragma unroll
      for (int j = 0; j < T::NV; ++j) own[j] = interp(j);
  }
  if (!live) return;
  auto val = [&](int j) {
    if constexpr (SPLIT)
      return res[j][ty][tx];
    else
      return own[j];
  };
  inject_rebuild<L, S, T::G>(c, run, Xn[0], Xn[1], Xn[2], par, resc, ref, tz, val, xf,
                             (xf != nullptr && a == 0) ? J.side[f] : -1);
}

// 3D rebuild with the tensor-product stencil of eq. spaceInt applied one
// axis at a time: the block stages the temporally interpolated parent window
// (TI / 2 + 3 by TJ / 2 + 3 parent nodes: exactly what the tile's stencils
// reach), interpolates it along t1 for every window row into shared memory
// (every thread the same four taps, even child positions weighting their
// co-located parent node by one), then each node interpolates along t2 (a
// warp holds one child row, so one or four taps uniformly) and rebuilds.
#ifndef INJ_SEP_UNROLL
#define INJ_SEP_UNROLL 4
#endif
template <class L>
struct InjSep {
  static constexpr int TI = InjTile<L>::TI, TJ = InjTile<L>::TJ;
  static constexpr int WI = TI / 2 + 3, WJ = TJ / 2 + 3;
  static constexpr int NV = 4 + L::Q;
  static constexpr int NT = TI * TJ;
  static constexpr int UNR = INJ_SEP_UNROLL;  // staging loop unroll
};

template <class L, class S>
__global__ void __launch_bounds__(InjSep<L>::NT)
    k_inject_sep(LevelView c, const __grid_constant__ InjDesc J,
                 const __grid_constant__ RingDesc R, float w0, float w1, float w2, int s_m1,
                 int s_0, int s_p1, float resc, int par, RefF ref, S* xf) {
  static_assert(L::D == 3, "k_inject_sep is the 3D rebuild");
  using T = InjSep<L>;
  __shared__ float sv[T::NV][T::WJ][T::WI];  // parent window, interpolated in time
  __shared__ float ta[T::NV][T::WJ][T::TI];  // ... and along t1
  const int run = blockIdx.y;
  int f = 0;
  while (f + 1 < J.nf && (long long)blockIdx.x >= J.tstart[f + 1]) ++f;
  const int tile = (int)(blockIdx.x - J.tstart[f]);
  const int a = J.axis[f], t1 = J.t1[f], t2 = J.t2[f];
  const int X0 = (tile % J.ntile1[f]) * T::TI;
  const int Y0 = (tile / J.ntile1[f]) * T::TJ;
  const int p0i = (X0 >> 1) - 1, p0j = (Y0 >> 1) - 1;  // window origin (parent)
  auto pick = [](const int (&v)[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); };
  const long long ext0 = R.ext[f][0], ext01 = ext0 * R.ext[f][1];
  const long long st1 = t1 == 0 ? 1 : (t1 == 1 ? ext0 : ext01);
  const long long st2 = t2 == 0 ? 1 : (t2 == 1 ? ext0 : ext01);
  const int bx1 = pick(R.boxed, t1), bx2 = pick(R.boxed, t2);
  const int e1 = pick(R.ext[f], t1), e2 = pick(R.ext[f], t2);
  const int pn1 = pick(R.pn, t1), pn2 = pick(R.pn, t2);
  const float* h = R.hist + (long long)run * 3 * R.nv * R.K;
  const long long K = R.K, nv = R.nv;
  const bool one_slot = w0 == 0.0f && w1 == 0.0f;  // uniform over the grid
  const int tid = threadIdx.y * T::TI + threadIdx.x;
  // stage (eq. TempInt)
#pragma unroll(T::UNR)
  for (int e = tid; e < T::NV * T::WJ * T::WI; e += T::NT) {
    const int pi = e % T::WI, pj = (e / T::WI) % T::WJ, vv = e / (T::WI * T::WJ);
    int ri = p0i + pi, rj = p0j + pj;
    bool ok = true;
    long long idx = R.start[f];
    if (bx1) {
      ok = ok && ri >= -1 && ri <= e1 - 2;
      idx += (long long)(ri + 1) * st1;
    } else {
      ri = ((ri % pn1) + pn1) % pn1;
      idx += (long long)ri * st1;
    }
    if (bx2) {
      ok = ok && rj >= -1 && rj <= e2 - 2;
      idx += (long long)(rj + 1) * st2;
    } else {
      rj = ((rj % pn2) + pn2) % pn2;
      idx += (long long)rj * st2;
    }
    float val = 0.0f;
    if (ok) {
      if (one_slot)  // the synchronous sub-step: t+1 only
        val = w2 * h[((long long)s_p1 * nv + vv) * K + idx];
      else
        val = w0 * h[((long long)s_m1 * nv + vv) * K + idx] +
              w1 * h[((long long)s_0 * nv + vv) * K + idx] +
              w2 * h[((long long)s_p1 * nv + vv) * K + idx];
    }
    sv[vv][pj][pi] = val;
  }
  __syncthreads();
  // along t1 (eq. spaceInt weights -1/16, 9/16, 9/16, -1/16 at odd child
  // positions; weight 1 on the co-located parent node at even ones)
  {
    const int tx = threadIdx.x;  // the child position along t1 is X0 + tx
    const bool odd = tx & 1;
    const int b = odd ? (tx - 1) >> 1 : tx >> 1;  // first tap in the window
    const float wa = odd ? -1.0f / 16.0f : 0.0f, wb = odd ? 9.0f / 16.0f : 1.0f;
    const float wc = odd ? 9.0f / 16.0f : 0.0f, wd = odd ? -1.0f / 16.0f : 0.0f;
    for (int r = threadIdx.y; r < T::NV * T::WJ; r += T::TJ) {
      const float* row = &sv[0][0][0] + r * T::WI + b;
      ta[0][0][r * T::TI + tx] = wa * row[0] + wb * row[1] + wc * row[2] + wd * row[3];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int xi = X0 + tx, xj = Y0 + ty;
  const int xa = J.side[f] ? pick(c.n, a) - 1 : 0;
  auto co = [&](int k) { return k == a ? xa : (k == t1 ? xi : xj); };
  const int Xn0 = co(0), Xn1 = co(1), Xn2 = co(2);
  bool live = xi < pick(c.n, t1) && xj < pick(c.n, t2);
  // each boundary node is written by the first face (lowest axis) holding it
  if (a > 0 && J.boxed[0] && (Xn0 == 0 || Xn0 == c.n[0] - 1)) live = false;
  if (a > 1 && J.boxed[1] && (Xn1 == 0 || Xn1 == c.n[1] - 1)) live = false;
  if (!live) return;
  // along t2: one tap (even xj) or four (odd xj), uniform over the warp
  float own[T::NV];
  if (ty & 1) {
    const int b = (ty - 1) >> 1;
#pragma unroll
    for (int j = 0; j < T::NV; ++j)
      own[j] = -1.0f / 16.0f * ta[j][b][tx] + 9.0f / 16.0f * ta[j][b + 1][tx] +
               9.0f / 16.0f * ta[j][b + 2][tx] - 1.0f / 16.0f * ta[j][b + 3][tx];
  } else {
    const int b = (ty >> 1) + 1;
#pragma unroll
    for (int j = 0; j < T::NV; ++j) own[j] = ta[j][b][tx];
  }
  inject_rebuild<L, S, 1>(c, run, Xn0, Xn1, Xn2, par, resc, ref, 0,
                          [&](int j) { return own[j]; }, xf,
                          (xf != nullptr && a == 0) ? J.side[f] : -1);
}

// Strain rate S = (grad u + grad u^T) / 2 by second-order central
// differences (hybrid collision, eq. a1ij_HRR), from the velocity deviations
// of the two neighbours along each axis:
// up[a][b] = du_b(x + e_a), um[a][b] = du_b(x - e_a).
template <class L>
__device__ __forceinline__ void strain_from(const float (&up)[3][3], const float (&um)[3][3],
                                            float (&S)[6]) {
  float gr[3][3];  // gr[a][b] = d_a u_b
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) gr[a][b] = (a < L::D) ? 0.5f * (up[a][b] - um[a][b]) : 0.0f;
  S[0] = gr[0][0];
  S[1] = gr[1][1];
  S[2] = gr[2][2];
  S[3] = 0.5f * (gr[0][1] + gr[1][0]);
  S[4] = 0.5f * (gr[0][2] + gr[2][0]);
  S[5] = 0.5f * (gr[1][2] + gr[2][1]);
}

// ----------------------------------------------------------- K4: restrict
// Face-tiled restriction.  The filter of
// eq. filterFneq is a tensor product of (1/4, 1/2, 1/4) along each axis, so
// a block that owns TI x TJ TN nodes of one face first forms, for every
// child node column of the tile's footprint (2 TI + 1 by 2 TJ + 1 columns
// along the face's tangent axes t1, t2), the normal-axis sum of the three
// children's weighted f^(1) -- each child node's f^(1) once per tile instead
// of once per TN node that uses it -- keeps them in shared memory, filters
// along t1 and t2 there, and rebuilds and stores the TN nodes with G threads
// per node (each for every G-th direction), t1-consecutive nodes on
// consecutive threads.  In the first step three consecutive lanes take the
// three children of one column (ten columns per warp), so that on faces
// normal to x one warp load fetches three neighbouring values per row
// instead of one, and the column's sum is formed by two warp shuffles in a
// fixed order.
// HRR (hybrid collision): the tile also keeps the velocity deviations of
// its children -- the centre node of every column and the two normal-axis
// neighbours of every TN column -- so that S^f at the co-located child node
// comes from central differences over its six axis neighbours; one thread
// per TN node then collides the rebuilt node with S = 2 S^f (eq. PijResc),
// stores its post-collision state for the parent's update of parity ppar
// (which skips TN nodes) and writes its velocity deviation to the parent's
// velocity planes pdu.
#ifndef RST_TJ_3D
#define RST_TJ_3D 4
#endif
#ifndef RST_NW_3D
#define RST_NW_3D (2 * RST_TJ_3D + 1)
#endif
#ifndef RST_MINB_3D
#define RST_MINB_3D (27 / RST_NW_3D)
#endif
template <class L>
struct RstTile {
  static constexpr int TI = (L::D == 3) ? 14 : 29;      // TN nodes along t1
  static constexpr int TJ = (L::D == 3) ? RST_TJ_3D : 1;  // ... along t2
  static constexpr int FI = 2 * TI + 1;                 // footprint columns along t1
  static constexpr int FJ = (L::D == 3) ? 2 * TJ + 1 : 1;
  static constexpr int NCH = (FI + 9) / 10;             // ten-column chunks per footprint row
  static constexpr int NW = (L::D == 3) ? RST_NW_3D : 3;  // warps
  static constexpr int NT = 32 * NW;
  static constexpr int NN = TI * TJ;                    // TN nodes per tile
  static constexpr int G = NT / NN;                     // threads per TN node in the rebuild
  static constexpr int MINB = (L::D == 3) ? RST_MINB_3D : 8;  // resident blocks per SM
  static constexpr int MINB_HRR = (L::D == 3) ? 2 : 6;         // ... with the collision
};

template <class L, class S, bool HRR, bool MOV>
__global__ void __launch_bounds__(RstTile<L>::NT, HRR ? RstTile<L>::MINB_HRR : RstTile<L>::MINB)
    k_restrict_tile(LevelView p, LevelView c, const __grid_constant__ TnDesc T,
                    const __grid_constant__ RstDesc J, float resc, int ppar, int cpar,
                    RefF ref, float* pdu, float omega_p, float sig, float ks_p) {
  using TT = RstTile<L>;
  constexpr int Q = L::Q, TI = TT::TI, TJ = TT::TJ, FI = TT::FI, FJ = TT::FJ;
  __shared__ float A[Q][FJ][FI];    // normal-filtered f^(1) per footprint column
  __shared__ float Cf[Q][TJ][TI];   // fully filtered f^(1) per TN node
  __shared__ float cm[TJ][TI][4];   // (drho, du) of the co-located child node
  // HRR: du of every column's centre node, and of the normal neighbours
  // (d = -1, +1) of every TN column
  __shared__ float cu0[HRR ? 3 : 1][HRR ? FJ : 1][HRR ? FI : 1];
  __shared__ float cun[HRR ? 2 : 1][HRR ? 3 : 1][HRR ? TJ : 1][HRR ? TI : 1];
  const int run = blockIdx.y;
  int f = 0;
  while (f + 1 < T.nf && (long long)blockIdx.x >= J.tstart[f + 1]) ++f;
  const int tile = (int)(blockIdx.x - J.tstart[f]);
  const int a = T.axis[f], t1 = J.t1[f], t2 = J.t2[f];
  // per-face values picked by axis without indexing local arrays
  auto pick = [](const int (&v)[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); };
  const int ti = tile % J.ntile1[f], tj = tile / J.ntile1[f];
  const int r1 = pick(T.rlo[f], t1) + ti * TI;  // first TN coordinate of the tile along t1, t2
  const int r2 = pick(T.rlo[f], t2) + tj * TJ;
  const int n1 = min(TI, pick(T.rlo[f], t1) + pick(T.rext[f], t1) - r1);
  const int n2 = min(TJ, pick(T.rlo[f], t2) + pick(T.rext[f], t2) - r2);
  const int ra = pick(T.rlo[f], a);
  // 1. normal-axis sums of the footprint columns
  {
    const int lane = threadIdx.x, col = lane / 3, d = lane - 3 * col - 1;
    const float w = d == 0 ? 0.5f : 0.25f;
    int xa = 2 * ra + d;
    if (pick(c.per, a)) xa = wrapi(xa, pick(c.n, a));
    const S* fcb = run_cptr<S>(c, run);
    for (int ch = threadIdx.y; ch < FJ * TT::NCH; ch += TT::NW) {
      const int v = ch / TT::NCH, u = (ch % TT::NCH) * 10 + col;
      const bool ok = col < 10 && u <= 2 * n1 && v <= ((L::D == 3) ? 2 * n2 : 0);
      float f1[Q], drho = 0.0f, dux = 0.0f, duy = 0.0f, duz = 0.0f;
      if (ok) {
        int x1 = 2 * r1 - 1 + u, x2 = (L::D == 3) ? 2 * r2 - 1 + v : 0;
        if (pick(c.per, t1)) x1 = wrapi(x1, pick(c.n, t1));
        if (L::D == 3 && pick(c.per, t2)) x2 = wrapi(x2, pick(c.n, t2));
        auto co = [&](int b) { return b == a ? xa : (b == t1 ? x1 : x2); };
        float g[Q];
        load_pre<L, S>(fcb, c.plane, node_addr<L>(c, co(0), co(1), co(2)), cpar, c.es, g);
        split_neq<L>(g, ref, drho, dux, duy, duz, f1);
#pragma unroll
        for (int i = 0; i < Q; ++i) f1[i] *= w;
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) f1[i] = 0.0f;
      }
      // lane 3 col gets (d = -1) + (d = 0) + (d = +1) of its column
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float s0 = __shfl_down_sync(0xffffffffu, f1[i], 1);
        const float s1 = __shfl_down_sync(0xffffffffu, f1[i], 2);
        if (ok && d == -1) A[i][v][u] = (f1[i] + s0) + s1;
      }
      const bool tn_col = (u & 1) && (L::D == 2 || (v & 1));
      if (ok && d == 0 && tn_col) {
        const int j = (L::D == 3) ? (v - 1) >> 1 : 0, i = (u - 1) >> 1;
        cm[j][i][0] = drho;
        cm[j][i][1] = dux;
        cm[j][i][2] = duy;
        cm[j][i][3] = duz;
      }
      if constexpr (HRR) {
        if (ok && d == 0) {
          cu0[0][v][u] = dux;
          cu0[1][v][u] = duy;
          cu0[2][v][u] = duz;
        }
        if (ok && d != 0 && tn_col) {
          const int j = (L::D == 3) ? (v - 1) >> 1 : 0, i = (u - 1) >> 1, k = d > 0;
          cun[k][0][j][i] = dux;
          cun[k][1][j][i] = duy;
          cun[k][2][j][i] = duz;
        }
      }
    }
  }
  __syncthreads();
  // 2. filter along t1 and t2: TN node (i, j) sits at footprint column
  // (2 i + 1, 2 j + 1)
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int e = tid; e < Q * TI * TJ; e += TT::NT) {
    const int i = e % TI, j = (e / TI) % TJ, q = e / (TI * TJ);
    if (i >= n1 || j >= n2) continue;
    float s;
    if constexpr (L::D == 3) {
      s = 0.0f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float* row = &A[q][2 * j + b][2 * i];
        const float rs = 0.25f * row[0] + 0.5f * row[1] + 0.25f * row[2];
        s += (b == 1 ? 0.5f : 0.25f) * rs;
      }
    } else {
      const float* row = &A[q][0][2 * i];
      s = 0.25f * row[0] + 0.5f * row[1] + 0.25f * row[2];
    }
    Cf[q][j][i] = s;
  }
  __syncthreads();
  // 3. rebuild f = f0(rho, u) + resc f^(1) (eq. rescfc) and store for the
  // parent's update of parity ppar
  const int node = tid % TT::NN, grp = tid / TT::NN;
  const int i = node % TI, j = node / TI;
  if (grp >= TT::G || i >= n1 || j >= n2) return;
  // parent coordinates: box-relative + lo on axes the box spans
  auto pc = [&](int b) {
    int r = b == a ? ra : (b == t1 ? r1 + i : ((L::D == 3) ? r2 + j : 0));
    if (pick(T.boxed, b)) {
      r += pick(T.lo, b);
      if (pick(p.per, b)) r = wrapi(r, pick(p.n, b));
    }
    return r;
  };
  if constexpr (HRR) {
    if (grp != 0) return;
    float g[Q];
    equilibrium_f<L>(cm[j][i][0], cm[j][i][1], cm[j][i][2], cm[j][i][3], ref, g);
#pragma unroll
    for (int q = 0; q < Q; ++q) g[q] += resc * Cf[q][j][i];
    // S^f by central differences (child spacing) at the co-located node,
    // whose footprint column is (2 i + 1, 2 j + 1)
    const int u = 2 * i + 1, v = (L::D == 3) ? 2 * j + 1 : 0;
    float up[3][3] = {}, um[3][3] = {};
#pragma unroll
    for (int ax = 0; ax < L::D; ++ax)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (ax == a) {
          up[ax][b] = cun[1][b][j][i];
          um[ax][b] = cun[0][b][j][i];
        } else if (ax == t1) {
          up[ax][b] = cu0[b][v][u + 1];
          um[ax][b] = cu0[b][v][u - 1];
        } else if constexpr (L::D == 3) {
          up[ax][b] = cu0[b][v + 1][u];
          um[ax][b] = cu0[b][v - 1][u];
        }
      }
    HrrIn hy;
    hy.sig = sig;
    hy.ks = ks_p;
    strain_from<L>(up, um, hy.s);
#pragma unroll
    for (int k = 0; k < 6; ++k) hy.s[k] *= 2.0f;  // eq. PijResc
    S* fp = run_ptr<S>(p, run);
    const NodeAddr ad = node_addr<L>(p, pc(0), pc(1), pc(2));
    const int es = p.es;
    collide_emit<L, 3, MOV>(
        g, omega_p, ref,
        [&](auto I, float val) {
          constexpr int q = decltype(I)::value;
          if (ppar == 0)
            Store<S>::st(fp + (long long)opp<L>(q) * p.plane + es * ad.at(0, 0, 0), val);
          else
            Store<S>::st(fp + (long long)q * p.plane +
                             es * ad.at(L::c(q, 0), L::c(q, 1), L::c(q, 2)),
                         val);
        },
        &hy);
    float* dp = pdu + (long long)run * L::D * p.plane + ad.at(0, 0, 0);
    for (int b = 0; b < L::D; ++b) dp[(long long)b * p.plane] = cm[j][i][1 + b];
    return;
  }
  const float drho = cm[j][i][0], dux = cm[j][i][1], duy = cm[j][i][2];
  const float duz = (L::D == 3) ? cm[j][i][3] : 0.0f;
  const float Ux = ref.Ux, Uy = ref.Uy, Uz = (L::D == 3) ? ref.Uz : 0.0f;
  const float ux = Ux + dux, uy = Uy + duy, uz = Uz + duz;
  float Ac[7], dA[7];
  third_coeffs(ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, Ac, dA);
  const float dusq = 1.5f * (dux * (ux + Ux) + duy * (uy + Uy) + duz * (uz + Uz));
  const float rho = ref.rho0 + drho;
  S* fp = run_ptr<S>(p, run);
  const NodeAddr ad = node_addr<L>(p, pc(0), pc(1), pc(2));
  sfor<Q>([&](auto I) {
    constexpr int q = decltype(I)::value;
    if (q % TT::G == grp) {
      const float g = eq_i<L, q, true>(drho, rho, dux, duy, duz, dusq, dA, ref) +
                      resc * Cf[q][j][i];
      store_pre_i<L, S, q>(fp, p.plane, ad, ppar, p.es, g);
    }
  });
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
// update (post-collision g_i at plane opp(i) of the node), in FP64 up to the
// final rounding to the storage type.
template <class L, class S>
// Nodes t0 .. t0 + cnt - 1 of the level (x fastest), from rho[t - t0] and
// u[a * us + t - t0] (a chunk of the fields; us: the chunk's component
// stride).  The deviations from the reference state are formed in FP64 and
// the equilibrium deviation in binary32, in the same deviation form as the
// level update's collision (FP64 arithmetic is a small fraction of binary32
// on this GPU; the stored populations are binary32 or binary16 either way).
__global__ void k_init(LevelView v, int run, const double* rho, const double* u, long long us,
                       long long t0, long long cnt, RefState ref, RefF R) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  const long long t = t0 + k;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  float g0[L::Q];
  equilibrium_f<L>((float)(rho[k] - ref.rho0), (float)(u[k] - ref.U[0]),
                   (float)(u[us + k] - ref.U[1]), (float)(u[2 * us + k] - ref.U[2]), R, g0);
  S* f = run_ptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Store<S>::st(f + (long long)opp<L>(i) * v.plane + v.es * a.at(0, 0, 0), g0[i]);
  });
}

// Moments of one node's binary32 populations for the read-out and the
// diagnostics, as accurate as FP64 sums of the same values but formed with
// binary32 instructions (GB300 executes FP64 at a small fraction of its
// binary32 rate): each sum is accumulated in binary32 with the rounding
// error of every addition recovered exactly by Knuth's TwoSum and summed
// alongside (the cascaded summation Sum2 of Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005); the pair is added in
// FP64 at the end.  The result differs from the exact sum by at most
// gamma_{n-1}^2 sum |g_i| (gamma_k = k u / (1 - k u), u = 2^-24, n <= 28
// terms: below 1e-12 of sum |g_i|), plus the final FP64 rounding.
struct Acc2 {
  float s = 0.0f, e = 0.0f;
  __device__ __forceinline__ void add(float b) {
    const float x = s + b;  // TwoSum(s, b): x + err == s + b exactly
    const float z = x - s;
    e += (s - (x - z)) + (b - z);
    s = x;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

// drho = sum g and j = sum xi g (shifted populations), each through Acc2.
template <class L>
__device__ __forceinline__ void moments_acc(const float (&g)[L::Q], double& drho, double& jx,
                                            double& jy, double& jz) {
  Acc2 r, m[3];
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    r.add(g[i]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (L::c(i, a) == 1) m[a].add(g[i]);
      if (L::c(i, a) == -1) m[a].add(-g[i]);
    }
  });
  drho = r.value();
  jx = m[0].value();
  jy = m[1].value();
  jz = m[2].value();
}

// FP64 partials of the noise diagnostic: max |drho_a - drho_b| and the sum
// of squares over level-0 nodes outside the child box by at least
// `margin` cells (on every bounded axis the node lies outside the box
// grown by margin), plus the node count.
template <class L, class S>
__global__ void __launch_bounds__(kDiagThreads)
    k_noise_partial(LevelView va, int last_a, RefState ra, LevelView vb, int last_b,
                    RefState rb, int run, NoiseRegion reg, double* partial) {
  __shared__ double sh[3][kDiagThreads];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0, ss = 0.0, cnt = 0.0;
  int x, y, z;
  if (node_of(va, t, x, y, z)) {
    const int P[3] = {x, y, z};
    bool near = true;
    for (int a = 0; a < 3; ++a) {
      if (!reg.boxed[a]) continue;
      int rel = P[a] - reg.lo[a];
      rel = ((rel % reg.n[a]) + reg.n[a]) % reg.n[a];
      const bool in_grown = rel <= reg.E[a] + reg.margin || rel >= reg.n[a] - reg.margin;
      near = near && in_grown;
    }
    if (!near) {
      float ga[L::Q], gb[L::Q];
      const S* fa = run_cptr<S>(va, run);
      const S* fb = run_cptr<S>(vb, run);
      load_post<L, S>(fa, va.plane, node_addr<L>(va, x, y, z), last_a, va.es, ga);
      load_post<L, S>(fb, vb.plane, node_addr<L>(vb, x, y, z), last_b, vb.es, gb);
      Acc2 sa, sb;  // (drho of both states to FP64 accuracy)
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        sa.add(ga[i]);
        sb.add(gb[i]);
      }
      const double da = sa.value(), db = sb.value();
      const double d = fabs((ra.rho0 + da) - (rb.rho0 + db));
      mx = d;
      ss = d * d;
      cnt = 1.0;
    }
  }
  sh[0][threadIdx.x] = mx;
  sh[1][threadIdx.x] = ss;
  sh[2][threadIdx.x] = cnt;
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + w]);
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) partial[(long long)j * gridDim.x + blockIdx.x] = sh[j][0];
}

// rho and u (FP64 or FP32 outputs) of the post-collision state; NaN at
// inactive nodes.
template <class L, class S, class T>
// (nodes t0 .. t0 + cnt - 1 into rho[t - t0], u[a * us + t - t0])
__global__ void k_macros(LevelView v, int run, int last, T* rho, T* u, long long us,
                         long long t0, long long cnt, RefState ref) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  const long long t = t0 + k;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  if (inactive(v, x, y, z)) {
    const T nan = T(__longlong_as_double(0x7ff8000000000000ULL));
    rho[k] = nan;
    u[k] = u[us + k] = u[2 * us + k] = nan;
    return;
  }
  const S* f = run_cptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_post<L, S>(f, v.plane, a, last, v.es, g);
  // moments to FP64 accuracy (moments_acc): rho u = sum xi g + rho0 U
  double drho, jx, jy, jz;
  moments_acc<L>(g, drho, jx, jy, jz);
  const double r = ref.rho0 + drho, ri = 1.0 / r;
  rho[k] = T(r);
  u[k] = T((jx + ref.rho0 * ref.U[0]) * ri);
  u[us + k] = T((jy + ref.rho0 * ref.U[1]) * ri);
  u[2 * us + k] = T(L::D == 3 ? (jz + ref.rho0 * ref.U[2]) * ri : 0.0);
}

// Post-collision populations shifted by the rest state, f_i - w_i rho0,
// [q][N] FP64 (the stored deviations plus f0_i(rho0, U) - w_i rho0).
template <class L, class S>
__global__ void k_populations(LevelView v, int run, int last, double* out, RefState ref) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  const S* f = run_cptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_post<L, S>(f, v.plane, a, last, v.es, g);
  double base[L::Q];
  equilibrium_dev<L, double>(0.0, ref.U[0], ref.U[1], ref.U[2], ref.rho0, 0.0, 0.0, 0.0, base);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) out[(long long)i * N + t] = (double)g[i] + base[i];
}

// FP64 per-block partial sums of (drho, rho u) over active nodes; a fixed
// shared-memory tree order makes the result deterministic.
template <class L, class S>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(LevelView v, int run, int last,
                                                               double* partial, RefState ref) {
  __shared__ double sh[4][kDiagThreads];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s[4] = {0, 0, 0, 0};
  int x, y, z;
  if (node_of(v, t, x, y, z) && !inactive(v, x, y, z)) {
    const S* f = run_cptr<S>(v, run);
    const NodeAddr a = node_addr<L>(v, x, y, z);
    float g[L::Q];
    load_post<L, S>(f, v.plane, a, last, v.es, g);
    moments_acc<L>(g, s[0], s[1], s[2], s[3]);
    for (int a = 0; a < 3; ++a) s[1 + a] += ref.rho0 * ref.U[a];
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
                        unsigned long long* counter, RefState ref) {
  __shared__ unsigned long long slot;
  if (threadIdx.x == 0) slot = *counter;
  __syncthreads();
  const long long base = (long long)(slot % (unsigned long long)cap) * v.batch * n;
  for (int t = threadIdx.x; t < n * v.batch; t += blockDim.x) {
    const int run = t / n, k = t - run * n;
    const S* f = run_cptr<S>(v, run);
    const NodeAddr a = node_addr<L>(v, ijk[3 * k], ijk[3 * k + 1], ijk[3 * k + 2]);
    float g[L::Q];
    load_post<L, S>(f, v.plane, a, last, v.es, g);
    double gd[L::Q], drho, jx, jy, jz;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) gd[i] = (double)g[i];
    moments<L, double>(gd, drho, jx, jy, jz);
    const double r = ref.rho0 + drho;
    double* o = rec + (base + (long long)run * n + k) * 4;
    o[0] = r;
    o[1] = (jx + ref.rho0 * ref.U[0]) / r;
    o[2] = (jy + ref.rho0 * ref.U[1]) / r;
    o[3] = (L::D == 3) ? (jz + ref.rho0 * ref.U[2]) / r : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = slot + 1;
}

}  // namespace mlbm
