// Persistent fused step: one cooperative launch advances a run (or a batch
// of runs) by n coarse steps.  The host scheduler records, once, the phases
// of six consecutive coarse steps (the schedule repeats with period six:
// parities and history slots) as a program; the kernel walks the program
// for each coarse step, every block taking a grid-stride share of each
// phase's items, and separates dependent phases by a grid barrier.  For
// small runs, where a level update or an interface rebuild is a few
// microseconds of work, this removes the per-kernel launch and drain cost of
// the 7 (two levels) to 19 (three levels) launches of each coarse step.
//
// The phases compute what the per-phase kernels compute, one item per
// thread and without shared-memory staging (their launch shapes do not fit
// one persistent block shape):
//   update       one node: streaming and collision (eq. LBMequation);
//   capture      one history-ring entry (capture_item);
//   rebuild      one TF / IE node: temporal (eq. TempInt) and spatial
//                (eq. spaceInt) interpolation straight from the history,
//                then eq. rescff (inject_rebuild);
//   restriction  one TN node: the 3^D filtered f^(1) of eq. filterFneq in a
//                fixed order, then eq. rescfc;
//   probe        block 0: the probe record of k_probe.
// Plain, regularized and recursive regularized collisions (not the hybrid
// one, whose extra passes stay on the per-phase kernels).
//
// Phases recorded with nobar (the scheduler's side-stream pairs: a
// restriction and the child's second rebuild; a parent update and the
// child's next phase; the probe and the next step's capture) run without a
// barrier between them.  The tables and the programs are read into shared
// memory once per launch.
//
// Grid barrier: arrival counter and generation word in device memory; the
// last block to arrive resets the counter and advances the generation, the
// others wait for the generation to change.  Every wait is bounded (spin
// limit); a wait that runs out sets the error word, every block then leaves
// the program, and the host reads the error word (mapped host memory)
// after the launch.  The launch is cooperative, so all blocks are resident.
// A run small enough for one thread-block cluster (at most 16 blocks, a few
// items per thread) is launched as one cluster instead and takes the
// cluster's hardware barrier (cluster_barrier), a fraction of the cost of
// the global one.
#pragma once
#include "kernels.cuh"

namespace mlbm {

constexpr int kFusedThreads = 256;
#ifndef FUSED_MINB
#define FUSED_MINB 1  // resident blocks per SM the fused kernel is compiled for
#endif

// Descriptors the phases read, per level (ring / bnd / tn of level l describe
// its interface with level l - 1).
struct FusedTables {
  LevelView v[kFusedLevels];
  RingDesc ring[kFusedLevels];
  BndDesc bnd[kFusedLevels];
  TnDesc tn[kFusedLevels];
  RefF ref;
  RefState refd;
  int coll;
  int probe_n, probe_cap;
  const int* probe_ijk;
  double* probe_rec;
  unsigned long long* probe_counter;
};

// Returns false once any block has given up waiting.
__device__ __forceinline__ bool fused_barrier(const FusedArgs& A) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = A.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned expected = gridDim.x + (unsigned)A.expect_extra;
    const unsigned arrived = atomicAdd(A.bar, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(A.bar, 0u);
      __threadfence();
      atomicAdd(A.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (*(volatile int*)A.err != 0) break;
        if (++spins > A.spin_limit) {
          atomicExch(A.err, 1);
          break;
        }
        if (spins > 256) __nanosleep(64);  // poll tightly first: phases are short
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)A.err == 0;
}

// The barrier of a grid that is one thread-block cluster: the cluster's
// hardware barrier, with release / acquire ordering at cluster scope (the
// blocks' global-memory writes before it are visible to every block after
// it).  Every block takes every barrier of the program (the phase loop is
// the same for all blocks and none leaves it early), so it cannot wait on
// a block that never arrives; the bounded software barrier serves the
// timeout test.
__device__ __forceinline__ bool cluster_barrier() {
  __threadfence();
  __syncthreads();
  asm volatile(
      "barrier.cluster.arrive.release;\n\t"
      "barrier.cluster.wait.acquire;" ::
          : "memory");
  return true;
}

// Level update of node item t (run-major over the level's nodes).
template <class L, class S>
__device__ __forceinline__ void fused_update(const LevelView& v, int coll, int par, float omega,
                                             const RefF& R, long long t) {
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  const int run = (int)(t / N);
  long long r = t - run * N;
  const int x = (int)(r % v.n[0]);
  r /= v.n[0];
  const int y = (int)(r % v.n[1]);
  const int z = (int)(r / v.n[1]);
  if (inactive(v, x, y, z)) return;
  S* f = run_ptr<S>(v, run);
  const NodeAddr a = node_addr<L>(v, x, y, z);
  float g[L::Q];
  load_pre<L, S>(f, v.plane, a, par, v.es, g);
  auto emit = [&](auto I, float val) {
    constexpr int i = decltype(I)::value;
    if (par == 0)
      Store<S>::st(f + (long long)opp<L>(i) * v.plane + v.es * a.at(0, 0, 0), val);
    else
      Store<S>::st(f + (long long)i * v.plane + v.es * a.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)),
                   val);
  };
  if (coll == 0)
    collide_emit<L, 0, true>(g, omega, R, emit);
  else if (coll == 1)
    collide_emit<L, 1, true>(g, omega, R, emit);
  else
    collide_emit<L, 2, true>(g, omega, R, emit);
}

// Rebuild of boundary node item t of child level c (run-major over the
// boundary nodes): the same taps and weights as k_inject, read straight
// from the history ring.
template <class L, class S>
__device__ __forceinline__ void fused_inject(const LevelView& c, const BndDesc& B,
                                             const RingDesc& R, const Phase& ph, const RefF& ref,
                                             long long t) {
  constexpr int NV = 4 + L::Q;
  const int run = (int)(t / B.count);
  const long long k = t - (long long)run * B.count;
  const int f = ring_face(B.start, B.nf, k);
  long long loc = k - B.start[f];
  const int e0 = B.ext[f][0], e1x = B.ext[f][1];
  const int X0 = B.lo[f][0] + (int)(loc % e0);
  loc /= e0;
  const int X1 = B.lo[f][1] + (int)(loc % e1x);
  loc /= e1x;
  const int X2 = B.lo[f][2] + (int)loc;
  const int a = B.axis[f];
  const int t1 = (L::D == 2) ? 1 - a : (a == 0 ? 1 : 0);
  const int t2 = (L::D == 2) ? 2 : (a == 2 ? 1 : 2);
  auto pick = [](int v0, int v1, int v2, int q) { return q == 0 ? v0 : (q == 1 ? v1 : v2); };
  const int xi = pick(X0, X1, X2, t1), xj = pick(X0, X1, X2, t2);
  const long long ext0 = R.ext[f][0], ext01 = ext0 * R.ext[f][1];
  const long long st1 = t1 == 0 ? 1 : (t1 == 1 ? ext0 : ext01);
  const long long st2 = t2 == 0 ? 1 : (t2 == 1 ? ext0 : ext01);
  const int bx1 = pick(R.boxed[0], R.boxed[1], R.boxed[2], t1);
  const int bx2 = pick(R.boxed[0], R.boxed[1], R.boxed[2], t2);
  const int pn1 = pick(R.pn[0], R.pn[1], R.pn[2], t1), pn2 = pick(R.pn[0], R.pn[1], R.pn[2], t2);
  const float* h = R.hist + (long long)run * 3 * R.nv * R.K;
  const long long K = R.K, nv = R.nv;
  const bool oi = xi & 1, oj = (L::D == 3) && (xj & 1);
  const int ni = oi ? 4 : 1, nj = oj ? 4 : 1;
  const int bi = oi ? (xi - 3) / 2 : xi / 2;
  const int bj = (L::D == 3) ? (oj ? (xj - 3) / 2 : xj / 2) : 0;
  auto sw = [](int q) { return (q == 0 || q == 3) ? -1.0f / 16.0f : 9.0f / 16.0f; };
  const bool one_slot = ph.w[0] == 0.0f && ph.w[1] == 0.0f;
  float val[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) val[j] = 0.0f;
  for (int sj = 0; sj < nj; ++sj) {
    int rj = bj + sj;
    long long base = R.start[f];
    if (L::D == 3) {
      if (bx2) {
        base += (long long)(rj + 1) * st2;
      } else {
        rj = ((rj % pn2) + pn2) % pn2;
        base += (long long)rj * st2;
      }
    }
    for (int si = 0; si < ni; ++si) {
      int ri = bi + si;
      long long idx = base;
      if (bx1) {
        idx += (long long)(ri + 1) * st1;
      } else {
        ri = ((ri % pn1) + pn1) % pn1;
        idx += (long long)ri * st1;
      }
      const float w = (oi ? sw(si) : 1.0f) * (oj ? sw(sj) : 1.0f);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        float hv;
        if (one_slot)
          hv = ph.w[2] * h[((long long)ph.slot[2] * nv + j) * K + idx];
        else
          hv = ph.w[0] * h[((long long)ph.slot[0] * nv + j) * K + idx] +
               ph.w[1] * h[((long long)ph.slot[1] * nv + j) * K + idx] +
               ph.w[2] * h[((long long)ph.slot[2] * nv + j) * K + idx];
        val[j] += w * hv;
      }
    }
  }
  inject_rebuild<L, S, 1>(c, run, X0, X1, X2, ph.par, ph.resc, ref, 0,
                          [&](int j) { return val[j]; }, static_cast<S*>(nullptr), -1);
}

// Restriction of TN node item t (run-major over the TN nodes of the child
// level's interface): the 3^D children in a fixed order.
template <class L, class S>
__device__ __forceinline__ void fused_restrict(const LevelView& p, const LevelView& c,
                                               const TnDesc& T, const Phase& ph, const RefF& ref,
                                               long long t) {
  constexpr int Q = L::Q, NB = (L::D == 3) ? 27 : 9;
  const int run = (int)(t / T.count);
  const long long k = t - (long long)run * T.count;
  const int fc = ring_face(T.start, T.nf, k);
  long long loc = k - T.start[fc];
  int P[3], X[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int e = T.rext[fc][a];
    const int r = T.rlo[fc][a] + (int)(loc % e);
    loc /= e;
    int pc = r;
    if (T.boxed[a]) {
      pc = T.lo[a] + r;
      if (p.per[a]) pc = wrapi(pc, p.n[a]);
    }
    P[a] = pc;
    X[a] = 2 * r;
  }
  const S* fcb = run_cptr<S>(c, run);
  float acc[Q], m4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < Q; ++i) acc[i] = 0.0f;
  for (int kn = 0; kn < NB; ++kn) {
    const int dx = kn % 3 - 1, dy = (kn / 3) % 3 - 1, dz = (L::D == 3) ? kn / 9 - 1 : 0;
    int xx = X[0] + dx, yy = X[1] + dy, zz = X[2] + dz;
    if (c.per[0]) xx = wrapi(xx, c.n[0]);
    if (c.per[1]) yy = wrapi(yy, c.n[1]);
    if (L::D == 3 && c.per[2]) zz = wrapi(zz, c.n[2]);
    float g[Q], f1[Q], drho, ux, uy, uz;
    load_pre<L, S>(fcb, c.plane, node_addr<L>(c, xx, yy, zz), ph.cpar, c.es, g);
    split_neq<L>(g, ref, drho, ux, uy, uz, f1);
    const float w = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f) *
                    (L::D == 3 ? (dz == 0 ? 0.5f : 0.25f) : 1.0f);
#pragma unroll
    for (int i = 0; i < Q; ++i) acc[i] += w * f1[i];
    if (dx == 0 && dy == 0 && dz == 0) {
      m4[0] = drho;
      m4[1] = ux;
      m4[2] = uy;
      m4[3] = uz;
    }
  }
  float g[Q];
  equilibrium_f<L>(m4[0], m4[1], m4[2], m4[3], ref, g);
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] += ph.resc * acc[i];
  store_pre<L, S>(run_ptr<S>(p, run), p.plane, node_addr<L>(p, P[0], P[1], P[2]), ph.par, p.es,
                  g);
}

// Probe sampling (block 0 only; the body of k_probe).
template <class L, class S>
__device__ __forceinline__ void fused_probe(const FusedTables& T, const LevelView& v, int last) {
  __shared__ unsigned long long slot;
  if (threadIdx.x == 0) slot = *T.probe_counter;
  __syncthreads();
  const int n = T.probe_n;
  const long long base = (long long)(slot % (unsigned long long)T.probe_cap) * v.batch * n;
  for (int t = threadIdx.x; t < n * v.batch; t += blockDim.x) {
    const int run = t / n, k = t - run * n;
    const S* f = run_cptr<S>(v, run);
    const int* ijk = T.probe_ijk + 3 * k;
    const NodeAddr a = node_addr<L>(v, ijk[0], ijk[1], ijk[2]);
    float g[L::Q];
    load_post<L, S>(f, v.plane, a, last, v.es, g);
    double gd[L::Q], drho, jx, jy, jz;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) gd[i] = (double)g[i];
    moments<L, double>(gd, drho, jx, jy, jz);
    const double r = T.refd.rho0 + drho;
    double* o = T.probe_rec + (base + (long long)run * n + k) * 4;
    o[0] = r;
    o[1] = (jx + T.refd.rho0 * T.refd.U[0]) / r;
    o[2] = (jy + T.refd.rho0 * T.refd.U[1]) / r;
    o[3] = (L::D == 3) ? (jz + T.refd.rho0 * T.refd.U[2]) / r : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *T.probe_counter = slot + 1;
}

template <class L, class S>
__global__ void __launch_bounds__(kFusedThreads, FUSED_MINB) k_fused(const __grid_constant__ FusedArgs A) {
  // the tables and the programs, read once per launch into shared memory
  __shared__ __align__(16) FusedTables T;
  __shared__ __align__(16) Phase prog[kFusedMaxPhases];
  __shared__ int start[7];
  {
    const int4* src = reinterpret_cast<const int4*>(A.tab);
    int4* dst = reinterpret_cast<int4*>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(FusedTables) / 16); i += blockDim.x) dst[i] = src[i];
    const int* srcb = reinterpret_cast<const int*>(A.tab);
    int* dstb = reinterpret_cast<int*>(&T);
    for (int i = (int)(sizeof(FusedTables) / 16) * 4 + threadIdx.x;
         i < (int)(sizeof(FusedTables) / 4); i += blockDim.x)
      dstb[i] = srcb[i];
    if (threadIdx.x < 7) start[threadIdx.x] = A.prog_start[threadIdx.x];
    __syncthreads();
    const int* sp = reinterpret_cast<const int*>(A.prog);
    int* dp = reinterpret_cast<int*>(prog);
    for (int i = threadIdx.x; i < start[6] * (int)(sizeof(Phase) / 4); i += blockDim.x)
      dp[i] = sp[i];
    __syncthreads();
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = true;
  for (int s = 0; s < A.nsteps && ok; ++s) {
    const int key = (A.first_key + s) % 6;
    for (int k = start[key]; k < start[key + 1] && ok; ++k) {
      const Phase& ph = prog[k];
      const int l = ph.level;
      switch (ph.kind) {
        case 0: {
          const LevelView& v = T.v[l];
          const long long n = (long long)v.n[0] * v.n[1] * v.n[2] * v.batch;
          for (long long t = t0; t < n; t += stride)
            fused_update<L, S>(v, T.coll, ph.par, ph.omega, T.ref, t);
          break;
        }
        case 1: {
          const RingDesc& R = T.ring[l + 1];
          const long long n = R.K * T.v[l].batch;
          for (long long t = t0; t < n; t += stride) {
            const int run = (int)(t / R.K);
            capture_item<L, S>(T.v[l], R, ph.par, 0, ph.slot[0], ph.slot[0], T.ref,
                               t - (long long)run * R.K, run);
          }
          break;
        }
        case 2: {
          const BndDesc& B = T.bnd[l];
          const long long n = B.count * T.v[l].batch;
          for (long long t = t0; t < n; t += stride)
            fused_inject<L, S>(T.v[l], B, T.ring[l], ph, T.ref, t);
          break;
        }
        case 3: {
          const TnDesc& Tn = T.tn[l + 1];
          const long long n = Tn.count * T.v[l].batch;
          for (long long t = t0; t < n; t += stride)
            fused_restrict<L, S>(T.v[l], T.v[l + 1], Tn, ph, T.ref, t);
          break;
        }
        default:
          if (blockIdx.x == 0) fused_probe<L, S>(T, T.v[l], ph.par);
          break;
      }
      if (!ph.nobar) ok = A.cluster ? cluster_barrier() : fused_barrier(A);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    __threadfence_system();
    *(volatile int*)A.err_host = *(volatile int*)A.err;
  }
}

}  // namespace mlbm
