// Per-lattice launch table.  Each lattice's kernels are instantiated in its
// own translation unit (ops_d2q9.cu, ops_d3q19.cu, ops_d3q27.cu) so the
// build compiles them in parallel; the host scheduler only sees this table.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "desc.h"

namespace mlbm {

struct Ops {
  int q, d;
  // K1: fused stream + collide of every active node of a level.
  // (bx, by: block shape, bx a multiple of 32, bx * by <= 128; xf: the
  // level's face buffer, or null when the rebuild writes the planes)
  cudaError_t (*stream_collide)(const LevelView& v, int coll, int storage, int par, float omega,
                                const RefState& ref, int bx, int by, const void* xf,
                                cudaStream_t s);
  // K2: history capture (mode 0) or set-up (mode 1).
  cudaError_t (*capture)(const LevelView& p, const RingDesc& R, int storage, int par, int mode,
                         int s_new, int s_also, const RefState& ref, cudaStream_t s);
  // K3: coarse -> fine boundary rebuild (xf: face buffer of the nodes on
  // faces normal to x, or null: every node into the planes).
  cudaError_t (*inject)(const LevelView& c, const BndDesc& B, const RingDesc& R, int storage,
                        const float* wt, const int* slots, float resc, int par, const RefState& ref,
                        void* xf, cudaStream_t s);
  // K4: fine -> coarse restriction.
  cudaError_t (*restrict_tn)(const LevelView& p, const LevelView& c, const TnDesc& T, int storage,
                             float resc, int ppar, int cpar, const RefState& ref, cudaStream_t s);
  // Hybrid collision (H-RR): velocity planes, the level update with
  // finite-difference strain, the parent strain history, the child's outer
  // layer collision and the restriction that collides TN nodes.
  cudaError_t (*velocity)(const LevelView& v, int storage, int par, float* du, const RefState& ref,
                          cudaStream_t s);
  cudaError_t (*stream_collide_hrr)(const LevelView& v, int storage, int par, float omega,
                                    const float* du, float sig, float ks, const RefState& ref,
                                    cudaStream_t s);
  cudaError_t (*parent_strain)(const LevelView& p, const LevelView& c, const RingDesc& R,
                               const TnDesc& T, int storage, float* sh, int s_new, int s_also,
                               int ppar, int cpar, int mode, const RefState& ref, cudaStream_t s);
  cudaError_t (*collide_bnd)(const LevelView& c, const BndDesc& B, const RingDesc& R, int storage,
                             const float* sh, const float* wt, const int* slots, float omega,
                             float sig, float ks, int par, const RefState& ref, cudaStream_t s);
  cudaError_t (*restrict_hrr)(const LevelView& p, const LevelView& c, const TnDesc& T,
                              int storage, float resc, int ppar, int cpar, float* pdu,
                              float omega_p, float sig, float ks_p, const RefState& ref,
                              cudaStream_t s);
  // Non-hydrodynamic mode sensors (after the velocity pass) and their
  // compact read-out.
  cudaError_t (*sensors)(const LevelView& v, int storage, const float* du, int par,
                         const SensorState& st, const RefState& ref, cudaStream_t s);
  cudaError_t (*sensor_read)(const LevelView& v, int run, const SensorState& st,
                             unsigned char* flags, double* div, double* curl, double* gnorm,
                             cudaStream_t s);
  // (init, macros_d: nodes t0 .. t0 + cnt - 1 of the level, fields chunked
  // as rho[t - t0], u[a * us + t - t0])
  cudaError_t (*init)(const LevelView& v, int storage, int run, const double* rho, const double* u,
                      long long us, long long t0, long long cnt, const RefState& ref,
                      cudaStream_t s);
  cudaError_t (*macros_d)(const LevelView& v, int storage, int run, int last, double* rho,
                          double* u, long long us, long long t0, long long cnt,
                          const RefState& ref, cudaStream_t s);
  cudaError_t (*macros_f)(const LevelView& v, int storage, int run, int last, float* rho, float* u,
                          const RefState& ref, cudaStream_t s);
  cudaError_t (*populations)(const LevelView& v, int storage, int run, int last, double* out,
                             const RefState& ref, cudaStream_t s);
  cudaError_t (*diag_partial)(const LevelView& v, int storage, int run, int last, double* partial,
                              int nblocks, const RefState& ref, cudaStream_t s);
  cudaError_t (*noise_partial)(const LevelView& a, int last_a, const RefState& ra,
                               const LevelView& b, int last_b, const RefState& rb, int storage,
                               int run, const NoiseRegion& reg, double* partial, int nblocks,
                               cudaStream_t s);
  cudaError_t (*probe)(const LevelView& v, int storage, int last, const int* ijk, int n,
                       double* rec, int cap, unsigned long long* counter, const RefState& ref,
                       cudaStream_t s);
  // Persistent fused step (kernels_fused.cuh): bytes of the device tables;
  // fill them from the host description (synchronous copy); the largest
  // co-resident grid; the largest cluster; one launch of `blocks` blocks
  // (cooperative, or one cluster when A.cluster).
  size_t (*fused_tab_bytes)();
  cudaError_t (*fused_setup)(const FusedHost& hst, void* d_tab);
  int (*fused_max_blocks)(int storage);
  int (*fused_max_cluster)(int storage);
  cudaError_t (*fused)(const FusedArgs& A, int storage, int blocks, cudaStream_t s);
};

// (instantiated per lattice in fused_d2q9.cu, fused_d3q19.cu, fused_d3q27.cu)
template <class L>
size_t fused_tab_bytes();
template <class L>
cudaError_t fused_setup(const FusedHost& hst, void* d_tab);
template <class L>
int fused_max_blocks(int storage);
template <class L>
int fused_max_cluster(int storage);
template <class L>
cudaError_t fused_launch(const FusedArgs& A, int storage, int blocks, cudaStream_t s);

struct D2Q9;
struct D3Q19;
struct D3Q27;
template <class L>
Ops make_ops();

}  // namespace mlbm
