// Launch wrappers of the kernels for one lattice (included by the three
// per-lattice translation units).
#pragma once
#include "kernels.cuh"
#include "ops.cuh"

namespace mlbm {
namespace detail {

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <class L, class S, int COLL>
cudaError_t sc_launch(const LevelView& v, int par, float omega, float rho0, cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid((v.n[0] + 31) / 32, (v.n[1] + 3) / 4, v.n[2] * v.batch);
  if (par == 0)
    k_stream_collide<L, COLL, S, 0><<<grid, block, 0, s>>>(v, omega, rho0);
  else
    k_stream_collide<L, COLL, S, 1><<<grid, block, 0, s>>>(v, omega, rho0);
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t sc_coll(const LevelView& v, int coll, int par, float omega, float rho0,
                    cudaStream_t s) {
  switch (coll) {
    case 0: return sc_launch<L, S, 0>(v, par, omega, rho0, s);
    case 1: return sc_launch<L, S, 1>(v, par, omega, rho0, s);
    default: return sc_launch<L, S, 2>(v, par, omega, rho0, s);
  }
}

template <class L>
cudaError_t stream_collide(const LevelView& v, int coll, int storage, int par, float omega,
                           float rho0, cudaStream_t s) {
  return storage == 0 ? sc_coll<L, float>(v, coll, par, omega, rho0, s)
                      : sc_coll<L, __half>(v, coll, par, omega, rho0, s);
}

template <class L>
cudaError_t capture(const LevelView& p, const RingDesc& R, int storage, int par, int mode,
                    float rho0, cudaStream_t s) {
  if (R.K == 0) return cudaSuccess;
  dim3 grid(blocks_for(R.K, 128), p.batch);
  if (storage == 0)
    k_capture<L, float><<<grid, 128, 0, s>>>(p, R, par, mode, rho0);
  else
    k_capture<L, __half><<<grid, 128, 0, s>>>(p, R, par, mode, rho0);
  return cudaGetLastError();
}

template <class L>
cudaError_t inject(const LevelView& c, const BndDesc& B, const RingDesc& R, int storage,
                   const float* wt, float resc, int par, float rho0, cudaStream_t s) {
  if (B.count == 0) return cudaSuccess;
  dim3 grid(blocks_for(B.count, 128), c.batch);
  if (storage == 0)
    k_inject<L, float><<<grid, 128, 0, s>>>(c, B, R, wt[0], wt[1], wt[2], resc, par, rho0);
  else
    k_inject<L, __half><<<grid, 128, 0, s>>>(c, B, R, wt[0], wt[1], wt[2], resc, par, rho0);
  return cudaGetLastError();
}

template <class L>
cudaError_t restrict_tn(const LevelView& p, const LevelView& c, const TnDesc& T, int storage,
                        float resc, int ppar, int cpar, float rho0, cudaStream_t s) {
  if (T.count == 0) return cudaSuccess;
  dim3 grid(blocks_for(T.count, 64), p.batch);
  if (storage == 0)
    k_restrict<L, float><<<grid, 64, 0, s>>>(p, c, T, resc, ppar, cpar, rho0);
  else
    k_restrict<L, __half><<<grid, 64, 0, s>>>(p, c, T, resc, ppar, cpar, rho0);
  return cudaGetLastError();
}

inline long long nodes(const LevelView& v) { return (long long)v.n[0] * v.n[1] * v.n[2]; }

template <class L>
cudaError_t init(const LevelView& v, int storage, int run, const double* rho, const double* u,
                 double rho0, cudaStream_t s) {
  unsigned g = blocks_for(nodes(v), 128);
  if (storage == 0)
    k_init<L, float><<<g, 128, 0, s>>>(v, run, rho, u, rho0);
  else
    k_init<L, __half><<<g, 128, 0, s>>>(v, run, rho, u, rho0);
  return cudaGetLastError();
}

template <class L>
cudaError_t macros_d(const LevelView& v, int storage, int run, int last, double* rho, double* u,
                     double rho0, cudaStream_t s) {
  unsigned g = blocks_for(nodes(v), 128);
  if (storage == 0)
    k_macros<L, float, double><<<g, 128, 0, s>>>(v, run, last, rho, u, rho0);
  else
    k_macros<L, __half, double><<<g, 128, 0, s>>>(v, run, last, rho, u, rho0);
  return cudaGetLastError();
}

template <class L>
cudaError_t macros_f(const LevelView& v, int storage, int run, int last, float* rho, float* u,
                     double rho0, cudaStream_t s) {
  unsigned g = blocks_for(nodes(v), 128);
  if (storage == 0)
    k_macros<L, float, float><<<g, 128, 0, s>>>(v, run, last, rho, u, rho0);
  else
    k_macros<L, __half, float><<<g, 128, 0, s>>>(v, run, last, rho, u, rho0);
  return cudaGetLastError();
}

template <class L>
cudaError_t populations(const LevelView& v, int storage, int run, int last, double* out,
                        cudaStream_t s) {
  unsigned g = blocks_for(nodes(v), 128);
  if (storage == 0)
    k_populations<L, float><<<g, 128, 0, s>>>(v, run, last, out);
  else
    k_populations<L, __half><<<g, 128, 0, s>>>(v, run, last, out);
  return cudaGetLastError();
}

template <class L>
cudaError_t diag_partial(const LevelView& v, int storage, int run, int last, double* partial,
                         int nblocks, cudaStream_t s) {
  if (storage == 0)
    k_diag_partial<L, float><<<nblocks, kDiagThreads, 0, s>>>(v, run, last, partial);
  else
    k_diag_partial<L, __half><<<nblocks, kDiagThreads, 0, s>>>(v, run, last, partial);
  return cudaGetLastError();
}

template <class L>
cudaError_t probe(const LevelView& v, int storage, int last, const int* ijk, int n, double* rec,
                  int cap, unsigned long long* counter, double rho0, cudaStream_t s) {
  if (storage == 0)
    k_probe<L, float><<<1, 256, 0, s>>>(v, last, ijk, n, rec, cap, counter, rho0);
  else
    k_probe<L, __half><<<1, 256, 0, s>>>(v, last, ijk, n, rec, cap, counter, rho0);
  return cudaGetLastError();
}

}  // namespace detail

template <class L>
Ops make_ops() {
  Ops o;
  o.q = L::Q;
  o.d = L::D;
  o.stream_collide = detail::stream_collide<L>;
  o.capture = detail::capture<L>;
  o.inject = detail::inject<L>;
  o.restrict_tn = detail::restrict_tn<L>;
  o.init = detail::init<L>;
  o.macros_d = detail::macros_d<L>;
  o.macros_f = detail::macros_f<L>;
  o.populations = detail::populations<L>;
  o.diag_partial = detail::diag_partial<L>;
  o.probe = detail::probe<L>;
  return o;
}

}  // namespace mlbm
