// Launch wrappers of the kernels for one lattice (included by the three
// per-lattice translation units).
#pragma once
#include "kernels.cuh"
#include "kernels_hrr.cuh"
#include "kernels_sensor.cuh"
#include "ops.cuh"

namespace mlbm {
namespace detail {

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// binary32 reference state with the per-direction constants 1 + e_i(U) and
// 2 xi_i.U, formed in double precision.
template <class L>
RefF make_ref_f(const RefState& r) {
  RefF R{};
  R.rho0 = (float)r.rho0;
  R.Ux = (float)r.U[0];
  R.Uy = (float)r.U[1];
  R.Uz = L::D == 3 ? (float)r.U[2] : 0.0f;
  const double Uz = L::D == 3 ? r.U[2] : 0.0;
  double eU[L::Q];
  // e_i(U) = (f0_i(1, U) - w_i) / w_i
  double f0[L::Q];
  equilibrium_dev<L, double>(0.0, r.U[0], r.U[1], Uz, 1.0, 0.0, 0.0, 0.0, f0);
  for (int i = 0; i < L::Q; ++i) {
    eU[i] = f0[i] / L::w(i);
    R.c1[i] = (float)(1.0 + eU[i]);
    R.cU2[i] = (float)(2.0 * (L::c(i, 0) * r.U[0] + L::c(i, 1) * r.U[1] + L::c(i, 2) * Uz));
  }
  return R;
}

template <class L, class S, int COLL>
cudaError_t sc_x2_launch(const LevelView& v, int par, float omega, const RefState& ref, int bx,
                         int by, const S* xf, cudaStream_t s) {
  if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 128) return cudaErrorInvalidValue;
  if (v.run_stride >= (1LL << 31)) return cudaErrorInvalidValue;  // (32-bit offsets)
  dim3 block(bx, by, 1);
  dim3 grid((v.n[0] + bx - 1) / bx, (v.n[1] + 2 * by - 1) / (2 * by),
            (v.n[2] + K1X2Pfz<S>::PZ - 1) / K1X2Pfz<S>::PZ * v.batch);
  const bool mov = ref.U[0] != 0.0 || ref.U[1] != 0.0 || ref.U[2] != 0.0;
  const RefF R = make_ref_f<L>(ref);
  if (mov) {
    if (par == 0)
      k_stream_collide_x2<L, S, COLL, 0, true><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide_x2<L, S, COLL, 1, true><<<grid, block, 0, s>>>(v, omega, R, xf);
  } else {
    if (par == 0)
      k_stream_collide_x2<L, S, COLL, 0, false><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide_x2<L, S, COLL, 1, false><<<grid, block, 0, s>>>(v, omega, R, xf);
  }
  return cudaGetLastError();
}

template <class L, class S, int COLL>
cudaError_t sc_launch(const LevelView& v, int par, float omega, const RefState& ref, int bx, int by,
                      const S* xf, cudaStream_t s) {
  // (the two-node update addresses a run with 32-bit offsets: larger runs
  // take the one-node update)
  if constexpr ((std::is_same<S, float>::value && K1X2Tune<L>::ON) ||
                (std::is_same<S, __half>::value && K1X2Tune<L>::ON_H))
    if (v.run_stride < (1LL << 31)) return sc_x2_launch<L, S, COLL>(v, par, omega, ref, bx, by, xf, s);
  constexpr int NPT = K1Tune<L, S>::NPT;
  if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 128) return cudaErrorInvalidValue;
  dim3 block(bx, by, 1);
  dim3 grid((v.n[0] + bx - 1) / bx, (v.n[1] + by * NPT - 1) / (by * NPT), v.n[2] * v.batch);
  const bool mov = ref.U[0] != 0.0 || ref.U[1] != 0.0 || ref.U[2] != 0.0;
  const RefF R = make_ref_f<L>(ref);
  if (mov) {
    if (par == 0)
      k_stream_collide<L, COLL, S, 0, true><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide<L, COLL, S, 1, true><<<grid, block, 0, s>>>(v, omega, R, xf);
  } else {
    if (par == 0)
      k_stream_collide<L, COLL, S, 0, false><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide<L, COLL, S, 1, false><<<grid, block, 0, s>>>(v, omega, R, xf);
  }
  return cudaGetLastError();
}

template <class L, int COLL>
cudaError_t sc_pair_launch(const LevelView& v, int par, float omega, const RefState& ref, int bx,
                           int by, const __half* xf, cudaStream_t s) {
  if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 128) return cudaErrorInvalidValue;
  dim3 block(bx, by, 1);
  dim3 grid((v.n[0] + bx - 1) / bx, (v.n[1] + by - 1) / by, v.n[2] * ((v.batch + 1) / 2));
  const bool mov = ref.U[0] != 0.0 || ref.U[1] != 0.0 || ref.U[2] != 0.0;
  const RefF R = make_ref_f<L>(ref);
  if (mov) {
    if (par == 0)
      k_stream_collide_pair<L, COLL, 0, true><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide_pair<L, COLL, 1, true><<<grid, block, 0, s>>>(v, omega, R, xf);
  } else {
    if (par == 0)
      k_stream_collide_pair<L, COLL, 0, false><<<grid, block, 0, s>>>(v, omega, R, xf);
    else
      k_stream_collide_pair<L, COLL, 1, false><<<grid, block, 0, s>>>(v, omega, R, xf);
  }
  return cudaGetLastError();
}

template <class L, class S>
cudaError_t sc_coll(const LevelView& v, int coll, int par, float omega, const RefState& ref,
                    int bx, int by, const void* xf, cudaStream_t s) {
  const S* xs = static_cast<const S*>(xf);
  if (std::is_same<S, __half>::value && v.es == 2) {
    const __half* xh = static_cast<const __half*>(xf);
    switch (coll) {
      case 0: return sc_pair_launch<L, 0>(v, par, omega, ref, bx, by, xh, s);
      case 1: return sc_pair_launch<L, 1>(v, par, omega, ref, bx, by, xh, s);
      default: return sc_pair_launch<L, 2>(v, par, omega, ref, bx, by, xh, s);
    }
  }
  switch (coll) {
    case 0: return sc_launch<L, S, 0>(v, par, omega, ref, bx, by, xs, s);
    case 1: return sc_launch<L, S, 1>(v, par, omega, ref, bx, by, xs, s);
    default: return sc_launch<L, S, 2>(v, par, omega, ref, bx, by, xs, s);
  }
}

template <class L>
cudaError_t stream_collide(const LevelView& v, int coll, int storage, int par, float omega,
                           const RefState& ref, int bx, int by, const void* xf,
                           cudaStream_t s) {
  return storage == 0 ? sc_coll<L, float>(v, coll, par, omega, ref, bx, by, xf, s)
                      : sc_coll<L, __half>(v, coll, par, omega, ref, bx, by, xf, s);
}

template <class L>
cudaError_t capture(const LevelView& p, const RingDesc& R, int storage, int par, int mode,
                    int s_new, int s_also, const RefState& ref, cudaStream_t s) {
  if (R.K == 0) return cudaSuccess;
  dim3 grid(blocks_for(R.K, 64), p.batch);
  if (storage == 0)
    k_capture<L, float><<<grid, 64, 0, s>>>(p, R, par, mode, s_new, s_also, make_ref_f<L>(ref));
  else
    k_capture<L, __half><<<grid, 64, 0, s>>>(p, R, par, mode, s_new, s_also, make_ref_f<L>(ref));
  return cudaGetLastError();
}

template <class L>
cudaError_t inject(const LevelView& c, const BndDesc& B, const RingDesc& R, int storage,
                   const float* wt, const int* slots, float resc, int par, const RefState& ref,
                   void* xf, cudaStream_t s) {
  if (B.count == 0) return cudaSuccess;
  using T = InjTile<L>;
  InjDesc J{};
  J.nf = B.nf;
  J.tstart[0] = 0;
  for (int a = 0; a < 3; ++a) J.boxed[a] = R.boxed[a];
  for (int f = 0; f < B.nf; ++f) {
    const int a = B.axis[f];
    J.axis[f] = a;
    J.side[f] = B.side[f];
    if (L::D == 2) {
      J.t1[f] = 1 - a;
      J.t2[f] = 2;
    } else {
      J.t1[f] = (a == 0) ? 1 : 0;
      J.t2[f] = (a == 2) ? 1 : 2;
    }
    J.ntile1[f] = (c.n[J.t1[f]] + T::TI - 1) / T::TI;
    J.ntile2[f] = (L::D == 3) ? (c.n[J.t2[f]] + T::TJ - 1) / T::TJ : 1;
    J.tstart[f + 1] = J.tstart[f] + (long long)J.ntile1[f] * J.ntile2[f];
  }
  dim3 grid((unsigned)J.tstart[J.nf], c.batch);
  if constexpr (L::D == 3) {
    dim3 block(T::TI, T::TJ);
    if (storage == 0)
      k_inject_sep<L, float><<<grid, block, 0, s>>>(c, J, R, wt[0], wt[1], wt[2], slots[0],
                                                    slots[1], slots[2], resc, par,
                                                    make_ref_f<L>(ref), static_cast<float*>(xf));
    else
      k_inject_sep<L, __half><<<grid, block, 0, s>>>(c, J, R, wt[0], wt[1], wt[2], slots[0],
                                                     slots[1], slots[2], resc, par,
                                                     make_ref_f<L>(ref), static_cast<__half*>(xf));
    return cudaGetLastError();
  }
  dim3 block(T::TI, T::TJ, T::G);
  if (storage == 0)
    k_inject<L, float><<<grid, block, 0, s>>>(c, J, R, wt[0], wt[1], wt[2], slots[0], slots[1],
                                              slots[2], resc, par, make_ref_f<L>(ref),
                                              static_cast<float*>(xf));
  else
    k_inject<L, __half><<<grid, block, 0, s>>>(c, J, R, wt[0], wt[1], wt[2], slots[0], slots[1],
                                               slots[2], resc, par, make_ref_f<L>(ref),
                                               static_cast<__half*>(xf));
  return cudaGetLastError();
}

// Face tiles of the TN nodes for k_restrict_tile.
template <class L>
RstDesc rst_desc(const TnDesc& T) {
  using TT = RstTile<L>;
  RstDesc J{};
  J.tstart[0] = 0;
  for (int f = 0; f < T.nf; ++f) {
    const int a = T.axis[f];
    if (L::D == 2) {
      J.t1[f] = 1 - a;
      J.t2[f] = 2;
    } else {
      J.t1[f] = (a == 0) ? 1 : 0;
      J.t2[f] = (a == 2) ? 1 : 2;
    }
    J.ntile1[f] = (T.rext[f][J.t1[f]] + TT::TI - 1) / TT::TI;
    const int nt2 = (T.rext[f][J.t2[f]] + TT::TJ - 1) / TT::TJ;
    J.tstart[f + 1] = J.tstart[f] + (long long)J.ntile1[f] * nt2;
  }
  return J;
}

template <class L>
cudaError_t restrict_tn(const LevelView& p, const LevelView& c, const TnDesc& T, int storage,
                        float resc, int ppar, int cpar, const RefState& ref, cudaStream_t s) {
  if (T.count == 0) return cudaSuccess;
  const RstDesc J = rst_desc<L>(T);
  dim3 block(32, RstTile<L>::NW);
  dim3 grid((unsigned)J.tstart[T.nf], p.batch);
  const RefF R = make_ref_f<L>(ref);
  if (storage == 0)
    k_restrict_tile<L, float, false, false><<<grid, block, 0, s>>>(p, c, T, J, resc, ppar, cpar,
                                                                   R, nullptr, 0.0f, 1.0f, 0.0f);
  else
    k_restrict_tile<L, __half, false, false><<<grid, block, 0, s>>>(
        p, c, T, J, resc, ppar, cpar, R, nullptr, 0.0f, 1.0f, 0.0f);
  return cudaGetLastError();
}

inline bool moving(const RefState& ref) {
  return ref.U[0] != 0.0 || ref.U[1] != 0.0 || ref.U[2] != 0.0;
}

template <class L, class S, bool MOV>
void restrict_hrr_t(const LevelView& p, const LevelView& c, const TnDesc& T, float resc, int ppar,
                    int cpar, float* pdu, float omega_p, float sig, float ks_p, const RefF& R,
                    cudaStream_t s) {
  const RstDesc J = rst_desc<L>(T);
  dim3 block(32, RstTile<L>::NW);
  dim3 grid((unsigned)J.tstart[T.nf], p.batch);
  k_restrict_tile<L, S, true, MOV><<<grid, block, 0, s>>>(p, c, T, J, resc, ppar, cpar, R, pdu,
                                                          omega_p, sig, ks_p);
}

template <class L>
cudaError_t restrict_hrr(const LevelView& p, const LevelView& c, const TnDesc& T, int storage,
                         float resc, int ppar, int cpar, float* pdu, float omega_p, float sig,
                         float ks_p, const RefState& ref, cudaStream_t s) {
  if (T.count == 0) return cudaSuccess;
  const RefF R = make_ref_f<L>(ref);
  const bool mov = moving(ref);
  if (storage == 0) {
    if (mov)
      restrict_hrr_t<L, float, true>(p, c, T, resc, ppar, cpar, pdu, omega_p, sig, ks_p, R, s);
    else
      restrict_hrr_t<L, float, false>(p, c, T, resc, ppar, cpar, pdu, omega_p, sig, ks_p, R, s);
  } else {
    if (mov)
      restrict_hrr_t<L, __half, true>(p, c, T, resc, ppar, cpar, pdu, omega_p, sig, ks_p, R, s);
    else
      restrict_hrr_t<L, __half, false>(p, c, T, resc, ppar, cpar, pdu, omega_p, sig, ks_p, R, s);
  }
  return cudaGetLastError();
}

template <class L>
cudaError_t velocity(const LevelView& v, int storage, int par, float* du, const RefState& ref,
                     cudaStream_t s) {
  const long long n = (long long)v.n[0] * v.n[1] * v.n[2];
  dim3 grid(blocks_for(n, 128), v.batch);
  if (storage == 0)
    k_velocity<L, float><<<grid, 128, 0, s>>>(v, du, par, make_ref_f<L>(ref));
  else
    k_velocity<L, __half><<<grid, 128, 0, s>>>(v, du, par, make_ref_f<L>(ref));
  return cudaGetLastError();
}

template <class L, class S, bool MOV>
void sc_hrr_t(const LevelView& v, int par, float omega, const float* du, float sig, float ks,
              const RefF& R, cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid((v.n[0] + 31) / 32, (v.n[1] + 3) / 4, v.n[2] * v.batch);
  if (par == 0)
    k_stream_collide_hrr<L, S, 0, MOV><<<grid, block, 0, s>>>(v, omega, R, du, sig, ks);
  else
    k_stream_collide_hrr<L, S, 1, MOV><<<grid, block, 0, s>>>(v, omega, R, du, sig, ks);
}

template <class L>
cudaError_t stream_collide_hrr(const LevelView& v, int storage, int par, float omega,
                               const float* du, float sig, float ks, const RefState& ref,
                               cudaStream_t s) {
  const RefF R = make_ref_f<L>(ref);
  const bool mov = moving(ref);
  if (storage == 0) {
    if (mov)
      sc_hrr_t<L, float, true>(v, par, omega, du, sig, ks, R, s);
    else
      sc_hrr_t<L, float, false>(v, par, omega, du, sig, ks, R, s);
  } else {
    if (mov)
      sc_hrr_t<L, __half, true>(v, par, omega, du, sig, ks, R, s);
    else
      sc_hrr_t<L, __half, false>(v, par, omega, du, sig, ks, R, s);
  }
  return cudaGetLastError();
}

template <class L>
cudaError_t parent_strain(const LevelView& p, const LevelView& c, const RingDesc& R,
                          const TnDesc& T, int storage, float* sh, int s_new, int s_also, int ppar,
                          int cpar, int mode, const RefState& ref, cudaStream_t s) {
  if (R.K == 0) return cudaSuccess;
  dim3 grid(blocks_for(R.K, 64), p.batch);
  if (storage == 0)
    k_parent_strain<L, float><<<grid, 64, 0, s>>>(p, c, R, T, sh, s_new, s_also, ppar, cpar,
                                                  mode, make_ref_f<L>(ref));
  else
    k_parent_strain<L, __half><<<grid, 64, 0, s>>>(p, c, R, T, sh, s_new, s_also, ppar, cpar,
                                                   mode, make_ref_f<L>(ref));
  return cudaGetLastError();
}

template <class L>
cudaError_t sensors(const LevelView& v, int storage, const float* du, int par,
                    const SensorState& st, const RefState& ref, cudaStream_t s) {
  const long long n = (long long)v.n[0] * v.n[1] * v.n[2];
  dim3 grid(blocks_for(n, 128), v.batch);
  if (storage == 0)
    k_sensors<L, float><<<grid, 128, 0, s>>>(v, du, par, st, make_ref_f<L>(ref));
  else
    k_sensors<L, __half><<<grid, 128, 0, s>>>(v, du, par, st, make_ref_f<L>(ref));
  return cudaGetLastError();
}

template <class L>
cudaError_t sensor_read(const LevelView& v, int run, const SensorState& st, unsigned char* flags,
                        double* div, double* curl, double* gnorm, cudaStream_t s) {
  const long long n = (long long)v.n[0] * v.n[1] * v.n[2];
  k_sensor_read<L><<<blocks_for(n, 128), 128, 0, s>>>(v, run, st, flags, div, curl, gnorm);
  return cudaGetLastError();
}

template <class L, class S, bool MOV>
void collide_bnd_t(const LevelView& c, const BndDesc& B, const RingDesc& R, const float* sh,
                   const float* wt, const int* slots, float omega, float sig, float ks, int par,
                   const RefF& ref, cudaStream_t s) {
  dim3 grid(blocks_for(B.count, 64), c.batch);
  k_collide_bnd<L, S, MOV><<<grid, 64, 0, s>>>(c, B, R, sh, wt[0], wt[1], wt[2], slots[0],
                                               slots[1], slots[2], omega, sig, ks, par, ref);
}

template <class L>
cudaError_t collide_bnd(const LevelView& c, const BndDesc& B, const RingDesc& R, int storage,
                        const float* sh, const float* wt, const int* slots, float omega, float sig,
                        float ks, int par, const RefState& ref, cudaStream_t s) {
  if (B.count == 0) return cudaSuccess;
  const RefF Rf = make_ref_f<L>(ref);
  const bool mov = moving(ref);
  if (storage == 0) {
    if (mov)
      collide_bnd_t<L, float, true>(c, B, R, sh, wt, slots, omega, sig, ks, par, Rf, s);
    else
      collide_bnd_t<L, float, false>(c, B, R, sh, wt, slots, omega, sig, ks, par, Rf, s);
  } else {
    if (mov)
      collide_bnd_t<L, __half, true>(c, B, R, sh, wt, slots, omega, sig, ks, par, Rf, s);
    else
      collide_bnd_t<L, __half, false>(c, B, R, sh, wt, slots, omega, sig, ks, par, Rf, s);
  }
  return cudaGetLastError();
}

inline long long nodes(const LevelView& v) { return (long long)v.n[0] * v.n[1] * v.n[2]; }

template <class L>
cudaError_t init(const LevelView& v, int storage, int run, const double* rho, const double* u,
                 long long us, long long t0, long long cnt, const RefState& ref,
                 cudaStream_t s) {
  if (cnt <= 0) return cudaSuccess;
  unsigned g = blocks_for(cnt, 128);
  if (storage == 0)
    k_init<L, float><<<g, 128, 0, s>>>(v, run, rho, u, us, t0, cnt, ref, make_ref_f<L>(ref));
  else
    k_init<L, __half><<<g, 128, 0, s>>>(v, run, rho, u, us, t0, cnt, ref,
                                        make_ref_f<L>(ref));
  return cudaGetLastError();
}

template <class L>
cudaError_t macros_d(const LevelView& v, int storage, int run, int last, double* rho, double* u,
                     long long us, long long t0, long long cnt, const RefState& ref,
                     cudaStream_t s) {
  if (cnt <= 0) return cudaSuccess;
  unsigned g = blocks_for(cnt, 128);
  if (storage == 0)
    k_macros<L, float, double><<<g, 128, 0, s>>>(v, run, last, rho, u, us, t0, cnt, ref);
  else
    k_macros<L, __half, double><<<g, 128, 0, s>>>(v, run, last, rho, u, us, t0, cnt, ref);
  return cudaGetLastError();
}

template <class L>
cudaError_t macros_f(const LevelView& v, int storage, int run, int last, float* rho, float* u,
                     const RefState& ref, cudaStream_t s) {
  const long long N = nodes(v);
  unsigned g = blocks_for(N, 128);
  if (storage == 0)
    k_macros<L, float, float><<<g, 128, 0, s>>>(v, run, last, rho, u, N, 0, N, ref);
  else
    k_macros<L, __half, float><<<g, 128, 0, s>>>(v, run, last, rho, u, N, 0, N, ref);
  return cudaGetLastError();
}

template <class L>
cudaError_t populations(const LevelView& v, int storage, int run, int last, double* out,
                        const RefState& ref, cudaStream_t s) {
  unsigned g = blocks_for(nodes(v), 128);
  if (storage == 0)
    k_populations<L, float><<<g, 128, 0, s>>>(v, run, last, out, ref);
  else
    k_populations<L, __half><<<g, 128, 0, s>>>(v, run, last, out, ref);
  return cudaGetLastError();
}

template <class L>
cudaError_t diag_partial(const LevelView& v, int storage, int run, int last, double* partial,
                         int nblocks, const RefState& ref, cudaStream_t s) {
  if (storage == 0)
    k_diag_partial<L, float><<<nblocks, kDiagThreads, 0, s>>>(v, run, last, partial, ref);
  else
    k_diag_partial<L, __half><<<nblocks, kDiagThreads, 0, s>>>(v, run, last, partial, ref);
  return cudaGetLastError();
}

template <class L>
cudaError_t noise_partial(const LevelView& a, int last_a, const RefState& ra, const LevelView& b,
                          int last_b, const RefState& rb, int storage, int run,
                          const NoiseRegion& reg, double* partial, int nblocks, cudaStream_t s) {
  if (storage == 0)
    k_noise_partial<L, float><<<nblocks, kDiagThreads, 0, s>>>(a, last_a, ra, b, last_b, rb, run,
                                                               reg, partial);
  else
    k_noise_partial<L, __half><<<nblocks, kDiagThreads, 0, s>>>(a, last_a, ra, b, last_b, rb,
                                                                run, reg, partial);
  return cudaGetLastError();
}

template <class L>
cudaError_t probe(const LevelView& v, int storage, int last, const int* ijk, int n, double* rec,
                  int cap, unsigned long long* counter, const RefState& ref, cudaStream_t s) {
  if (storage == 0)
    k_probe<L, float><<<1, 256, 0, s>>>(v, last, ijk, n, rec, cap, counter, ref);
  else
    k_probe<L, __half><<<1, 256, 0, s>>>(v, last, ijk, n, rec, cap, counter, ref);
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
  o.velocity = detail::velocity<L>;
  o.stream_collide_hrr = detail::stream_collide_hrr<L>;
  o.parent_strain = detail::parent_strain<L>;
  o.collide_bnd = detail::collide_bnd<L>;
  o.restrict_hrr = detail::restrict_hrr<L>;
  o.sensors = detail::sensors<L>;
  o.sensor_read = detail::sensor_read<L>;
  o.init = detail::init<L>;
  o.macros_d = detail::macros_d<L>;
  o.macros_f = detail::macros_f<L>;
  o.populations = detail::populations<L>;
  o.diag_partial = detail::diag_partial<L>;
  o.noise_partial = detail::noise_partial<L>;
  o.probe = detail::probe<L>;
  o.fused_tab_bytes = fused_tab_bytes<L>;
  o.fused_setup = fused_setup<L>;
  o.fused_max_blocks = fused_max_blocks<L>;
  o.fused_max_cluster = fused_max_cluster<L>;
  o.fused = fused_launch<L>;
  return o;
}

}  // namespace mlbm
