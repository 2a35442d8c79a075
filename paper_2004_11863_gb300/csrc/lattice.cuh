// Velocity sets and the Hermite-equilibrium / collision arithmetic of the
// level update, evaluated in binary32 on shifted populations
// g_i = f_i - f0_i(rho0, U): deviations from the equilibrium of a reference
// state (rho0, U).  With U = 0 this is the rest-state shift f_i - w_i rho0;
// a reference velocity near the flow's mean velocity keeps the stored values
// (and every rounding of them) small where the flow is close to it.  All
// arithmetic below is written in the deviations drho = rho - rho0 and
// du = u - U, so that no large terms cancel.
//
// Lattices: D2Q9 in the velocity order of Sec. 3.1 (eqs. xi_i, w_i); D3Q19
// and D3Q27 built the same way (weights 1/3, 1/18, 1/36 and 8/27, 2/27, 1/54,
// 1/216).  c_s^2 = 1/3 on all three.
//
// Equilibrium (eq. fEqH truncated at third order, eq. fEqO3 in 2D):
//   f0_i = w_i rho [1 + 3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u + T3_i(u u u)],
// where T3 is the lattice-supported third-order Hermite term set:
//   D2Q9:  H_xxy, H_xyy with 1/(2 cs^6);
//   D3Q27: the six H_aab with 1/(2 cs^6) and H_xyz with 1/cs^6;
//   D3Q19: for each odd axis b the orthogonal pair H_aab +- H_ccb, with
//          1/(2 cs^6) on the sum and 1/(6 cs^6) on the difference
//          (H_aab and H_ccb are not orthogonal on D3Q19 and H_xyz vanishes).
// Regularized collisions (eqs. reguProcedure, a1Proj, LBMscheme_reg, f1RR,
// a13RR): a1 = sum H2 (f - f0) is formed directly from the shifted second
// moment, a1_ab = sum xi_a xi_b g - rho u_a u_b - drho cs^2 delta_ab, and the
// post-collision state is f0 + (1 - 1/tau) f1 with
//   f1_i = w_i [4.5 H2_i : a1 + T3_i(a1^(3))],
//   a1^(3)_abc = u_a a1_bc + u_b a1_ac + u_c a1_ab   (RR; zero for REG).
#pragma once
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

namespace mlbm {

// ---------------------------------------------------------------- unrolling
template <class F, int... I>
__host__ __device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------------------ lattices
struct D2Q9 {
  static constexpr int Q = 9, D = 2, ID = 0;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

// 3D sets: rest, then the 6 axis neighbours, then the 12 edge neighbours,
// then (D3Q27) the 8 corners; opposite pairs are adjacent (i, i+1) after 0.
struct D3Q19 {
  static constexpr int Q = 19, D = 3, ID = 1;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

struct D3Q27 {
  static constexpr int Q = 27, D = 3, ID = 2;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[27][3] = {
        {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
        {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
        {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},  {-1, -1, -1},
        {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
};

template <class L>
__host__ __device__ constexpr int opp(int i) {
  int k = 0;
  for (int j = 0; j < L::Q; ++j)
    if (L::c(j, 0) == -L::c(i, 0) && L::c(j, 1) == -L::c(i, 1) && L::c(j, 2) == -L::c(i, 2)) k = j;
  return k;
}

// Directions come in opposite pairs (i, opp(i)); pair_first<L>(p) is the
// lower index of the p-th pair, p = 0 .. (Q-1)/2 - 1.
template <class L>
__host__ __device__ constexpr int pair_first(int p) {
  int k = 0;
  for (int i = 1; i < L::Q; ++i)
    if (i < opp<L>(i)) {
      if (k == p) return i;
      ++k;
    }
  return -1;
}

// Third-order Hermite polynomial H_aab(xi_i) = xi_a^2 xi_b - cs^2 xi_b.
template <class L>
__host__ __device__ constexpr double h3(int i, int a, int b) {
  return double(L::c(i, a) * L::c(i, a) * L::c(i, b)) - double(L::c(i, b)) / 3.0;
}

// Third-order coefficient set, indexed [xxy, xxz, yyx, yyz, zzx, zzy, xyz].
enum { XXY = 0, XXZ, YYX, YYZ, ZZX, ZZY, XYZ };

// T3_i(A): the lattice-supported third-order term of the Hermite expansion
// for coefficients A (already including every factor except w_i).
template <class L, int I, class T>
__host__ __device__ __forceinline__ T third(const T (&A)[7]) {
  if constexpr (L::ID == 0) {
    constexpr T hxxy = T(13.5 * h3<L>(I, 0, 1)), hyyx = T(13.5 * h3<L>(I, 1, 0));
    return hxxy * A[XXY] + hyyx * A[YYX];
  } else if constexpr (L::ID == 2) {
    constexpr T k0 = T(13.5 * h3<L>(I, 0, 1)), k1 = T(13.5 * h3<L>(I, 0, 2)),
                k2 = T(13.5 * h3<L>(I, 1, 0)), k3 = T(13.5 * h3<L>(I, 1, 2)),
                k4 = T(13.5 * h3<L>(I, 2, 0)), k5 = T(13.5 * h3<L>(I, 2, 1)),
                k6 = T(27.0 * L::c(I, 0) * L::c(I, 1) * L::c(I, 2));
    return k0 * A[XXY] + k1 * A[XXZ] + k2 * A[YYX] + k3 * A[YYZ] + k4 * A[ZZX] + k5 * A[ZZY] +
           k6 * A[XYZ];
  } else {
    // odd axis y: (xxy, zzy); odd axis x: (yyx, zzx); odd axis z: (xxz, yyz)
    constexpr T py = T(13.5 * (h3<L>(I, 0, 1) + h3<L>(I, 2, 1))),
                my = T(4.5 * (h3<L>(I, 0, 1) - h3<L>(I, 2, 1)));
    constexpr T px = T(13.5 * (h3<L>(I, 1, 0) + h3<L>(I, 2, 0))),
                mx = T(4.5 * (h3<L>(I, 1, 0) - h3<L>(I, 2, 0)));
    constexpr T pz = T(13.5 * (h3<L>(I, 0, 2) + h3<L>(I, 1, 2))),
                mz = T(4.5 * (h3<L>(I, 0, 2) - h3<L>(I, 1, 2)));
    return py * (A[XXY] + A[ZZY]) + my * (A[XXY] - A[ZZY]) + px * (A[YYX] + A[ZZX]) +
           mx * (A[YYX] - A[ZZX]) + pz * (A[XXZ] + A[YYZ]) + mz * (A[XXZ] - A[YYZ]);
  }
}

// w_i * x without a systematic bias: binary32 cannot hold 1/9, 1/36, ...
// exactly, and a rounded weight would shift the equilibrium's mass and
// momentum by the same relative amount at every update (a drift that adds up
// over long runs).  The weight is split into a binary32 head and tail.
template <class L, int I, class T>
__host__ __device__ __forceinline__ T wmul(T x) {
  if constexpr (std::is_same<T, float>::value) {
    constexpr float hi = float(L::w(I));
    constexpr float lo = float(L::w(I) - double(hi));
    return fmaf(hi, x, lo * x);
  } else {
    return T(L::w(I)) * x;
  }
}

// xi_i . v with compile-time components.
template <class L, int I, class T>
__host__ __device__ __forceinline__ T cdot(T vx, T vy, T vz) {
  T s = T(0);
  if constexpr (L::c(I, 0) == 1) s += vx;
  if constexpr (L::c(I, 0) == -1) s -= vx;
  if constexpr (L::c(I, 1) == 1) s += vy;
  if constexpr (L::c(I, 1) == -1) s -= vy;
  if constexpr (L::D == 3) {
    if constexpr (L::c(I, 2) == 1) s += vz;
    if constexpr (L::c(I, 2) == -1) s -= vz;
  }
  return s;
}

// Macroscopic moments of shifted populations: drho = sum g, j = sum xi g.
template <class L, class T>
__host__ __device__ __forceinline__ void moments(const T (&g)[L::Q], T& drho, T& jx, T& jy,
                                                 T& jz) {
  drho = jx = jy = jz = T(0);
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    drho += g[i];
    if constexpr (L::c(i, 0) == 1) jx += g[i];
    if constexpr (L::c(i, 0) == -1) jx -= g[i];
    if constexpr (L::c(i, 1) == 1) jy += g[i];
    if constexpr (L::c(i, 1) == -1) jy -= g[i];
    if constexpr (L::c(i, 2) == 1) jz += g[i];
    if constexpr (L::c(i, 2) == -1) jz -= g[i];
  });
}

// Moments from per-axis class sums: S+_a = sum over xi_a = +1, S-_a = sum
// over xi_a = -1; then j_a = S+_a - S-_a and the diagonal second moment
// P_aa = S+_a + S-_a, and drho = S+_x + S-_x + (sum over xi_x = 0).  The
// off-diagonal P_ab sum the four directions with xi_a xi_b = +-1.
template <class L>
__device__ __forceinline__ void moments2(const float (&g)[L::Q], float& drho, float (&j)[3],
                                         float (&pd)[3], float (&po)[3]) {
  float sp[3] = {0, 0, 0}, sm[3] = {0, 0, 0}, s0 = 0.0f;
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (L::c(i, 0) == 1) sp[0] += g[i];
    if constexpr (L::c(i, 0) == -1) sm[0] += g[i];
    if constexpr (L::c(i, 0) == 0) s0 += g[i];
  });
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (L::c(i, 1) == 1) sp[1] += g[i];
    if constexpr (L::c(i, 1) == -1) sm[1] += g[i];
    if constexpr (L::D == 3) {
      if constexpr (L::c(i, 2) == 1) sp[2] += g[i];
      if constexpr (L::c(i, 2) == -1) sm[2] += g[i];
    }
  });
  drho = (sp[0] + sm[0]) + s0;
  for (int a = 0; a < 3; ++a) {
    j[a] = sp[a] - sm[a];
    pd[a] = sp[a] + sm[a];
  }
  float pxy_p = 0, pxy_m = 0, pxz_p = 0, pxz_m = 0, pyz_p = 0, pyz_m = 0;
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    if constexpr (cx * cy == 1) pxy_p += g[i];
    if constexpr (cx * cy == -1) pxy_m += g[i];
    if constexpr (cx * cz == 1) pxz_p += g[i];
    if constexpr (cx * cz == -1) pxz_m += g[i];
    if constexpr (cy * cz == 1) pyz_p += g[i];
    if constexpr (cy * cz == -1) pyz_m += g[i];
  });
  po[0] = pxy_p - pxy_m;
  po[1] = pxz_p - pxz_m;
  po[2] = pyz_p - pyz_m;
}

// Third-order coefficients of u (A) and their deviations from those of U
// (dA = A(u) - A(U)), in the order [xxy, xxz, yyx, yyz, zzx, zzy, xyz].
template <class T>
__host__ __device__ __forceinline__ void third_coeffs(T ux, T uy, T uz, T dux, T duy, T duz,
                                                      T Ux, T Uy, T Uz, T (&A)[7], T (&dA)[7]) {
  A[XXY] = ux * ux * uy;
  A[XXZ] = ux * ux * uz;
  A[YYX] = uy * uy * ux;
  A[YYZ] = uy * uy * uz;
  A[ZZX] = uz * uz * ux;
  A[ZZY] = uz * uz * uy;
  A[XYZ] = ux * uy * uz;
  // a^2 b - A^2 B = da (a + A) b + A^2 db
  dA[XXY] = dux * (ux + Ux) * uy + Ux * Ux * duy;
  dA[XXZ] = dux * (ux + Ux) * uz + Ux * Ux * duz;
  dA[YYX] = duy * (uy + Uy) * ux + Uy * Uy * dux;
  dA[YYZ] = duy * (uy + Uy) * uz + Uy * Uy * duz;
  dA[ZZX] = duz * (uz + Uz) * ux + Uz * Uz * dux;
  dA[ZZY] = duz * (uz + Uz) * uy + Uz * Uz * duy;
  dA[XYZ] = dux * uy * uz + Ux * (duy * uz + Uy * duz);
}

// Equilibrium deviation for direction I:
//   g0_i = f0_i(rho0 + drho, U + du) - f0_i(rho0, U)
//        = w_i [ drho (1 + e_i(u)) + rho0 (e_i(u) - e_i(U)) ],
//   e_i(u) = 3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u + T3_i(u u u),
//   e_i(u) - e_i(U) = 3 xi.du + 4.5 (xi.du)(xi.u + xi.U) - 1.5 du.(u + U) + T3_i(dA).
template <class L, int I, class T>
__host__ __device__ __forceinline__ T eq_dev_i(T drho, T rho0, T ux, T uy, T uz, T dux, T duy,
                                               T duz, T Ux, T Uy, T Uz, T usq, T dusq,
                                               const T (&A)[7], const T (&dA)[7]) {
  const T cu = cdot<L, I>(ux, uy, uz);
  const T cdu = cdot<L, I>(dux, duy, duz);
  const T cU = cdot<L, I>(Ux, Uy, Uz);
  const T e = T(3) * cu + T(4.5) * cu * cu - usq + third<L, I>(A);
  const T de = T(3) * cdu + T(4.5) * cdu * (cu + cU) - dusq + third<L, I>(dA);
  return wmul<L, I>(drho * (T(1) + e) + rho0 * de);
}

// All q equilibrium deviations at (rho0 + drho, U + du).
template <class L, class T>
__host__ __device__ __forceinline__ void equilibrium_dev(T drho, T dux, T duy, T duz, T rho0,
                                                         T Ux, T Uy, T Uz, T (&g0)[L::Q]) {
  if constexpr (L::D == 2) {
    duz = T(0);
    Uz = T(0);
  }
  const T ux = Ux + dux, uy = Uy + duy, uz = Uz + duz;
  T A[7], dA[7];
  third_coeffs(ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, A, dA);
  const T usq = T(1.5) * (ux * ux + uy * uy + uz * uz);
  const T dusq = T(1.5) * (dux * (ux + Ux) + duy * (uy + Uy) + duz * (uz + Uz));
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    g0[i] = eq_dev_i<L, i>(drho, rho0, ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, usq, dusq, A, dA);
  });
}

// Reference state (rho0, U) of the shifted storage, in binary32, with the
// per-direction constants the equilibrium deviation needs:
// c1[i] = 1 + e_i(U) and cU2[i] = 2 xi_i.U (formed once on the host).
struct RefF {
  float rho0, Ux, Uy, Uz;
  float c1[27];
  float cU2[27];
};

// Equilibrium deviation of direction I from the deviations alone:
//   g0_i = w_i [ drho (1 + e_i(U)) + (rho0 + drho) (e_i(u) - e_i(U)) ],
//   e_i(u) - e_i(U) = 3 xi.du + 4.5 (xi.du)(2 xi.U + xi.du) - dusq + T3_i(dA),
// with dusq = 1.5 du.(2U + du) and dA the deviations of the third-order
// coefficients (third_coeffs).  MOV = false folds U = 0: c1 = 1, cU2 = 0,
// and the expression is the rest-state equilibrium w_i [drho + rho e_i(u)].
template <class L, int I, bool MOV>
__device__ __forceinline__ float eq_i(float drho, float rho, float dux, float duy, float duz,
                                      float dusq, const float (&dA)[7], const RefF& R) {
  const float cdu = cdot<L, I>(dux, duy, duz);
  const float cu2 = MOV ? R.cU2[I] : 0.0f;
  const float c1 = MOV ? R.c1[I] : 1.0f;
  const float de = 3.0f * cdu + 4.5f * cdu * (cu2 + cdu) - dusq + third<L, I>(dA);
  return wmul<L, I>(drho * c1 + rho * de);
}

// All q equilibrium deviations (binary32) at (rho0 + drho, U + du).
template <class L>
__device__ __forceinline__ void equilibrium_f(float drho, float dux, float duy, float duz,
                                              const RefF& R, float (&g0)[L::Q]) {
  const float Ux = R.Ux, Uy = R.Uy, Uz = (L::D == 3) ? R.Uz : 0.0f;
  if constexpr (L::D == 2) duz = 0.0f;
  const float ux = Ux + dux, uy = Uy + duy, uz = Uz + duz;
  float A[7], dA[7];
  third_coeffs(ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, A, dA);
  const float dusq = 1.5f * (dux * (ux + Ux) + duy * (uy + Uy) + duz * (uz + Uz));
  const float rho = R.rho0 + drho;
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    g0[i] = eq_i<L, i, true>(drho, rho, dux, duy, duz, dusq, dA, R);
  });
}

// Density and velocity deviations of shifted populations:
// drho = sum g, du = (sum xi g - drho U) / (rho0 + drho).
template <class L>
__device__ __forceinline__ void deviations(const float (&g)[L::Q], const RefF& R, float& drho,
                                           float& dux, float& duy, float& duz) {
  float jx, jy, jz;
  moments<L>(g, drho, jx, jy, jz);
  const float inv = 1.0f / (R.rho0 + drho);
  dux = (jx - drho * R.Ux) * inv;
  duy = (jy - drho * R.Uy) * inv;
  duz = (L::D == 3) ? (jz - drho * R.Uz) * inv : 0.0f;
}

// Strain-rate input of the hybrid collision (eq. a1ij_HRR):
// a1 <- sig a1 + ks rho S with ks = -2 tau cs^2 (1 - sig);
// s = (S_xx, S_yy, S_zz, S_xy, S_xz, S_yz).
struct HrrIn {
  float sig, ks;
  float s[6];
};

// Collision of shifted populations; the post-collision value of each
// direction is handed to emit(integral_constant<i>, value) as soon as it is
// formed, so no array of outputs (or of equilibria) stays live.
// COLL: 0 BGK (eq. BGKmodel), 1 REG (eq. LBMscheme_reg with H^(2) only),
// 2 RR (eqs. f1RR, a13RR), 3 H-RR (eq. a1ij_HRR, then the RR recursion;
// needs hy).  omega = 1 - 1/tau.
// MOV = false: the reference velocity is zero (rest-state shift) and every
// term in U is folded away at compile time.
template <class L, int COLL, bool MOV, class Emit>
__device__ __forceinline__ void collide_emit(const float (&g)[L::Q], float omega, const RefF& Rin,
                                             Emit&& emit, const HrrIn* hy = nullptr) {
  // (moments, deviations and the equilibrium of each direction)
  const float Ux = MOV ? Rin.Ux : 0.0f, Uy = MOV ? Rin.Uy : 0.0f,
              Uz = (MOV && L::D == 3) ? Rin.Uz : 0.0f, rho0 = Rin.rho0;
  float drho, jv[3], pd[3], po[3];
  moments2<L>(g, drho, jv, pd, po);
  const float jx = jv[0], jy = jv[1], jz = jv[2];
  const float rho = rho0 + drho;
  const float inv = __frcp_rn(rho);  // correctly rounded, as 1.0f / rho
  const float dux = (jx - drho * Ux) * inv, duy = (jy - drho * Uy) * inv,
              duz = (L::D == 3) ? (jz - drho * Uz) * inv : 0.0f;
  const float ux = Ux + dux, uy = Uy + duy, uz = Uz + duz;
  float Ae[7], dAe[7];
  third_coeffs(ux, uy, uz, dux, duy, duz, Ux, Uy, Uz, Ae, dAe);
  const float dusq = 1.5f * (dux * (ux + Ux) + duy * (uy + Uy) + duz * (uz + Uz));
  // Opposite directions share the even part of the equilibrium deviation
  // and of f^(1) and differ in the sign of the odd part:
  //   de_i = Ev + Od, de_opp(i) = Ev - Od,
  //   Ev = 4.5 (xi.du)(2 xi.U + xi.du) - dusq,  Od = 3 xi.du + T3_i(dA).
  // X_i such that g0_i = w_i X_i
  auto eq_pair = [&](auto I, float& xi, float& xj) {
    constexpr int i = decltype(I)::value;
    constexpr int j = opp<L>(i);
    const float cdu = cdot<L, i>(dux, duy, duz);
    const float cu2 = MOV ? Rin.cU2[i] : 0.0f;
    const float ev = 4.5f * cdu * (cu2 + cdu) - dusq;
    const float od = 3.0f * cdu + third<L, i>(dAe);
    const float c1i = MOV ? Rin.c1[i] : 1.0f, c1j = MOV ? Rin.c1[j] : 1.0f;
    xi = drho * c1i + rho * (ev + od);
    xj = drho * c1j + rho * (ev - od);
  };
  const float x00 = drho * (MOV ? Rin.c1[0] : 1.0f) - rho * dusq;  // rest direction
  constexpr int NP = (L::Q - 1) / 2;
  if constexpr (COLL == 0) {
    const float g00 = wmul<L, 0>(x00);
    emit(std::integral_constant<int, 0>{}, g00 + omega * (g[0] - g00));
    sfor<NP>([&](auto P) {
      constexpr int i = pair_first<L>(decltype(P)::value);
      constexpr int j = opp<L>(i);
      float xi, xj;
      eq_pair(std::integral_constant<int, i>{}, xi, xj);
      const float gi = wmul<L, i>(xi), gj = wmul<L, j>(xj);
      emit(std::integral_constant<int, i>{}, gi + omega * (g[i] - gi));
      emit(std::integral_constant<int, j>{}, gj + omega * (g[j] - gj));
    });
  } else {
    // second moments of the deviations g
    const float pxx = pd[0], pyy = pd[1], pzz = pd[2], pxy = po[0], pxz = po[1], pyz = po[2];
    // a1 = sum xi xi g - drho cs^2 I - drho u u - rho0 (u u - U U),
    // with u_a u_b - U_a U_b = du_a u_b + U_a du_b
    const float dc = drho * (1.0f / 3.0f);
    float axx, ayy, azz, axy, axz, ayz;
    if constexpr (MOV) {
      axx = pxx - dc - drho * ux * ux - rho0 * dux * (ux + Ux);
      ayy = pyy - dc - drho * uy * uy - rho0 * duy * (uy + Uy);
      azz = (L::D == 3) ? pzz - dc - drho * uz * uz - rho0 * duz * (uz + Uz) : 0.0f;
      axy = pxy - drho * ux * uy - rho0 * (dux * uy + Ux * duy);
      axz = (L::D == 3) ? pxz - drho * ux * uz - rho0 * (dux * uz + Ux * duz) : 0.0f;
      ayz = (L::D == 3) ? pyz - drho * uy * uz - rho0 * (duy * uz + Uy * duz) : 0.0f;
    } else {  // U = 0
      axx = pxx - rho * ux * ux - dc;
      ayy = pyy - rho * uy * uy - dc;
      azz = (L::D == 3) ? pzz - rho * uz * uz - dc : 0.0f;
      axy = pxy - rho * ux * uy;
      axz = (L::D == 3) ? pxz - rho * ux * uz : 0.0f;
      ayz = (L::D == 3) ? pyz - rho * uy * uz : 0.0f;
    }
    if constexpr (COLL == 3) {
      const float kr = hy->ks * rho;
      axx = hy->sig * axx + kr * hy->s[0];
      ayy = hy->sig * ayy + kr * hy->s[1];
      axy = hy->sig * axy + kr * hy->s[3];
      if constexpr (L::D == 3) {
        azz = hy->sig * azz + kr * hy->s[2];
        axz = hy->sig * axz + kr * hy->s[4];
        ayz = hy->sig * ayz + kr * hy->s[5];
      }
    }
    float A[7] = {0, 0, 0, 0, 0, 0, 0};
    if constexpr (COLL >= 2) {
      A[XXY] = 2.0f * ux * axy + uy * axx;
      A[YYX] = 2.0f * uy * axy + ux * ayy;
      if constexpr (L::D == 3) {
        A[XXZ] = 2.0f * ux * axz + uz * axx;
        A[YYZ] = 2.0f * uy * ayz + uz * ayy;
        A[ZZX] = 2.0f * uz * axz + ux * azz;
        A[ZZY] = 2.0f * uz * ayz + uy * azz;
        A[XYZ] = ux * ayz + uy * axz + uz * axy;
      }
    }
    // f^(1): 4.5 H2:a1 is even in xi (shared by a pair), T3(a1^(3)) is odd
    auto h2a_of = [&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
      constexpr float dxx = float(4.5 * (double(cx * cx) - 1.0 / 3.0));
      constexpr float dyy = float(4.5 * (double(cy * cy) - 1.0 / 3.0));
      constexpr float oxy = 9.0f * float(cx * cy);
      float h = dxx * axx + dyy * ayy + oxy * axy;
      if constexpr (L::D == 3) {
        constexpr float dzz = float(4.5 * (double(cz * cz) - 1.0 / 3.0));
        constexpr float oxz = 9.0f * float(cx * cz), oyz = 9.0f * float(cy * cz);
        h += dzz * azz + oxz * axz + oyz * ayz;
      }
      return h;
    };
    // post_i = w_i (X_i + omega F_i) with F_i = 4.5 H2_i:a1 + T3_i(a1^(3))
    emit(std::integral_constant<int, 0>{},
         wmul<L, 0>(x00 + omega * h2a_of(std::integral_constant<int, 0>{})));
    sfor<NP>([&](auto P) {
      constexpr int i = pair_first<L>(decltype(P)::value);
      constexpr int j = opp<L>(i);
      float xi, xj;
      eq_pair(std::integral_constant<int, i>{}, xi, xj);
      const float h = h2a_of(std::integral_constant<int, i>{});
      float t = 0.0f;
      if constexpr (COLL >= 2) t = third<L, i>(A);
      emit(std::integral_constant<int, i>{}, wmul<L, i>(xi + omega * (h + t)));
      emit(std::integral_constant<int, j>{}, wmul<L, j>(xj + omega * (h - t)));
    });
  }
}

// ------------------------------------------------------------ storage types
template <class S>
struct Store;
template <>
struct Store<float> {
  __device__ __forceinline__ static float ld(const float* p) { return *p; }
  __device__ __forceinline__ static float ldg(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
  __device__ __forceinline__ static void stcs(float* p, float v) { __stcs(p, v); }
};
template <>
struct Store<__half> {
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(*p); }
  __device__ __forceinline__ static float ldg(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ __forceinline__ static void stcs(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};

}  // namespace mlbm
