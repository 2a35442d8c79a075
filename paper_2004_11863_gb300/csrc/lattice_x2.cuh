// Two-lane binary32 collision: the collision of lattice.cuh for two
// independent population sets at once (the two runs of an interleaved pair,
// one per lane), on Blackwell's packed FP32 instructions (__fadd2_rn,
// __fmul2_rn, __ffma2_rn).  Every instruction acts on both lanes, so a node
// of a run pair issues about half the floating-point instructions of two
// scalar collisions.  Each lane is rounded to nearest like the scalar
// operations; sums of products are written as fused multiply-adds here, so a
// lane can differ from the scalar collision in the last bit.
//
// Same formulas as collide_emit (equilibrium deviation of eq. fEqH in the
// deviations drho, du; eq. BGKmodel; eq. LBMscheme_reg with H^(2) (REG) or
// with the recursion of eq. a13RR (RR)).
#pragma once
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace mlbm {

struct F2 {
  float2 v;
};
__device__ __forceinline__ F2 f2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
// a - b, one instruction: b * (-1) is exact, the sum is rounded once
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 operator*(float k, F2 a) { return f2(k) * a; }

// Compile-time masked sums: the sum of g[i] over the directions for which
// P::test<L, i>() holds, starting from the first such term (no addition of
// a zero); zero if there is none.
template <int A, int V>
struct AxisIs {
  template <class L, int I>
  __host__ __device__ static constexpr bool test() { return L::c(I, A) == V; }
};
template <int A, int B, int V>
struct ProdIs {
  template <class L, int I>
  __host__ __device__ static constexpr bool test() { return L::c(I, A) * L::c(I, B) == V; }
};
template <class L, class P, int I, bool HAS>
__device__ __forceinline__ F2 msum_impl(const F2 (&g)[L::Q], F2 acc) {
  if constexpr (I == L::Q) {
    if constexpr (HAS)
      return acc;
    else
      return f2(0.0f);
  } else if constexpr (P::template test<L, I>()) {
    if constexpr (HAS)
      return msum_impl<L, P, I + 1, true>(g, acc + g[I]);
    else
      return msum_impl<L, P, I + 1, true>(g, g[I]);
  } else {
    return msum_impl<L, P, I + 1, HAS>(g, acc);
  }
}
template <class L, class P>
__device__ __forceinline__ F2 msum(const F2 (&g)[L::Q]) {
  return msum_impl<L, P, 0, false>(g, f2(0.0f));
}

// xi_I . v for a direction with at least one component +1 (every
// pair_first direction of the three lattices): positive terms first, then
// the negative ones subtracted.
template <class L, int I>
__device__ __forceinline__ F2 cdot_x2(F2 vx, F2 vy, F2 vz) {
  static_assert(L::c(I, 0) == 1 || L::c(I, 1) == 1 || L::c(I, 2) == 1,
                "cdot_x2 needs a direction with a +1 component");
  const F2 v[3] = {vx, vy, vz};
  F2 s;
  bool has = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (L::c(I, a) == 1) {
      s = has ? s + v[a] : v[a];
      has = true;
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (L::c(I, a) == -1) s = s - v[a];
  return s;
}

// T3_I(A) with compile-time coefficients (same term sets as third<>).
template <class L, int I>
__device__ __forceinline__ F2 third_x2(const F2 (&A)[7]) {
  if constexpr (L::ID == 0) {
    constexpr float hxxy = float(13.5 * h3<L>(I, 0, 1)), hyyx = float(13.5 * h3<L>(I, 1, 0));
    return fma2(f2(hxxy), A[XXY], hyyx * A[YYX]);
  } else if constexpr (L::ID == 2) {
    constexpr float k0 = float(13.5 * h3<L>(I, 0, 1)), k1 = float(13.5 * h3<L>(I, 0, 2)),
                    k2 = float(13.5 * h3<L>(I, 1, 0)), k3 = float(13.5 * h3<L>(I, 1, 2)),
                    k4 = float(13.5 * h3<L>(I, 2, 0)), k5 = float(13.5 * h3<L>(I, 2, 1)),
                    k6 = float(27.0 * L::c(I, 0) * L::c(I, 1) * L::c(I, 2));
    F2 s = k0 * A[XXY];
    s = fma2(f2(k1), A[XXZ], s);
    s = fma2(f2(k2), A[YYX], s);
    s = fma2(f2(k3), A[YYZ], s);
    s = fma2(f2(k4), A[ZZX], s);
    s = fma2(f2(k5), A[ZZY], s);
    if constexpr (k6 != 0.0f) s = fma2(f2(k6), A[XYZ], s);
    return s;
  } else {
    constexpr float py = float(13.5 * (h3<L>(I, 0, 1) + h3<L>(I, 2, 1))),
                    my = float(4.5 * (h3<L>(I, 0, 1) - h3<L>(I, 2, 1)));
    constexpr float px = float(13.5 * (h3<L>(I, 1, 0) + h3<L>(I, 2, 0))),
                    mx = float(4.5 * (h3<L>(I, 1, 0) - h3<L>(I, 2, 0)));
    constexpr float pz = float(13.5 * (h3<L>(I, 0, 2) + h3<L>(I, 1, 2))),
                    mz = float(4.5 * (h3<L>(I, 0, 2) - h3<L>(I, 1, 2)));
    F2 s = py * (A[XXY] + A[ZZY]);
    s = fma2(f2(my), A[XXY] - A[ZZY], s);
    s = fma2(f2(px), A[YYX] + A[ZZX], s);
    s = fma2(f2(mx), A[YYX] - A[ZZX], s);
    s = fma2(f2(pz), A[XXZ] + A[YYZ], s);
    s = fma2(f2(mz), A[XXZ] - A[YYZ], s);
    return s;
  }
}

// w_I * x with the weight split into a binary32 head and tail (see wmul).
template <class L, int I>
__device__ __forceinline__ F2 wmul_x2(F2 x) {
  constexpr float hi = float(L::w(I));
  constexpr float lo = float(L::w(I) - double(hi));
  return fma2(f2(hi), x, lo * x);
}

// 4.5 H2_I : a1 with the zero coefficients dropped at compile time.
template <class L, int I>
__device__ __forceinline__ F2 h2a_x2(F2 axx, F2 ayy, F2 azz, F2 axy, F2 axz, F2 ayz) {
  constexpr int cx = L::c(I, 0), cy = L::c(I, 1), cz = L::c(I, 2);
  constexpr float dxx = float(4.5 * (double(cx * cx) - 1.0 / 3.0));
  constexpr float dyy = float(4.5 * (double(cy * cy) - 1.0 / 3.0));
  F2 h = fma2(f2(dyy), ayy, dxx * axx);
  if constexpr (cx * cy != 0) h = fma2(f2(9.0f * float(cx * cy)), axy, h);
  if constexpr (L::D == 3) {
    constexpr float dzz = float(4.5 * (double(cz * cz) - 1.0 / 3.0));
    h = fma2(f2(dzz), azz, h);
    if constexpr (cx * cz != 0) h = fma2(f2(9.0f * float(cx * cz)), axz, h);
    if constexpr (cy * cz != 0) h = fma2(f2(9.0f * float(cy * cz)), ayz, h);
  }
  return h;
}

// The collision of two population sets (lanes); emit(integral_constant<i>,
// F2 value) receives each post-collision direction of both lanes.
// COLL: 0 BGK, 1 REG, 2 RR.
template <class L, int COLL, bool MOV, class Emit>
__device__ __forceinline__ void collide_emit_x2(const F2 (&g)[L::Q], float omega, const RefF& R,
                                                Emit&& emit) {
  const F2 om = f2(omega);
  // moments from per-axis class sums
  const F2 spx = msum<L, AxisIs<0, 1>>(g), smx = msum<L, AxisIs<0, -1>>(g);
  const F2 spy = msum<L, AxisIs<1, 1>>(g), smy = msum<L, AxisIs<1, -1>>(g);
  const F2 s0 = msum<L, AxisIs<0, 0>>(g);
  const F2 drho = (spx + smx) + s0;
  const F2 jx = spx - smx, jy = spy - smy;
  F2 jz = f2(0.0f), spz = f2(0.0f), smz = f2(0.0f);
  if constexpr (L::D == 3) {
    spz = msum<L, AxisIs<2, 1>>(g);
    smz = msum<L, AxisIs<2, -1>>(g);
    jz = spz - smz;
  }
  const float rho0 = R.rho0;
  const F2 rho = f2(rho0) + drho;
  const F2 inv = {make_float2(__frcp_rn(rho.v.x), __frcp_rn(rho.v.y))};
  F2 dux, duy, duz = f2(0.0f), ux, uy, uz = f2(0.0f);
  const float Ux = MOV ? R.Ux : 0.0f, Uy = MOV ? R.Uy : 0.0f,
              Uz = (MOV && L::D == 3) ? R.Uz : 0.0f;
  if constexpr (MOV) {
    dux = fma2(drho, f2(-Ux), jx) * inv;
    duy = fma2(drho, f2(-Uy), jy) * inv;
    if constexpr (L::D == 3) duz = fma2(drho, f2(-Uz), jz) * inv;
    ux = f2(Ux) + dux;
    uy = f2(Uy) + duy;
    if constexpr (L::D == 3) uz = f2(Uz) + duz;
  } else {
    dux = jx * inv;
    duy = jy * inv;
    if constexpr (L::D == 3) duz = jz * inv;
    ux = dux;
    uy = duy;
    uz = duz;
  }
  // u + U (the sum the deviation formulas use)
  const F2 sx = MOV ? ux + f2(Ux) : ux, sy = MOV ? uy + f2(Uy) : uy;
  const F2 sz = (MOV && L::D == 3) ? uz + f2(Uz) : uz;
  // deviations of the third-order coefficients, dA = A(u) - A(U)
  F2 dA[7];
  if constexpr (MOV) {
    dA[XXY] = fma2(dux * sx, uy, (Ux * Ux) * duy);
    dA[YYX] = fma2(duy * sy, ux, (Uy * Uy) * dux);
    if constexpr (L::D == 3) {
      dA[XXZ] = fma2(dux * sx, uz, (Ux * Ux) * duz);
      dA[YYZ] = fma2(duy * sy, uz, (Uy * Uy) * duz);
      dA[ZZX] = fma2(duz * sz, ux, (Uz * Uz) * dux);
      dA[ZZY] = fma2(duz * sz, uy, (Uz * Uz) * duy);
      dA[XYZ] = fma2(dux * uy, uz, Ux * fma2(duy, uz, Uy * duz));
    }
  } else {
    dA[XXY] = (ux * ux) * uy;
    dA[YYX] = (uy * uy) * ux;
    if constexpr (L::D == 3) {
      dA[XXZ] = (ux * ux) * uz;
      dA[YYZ] = (uy * uy) * uz;
      dA[ZZX] = (uz * uz) * ux;
      dA[ZZY] = (uz * uz) * uy;
      dA[XYZ] = (ux * uy) * uz;
    }
  }
  F2 dsum = dux * sx;
  dsum = fma2(duy, sy, dsum);
  if constexpr (L::D == 3) dsum = fma2(duz, sz, dsum);
  const F2 ndusq = -1.5f * dsum;  // -dusq
  // X_i such that g0_i = w_i X_i, for both directions of a pair
  auto eq_pair = [&](auto I, F2& xi, F2& xj) {
    constexpr int i = decltype(I)::value;
    constexpr int j = opp<L>(i);
    const F2 cdu = cdot_x2<L, i>(dux, duy, duz);
    const F2 c45 = 4.5f * cdu;
    const F2 ev = MOV ? fma2(c45, f2(R.cU2[i]) + cdu, ndusq) : fma2(c45, cdu, ndusq);
    const F2 od = fma2(f2(3.0f), cdu, third_x2<L, i>(dA));
    if constexpr (MOV) {
      xi = fma2(drho, f2(R.c1[i]), rho * (ev + od));
      xj = fma2(drho, f2(R.c1[j]), rho * (ev - od));
    } else {
      xi = fma2(rho, ev + od, drho);
      xj = fma2(rho, ev - od, drho);
    }
  };
  const F2 x00 = MOV ? fma2(rho, ndusq, drho * f2(R.c1[0])) : fma2(rho, ndusq, drho);
  constexpr int NP = (L::Q - 1) / 2;
  if constexpr (COLL == 0) {
    const F2 g00 = wmul_x2<L, 0>(x00);
    emit(std::integral_constant<int, 0>{}, fma2(om, g[0] - g00, g00));
    sfor<NP>([&](auto P) {
      constexpr int i = pair_first<L>(decltype(P)::value);
      constexpr int j = opp<L>(i);
      F2 xi, xj;
      eq_pair(std::integral_constant<int, i>{}, xi, xj);
      const F2 gi = wmul_x2<L, i>(xi), gj = wmul_x2<L, j>(xj);
      emit(std::integral_constant<int, i>{}, fma2(om, g[i] - gi, gi));
      emit(std::integral_constant<int, j>{}, fma2(om, g[j] - gj, gj));
    });
  } else {
    // second moments of the deviations
    const F2 pxx = spx + smx, pyy = spy + smy;
    const F2 pxy = msum<L, ProdIs<0, 1, 1>>(g) - msum<L, ProdIs<0, 1, -1>>(g);
    F2 pzz = f2(0.0f), pxz = f2(0.0f), pyz = f2(0.0f);
    if constexpr (L::D == 3) {
      pzz = spz + smz;
      pxz = msum<L, ProdIs<0, 2, 1>>(g) - msum<L, ProdIs<0, 2, -1>>(g);
      pyz = msum<L, ProdIs<1, 2, 1>>(g) - msum<L, ProdIs<1, 2, -1>>(g);
    }
    const F2 dc = (1.0f / 3.0f) * drho;
    F2 axx, ayy, azz = f2(0.0f), axy, axz = f2(0.0f), ayz = f2(0.0f);
    if constexpr (MOV) {
      // a1 = P - drho cs^2 I - drho u u - rho0 (du u + U du)
      const F2 nr0 = f2(-rho0), ndr = f2(-1.0f) * drho;
      axx = fma2(nr0, dux * sx, fma2(ndr * ux, ux, pxx - dc));
      ayy = fma2(nr0, duy * sy, fma2(ndr * uy, uy, pyy - dc));
      axy = fma2(nr0, fma2(dux, uy, Ux * duy), fma2(ndr * ux, uy, pxy));
      if constexpr (L::D == 3) {
        azz = fma2(nr0, duz * sz, fma2(ndr * uz, uz, pzz - dc));
        axz = fma2(nr0, fma2(dux, uz, Ux * duz), fma2(ndr * ux, uz, pxz));
        ayz = fma2(nr0, fma2(duy, uz, Uy * duz), fma2(ndr * uy, uz, pyz));
      }
    } else {
      const F2 nrho = f2(-1.0f) * rho;
      axx = fma2(nrho * ux, ux, pxx) - dc;
      ayy = fma2(nrho * uy, uy, pyy) - dc;
      axy = fma2(nrho * ux, uy, pxy);
      if constexpr (L::D == 3) {
        azz = fma2(nrho * uz, uz, pzz) - dc;
        axz = fma2(nrho * ux, uz, pxz);
        ayz = fma2(nrho * uy, uz, pyz);
      }
    }
    F2 A[7];
    if constexpr (COLL == 2) {
      const F2 ux2 = 2.0f * ux, uy2 = 2.0f * uy;
      A[XXY] = fma2(ux2, axy, uy * axx);
      A[YYX] = fma2(uy2, axy, ux * ayy);
      if constexpr (L::D == 3) {
        const F2 uz2 = 2.0f * uz;
        A[XXZ] = fma2(ux2, axz, uz * axx);
        A[YYZ] = fma2(uy2, ayz, uz * ayy);
        A[ZZX] = fma2(uz2, axz, ux * azz);
        A[ZZY] = fma2(uz2, ayz, uy * azz);
        A[XYZ] = fma2(ux, ayz, fma2(uy, axz, uz * axy));
      }
    }
    emit(std::integral_constant<int, 0>{},
         wmul_x2<L, 0>(fma2(om, h2a_x2<L, 0>(axx, ayy, azz, axy, axz, ayz), x00)));
    sfor<NP>([&](auto P) {
      constexpr int i = pair_first<L>(decltype(P)::value);
      constexpr int j = opp<L>(i);
      F2 xi, xj;
      eq_pair(std::integral_constant<int, i>{}, xi, xj);
      const F2 h = h2a_x2<L, i>(axx, ayy, azz, axy, axz, ayz);
      if constexpr (COLL == 2) {
        const F2 t = third_x2<L, i>(A);
        emit(std::integral_constant<int, i>{}, wmul_x2<L, i>(fma2(om, h + t, xi)));
        emit(std::integral_constant<int, j>{}, wmul_x2<L, j>(fma2(om, h - t, xj)));
      } else {
        emit(std::integral_constant<int, i>{}, wmul_x2<L, i>(fma2(om, h, xi)));
        emit(std::integral_constant<int, j>{}, wmul_x2<L, j>(fma2(om, h, xj)));
      }
    });
  }
}

}  // namespace mlbm
