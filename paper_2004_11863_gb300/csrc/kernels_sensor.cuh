// Non-hydrodynamic mode sensors (Sec. 7), evaluated per iteration of a level
// from its pre-collision state, after the velocity pass (kernels_hrr.cuh)
// and before the level update:
//   spuriousAc (eq. sensorSpuriousAc): div u(t-1) * div u(t) < 0;
//   spuriousS (eq. sensorSpuriousS):  curl u(t-1) . curl u(t) < 0;
//     each only where both factors exceed eps in magnitude (the sign of a
//     round-off-level value is noise; eps = 0 is the literal test);
//   spuriousG (eq. sensorSpuriousG): |f1G| above a threshold and neither of
//     the others, f1G = f^(1) minus its second-order Hermite projection
//     w_i / (2 cs^4) H2_i : a1 (eqs. fneqSplit, reguProceduref1S).
// Gradients by second-order central differences of the velocity planes;
// evaluated at middle nodes only (not inactive, not TN, not on a refined
// level's outer layer), other nodes read as no flag and zero div / curl.
#pragma once
#include "kernels_hrr.cuh"

namespace mlbm {

// |f1G|^2 of shifted pre-collision populations.
template <class L>
__device__ __forceinline__ float ghost_norm2(const float (&g)[L::Q], const RefF& R) {
  float drho, dux, duy, duz, f1[L::Q];
  split_neq<L>(g, R, drho, dux, duy, duz, f1);
  float a[3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) a[p][q] = 0.0f;
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
#pragma unroll
    for (int p = 0; p < L::D; ++p)
#pragma unroll
      for (int q = 0; q < L::D; ++q)
        a[p][q] += float(L::c(i, p) * L::c(i, q) - (p == q ? 1.0 / 3.0 : 0.0)) * f1[i];
  });
  float n2 = 0.0f;
  sfor<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    float h = 0.0f;
#pragma unroll
    for (int p = 0; p < L::D; ++p)
#pragma unroll
      for (int q = 0; q < L::D; ++q)
        h += float(L::c(i, p) * L::c(i, q) - (p == q ? 1.0 / 3.0 : 0.0)) * a[p][q];
    const float d = f1[i] - wmul<L, i>(4.5f * h);
    n2 += d * d;
  });
  return n2;
}

template <class L, class S>
__global__ void k_sensors(LevelView v, const float* du, int par, SensorState st, RefF ref) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int run = blockIdx.y;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const NodeAddr a = node_addr<L>(v, x, y, z);
  const int e = a.at(0, 0, 0);
  float* dv = st.div + (long long)run * v.plane + e;
  float* cv = st.curl + (long long)run * st.nc * v.plane + e;
  unsigned char* fl = st.flag + (long long)run * v.plane + e;
  float* gp = st.gn + (long long)run * v.plane + e;
  const bool middle = !inactive(v, x, y, z) && !tn_node(v, x, y, z) && !outer_geom<L>(v, x, y, z);
  if (!middle) {
    *fl = 0;
    *gp = 0.0f;
    *dv = 0.0f;
    for (int c = 0; c < st.nc; ++c) cv[(long long)c * v.plane] = 0.0f;
    return;
  }
  const float* d = du + (long long)run * L::D * v.plane;
  float up[3][3] = {}, um[3][3] = {};
#pragma unroll
  for (int ax = 0; ax < L::D; ++ax) {
    const int ep = a.at(ax == 0, ax == 1, ax == 2), em = a.at(-(ax == 0), -(ax == 1), -(ax == 2));
#pragma unroll
    for (int b = 0; b < L::D; ++b) {
      up[ax][b] = d[(long long)b * v.plane + ep];
      um[ax][b] = d[(long long)b * v.plane + em];
    }
  }
  float gr[3][3];  // gr[a][b] = d_a u_b
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) gr[p][q] = 0.5f * (up[p][q] - um[p][q]);
  const float div = gr[0][0] + gr[1][1] + gr[2][2];
  float curl[3] = {gr[1][2] - gr[2][1], gr[2][0] - gr[0][2], gr[0][1] - gr[1][0]};
  // (2D: only the z component; it is stored as the single curl plane)
  float pc[3] = {0.0f, 0.0f, 0.0f}, cc[3] = {0.0f, 0.0f, 0.0f};
  if (st.nc == 1) {
    pc[2] = cv[0];
    cc[2] = curl[2];
  } else {
    for (int c = 0; c < 3; ++c) {
      pc[c] = cv[(long long)c * v.plane];
      cc[c] = curl[c];
    }
  }
  const float pdiv = *dv;
  const float np2 = pc[0] * pc[0] + pc[1] * pc[1] + pc[2] * pc[2];
  const float nc2 = cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2];
  const float e2 = st.eps * st.eps;
  const bool ac = pdiv * div < 0.0f && fabsf(pdiv) > st.eps && fabsf(div) > st.eps;
  const bool sh = pc[0] * cc[0] + pc[1] * cc[1] + pc[2] * cc[2] < 0.0f && np2 > e2 && nc2 > e2;
  const S* f = run_cptr<S>(v, run);
  float g[L::Q];
  load_pre<L, S>(f, v.plane, a, par, v.es, g);
  const float n2 = ghost_norm2<L>(g, ref);
  const bool gh = n2 > st.g2 && !ac && !sh;
  *fl = (unsigned char)((ac ? 1 : 0) | (sh ? 2 : 0) | (gh ? 4 : 0));
  *gp = sqrtf(n2);
  *dv = div;
  if (st.nc == 1) {
    cv[0] = curl[2];
  } else {
    for (int c = 0; c < 3; ++c) cv[(long long)c * v.plane] = curl[c];
  }
}

// Compact read-out of one run's sensor state: flags [N], div [N], curl
// [3][N] (z only in 2D) and |f1G| [N] in node order (x fastest).
template <class L>
__global__ void k_sensor_read(LevelView v, int run, SensorState st, unsigned char* flags,
                              double* div, double* curl, double* gnorm) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!node_of(v, t, x, y, z)) return;
  const long long N = (long long)v.n[0] * v.n[1] * v.n[2];
  const int e = node_addr<L>(v, x, y, z).at(0, 0, 0);
  flags[t] = st.flag[(long long)run * v.plane + e];
  div[t] = st.div[(long long)run * v.plane + e];
  gnorm[t] = st.gn[(long long)run * v.plane + e];
  for (int c = 0; c < 3; ++c) {
    float val = 0.0f;
    if (st.nc == 3)
      val = st.curl[((long long)run * 3 + c) * v.plane + e];
    else if (c == 2)
      val = st.curl[(long long)run * v.plane + e];
    curl[c * N + t] = val;
  }
}

}  // namespace mlbm
