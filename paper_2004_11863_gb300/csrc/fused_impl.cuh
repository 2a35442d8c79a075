// Host side of the persistent fused step for one lattice (included by the
// three fused_<lattice>.cu translation units).
#pragma once
#include "kernels_fused.cuh"
#include "ops_impl.cuh"

namespace mlbm {

template <class L>
size_t fused_tab_bytes() {
  return sizeof(FusedTables);
}

template <class L>
cudaError_t fused_setup(const FusedHost& hst, void* d_tab) {
  FusedTables t{};
  for (int l = 0; l < kFusedLevels; ++l) {
    t.v[l] = hst.v[l];
    t.ring[l] = hst.ring[l];
    t.bnd[l] = hst.bnd[l];
    t.tn[l] = hst.tn[l];
  }
  t.ref = detail::make_ref_f<L>(hst.refd);
  t.refd = hst.refd;
  t.coll = hst.coll;
  t.probe_n = hst.probe_n;
  t.probe_cap = hst.probe_cap;
  t.probe_ijk = hst.probe_ijk;
  t.probe_rec = hst.probe_rec;
  t.probe_counter = hst.probe_counter;
  return cudaMemcpy(d_tab, &t, sizeof(t), cudaMemcpyHostToDevice);
}

template <class L>
int fused_max_blocks(int storage) {
  int per_sm = 0, dev = 0, sms = 0;
  const void* k = storage == 0 ? (const void*)k_fused<L, float> : (const void*)k_fused<L, __half>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFusedThreads, 0) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

// Largest cluster of fused-kernel blocks this device can place (at most 16:
// non-portable sizes above 8 are allowed), or 0.
template <class L>
int fused_max_cluster(int storage) {
  const void* k = storage == 0 ? (const void*)k_fused<L, float> : (const void*)k_fused<L, __half>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(kFusedThreads);
  cudaLaunchAttribute at{};
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 16;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&n, k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n < 16 ? n : 16;
}

template <class L>
cudaError_t fused_launch(const FusedArgs& A, int storage, int blocks, cudaStream_t s) {
  const void* k = storage == 0 ? (const void*)k_fused<L, float> : (const void*)k_fused<L, __half>;
  if (A.cluster) {  // one cluster of `blocks` blocks
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = blocks;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    if (storage == 0) return cudaLaunchKernelEx(&cfg, k_fused<L, float>, A);
    return cudaLaunchKernelEx(&cfg, k_fused<L, __half>, A);
  }
  void* args[] = {const_cast<FusedArgs*>(&A)};
  return cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(kFusedThreads), args, 0, s);
}

}  // namespace mlbm
