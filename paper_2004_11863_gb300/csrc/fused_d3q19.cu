// Persistent fused step for the D3Q19 lattice.
#include "fused_impl.cuh"

namespace mlbm {
template size_t fused_tab_bytes<D3Q19>();
template cudaError_t fused_setup<D3Q19>(const FusedHost&, void*);
template int fused_max_blocks<D3Q19>(int);
template int fused_max_cluster<D3Q19>(int);
template cudaError_t fused_launch<D3Q19>(const FusedArgs&, int, int, cudaStream_t);
}  // namespace mlbm
