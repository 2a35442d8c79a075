// Persistent fused step for the D3Q27 lattice.
#include "fused_impl.cuh"

namespace mlbm {
template size_t fused_tab_bytes<D3Q27>();
template cudaError_t fused_setup<D3Q27>(const FusedHost&, void*);
template int fused_max_blocks<D3Q27>(int);
template int fused_max_cluster<D3Q27>(int);
template cudaError_t fused_launch<D3Q27>(const FusedArgs&, int, int, cudaStream_t);
}  // namespace mlbm
