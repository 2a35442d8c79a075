// Persistent fused step for the D2Q9 lattice.
#include "fused_impl.cuh"

namespace mlbm {
template size_t fused_tab_bytes<D2Q9>();
template cudaError_t fused_setup<D2Q9>(const FusedHost&, void*);
template int fused_max_blocks<D2Q9>(int);
template int fused_max_cluster<D2Q9>(int);
template cudaError_t fused_launch<D2Q9>(const FusedArgs&, int, int, cudaStream_t);
}  // namespace mlbm
