// Kernel instantiations for the D3Q19 lattice.
#include "ops_impl.cuh"

namespace mlbm {
template Ops make_ops<D3Q19>();
}  // namespace mlbm
