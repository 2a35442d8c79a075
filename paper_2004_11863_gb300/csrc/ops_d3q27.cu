// Kernel instantiations for the D3Q27 lattice.
#include "ops_impl.cuh"

namespace mlbm {
template Ops make_ops<D3Q27>();
}  // namespace mlbm
