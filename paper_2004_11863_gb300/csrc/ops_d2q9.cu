// Kernel instantiations for the D2Q9 lattice.
#include "ops_impl.cuh"

namespace mlbm {
template Ops make_ops<D2Q9>();
}  // namespace mlbm
