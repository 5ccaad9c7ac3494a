// Fused FP32 step, L1_0 (tetragonal three-shell) stencil instantiation.
#include "kernels_fused.cuh"

namespace hamr {

template cudaError_t launch_fused_lattice<true>(int, bool, const FusedArgs &, int, cudaStream_t);
template int fused_blocks_lattice<true>(int);

}  // namespace hamr
