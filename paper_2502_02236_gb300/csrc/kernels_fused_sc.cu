// Fused FP32 step, simple-cubic stencil instantiation, and the variant table.
#include "kernels_fused.cuh"

namespace hamr {

template cudaError_t launch_fused_lattice<false>(int, bool, const FusedArgs &, int, cudaStream_t);
template int fused_blocks_lattice<false>(int);
// the L1_0 instantiation lives in its own translation unit (compiled in parallel)
extern template cudaError_t launch_fused_lattice<true>(int, bool, const FusedArgs &, int, cudaStream_t);
extern template int fused_blocks_lattice<true>(int);

cudaError_t launch_fused_step(int v, bool tet, bool zr, const FusedArgs &a, int grid, cudaStream_t st) {
    return tet ? launch_fused_lattice<true>(v, zr, a, grid, st) : launch_fused_lattice<false>(v, zr, a, grid, st);
}

int fused_max_blocks_per_sm(int v, bool tet) { return tet ? fused_blocks_lattice<true>(v) : fused_blocks_lattice<false>(v); }

bool fused_variant(int v, FusedVariant &out) {
#define X(I, NT, E, SW, SH, MINB) \
    if (v == I) {                 \
        out.threads = NT;         \
        out.columns = NT * E;     \
        out.pitch = SW;           \
        out.rows = SH;            \
        out.staged = SW * SH;     \
        return true;              \
    }
    HAMR_FUSED_VARIANTS(X)
#undef X
    return false;
}

}  // namespace hamr
