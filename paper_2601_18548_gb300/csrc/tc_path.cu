// BF16 tensor-core (tcgen05) fused GCDF kernel — placeholder until the kernel lands.
#include "gcdf_internal.cuh"

namespace gcdf {

int tc_tile_pairs() { return 128; }
bool tc_supported(int, int, int) { return false; }
size_t tc_slab_elems(int, int, int) { return 0; }
void tc_build_slabs(const float*, int, int, int, int, __nv_bfloat16*) {}
cudaError_t launch_tc(const WorkDesc&, const TcWeights&, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace gcdf
