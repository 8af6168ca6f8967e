// rsf_tiled_f16.cu -- instantiates the tiled iteration with FP16 storage of
// (a, b) (see rsf_tiled.cuh).
#include "rsf_tiled.cuh"

namespace rsf {
cudaError_t tiled_launch_f16(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    return tiled::launch_group_s<__half>(g, parity, prof, s);
}
cudaError_t tiled_prepare_f16(int R) { return tiled::prepare_group_s<__half>(R); }
}  // namespace rsf
