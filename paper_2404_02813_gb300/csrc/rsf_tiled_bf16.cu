// rsf_tiled_bf16.cu -- instantiates the tiled iteration with BF16 storage of
// (a, b) (see rsf_tiled.cuh).
#include "rsf_tiled.cuh"

namespace rsf {
cudaError_t tiled_launch_bf16(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    return tiled::launch_group_s<__nv_bfloat16>(g, parity, prof, s);
}
cudaError_t tiled_prepare_bf16(int R) { return tiled::prepare_group_s<__nv_bfloat16>(R); }
}  // namespace rsf
