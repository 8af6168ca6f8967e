// rsf_tiled_eq15.cu -- the tiled iteration of the paper's own data-term form,
// Eq. (15) with sigma_2 = 0 (Sec. 5.3): e_i = (I - f_i)^2, no group-B
// convolutions.  Group A convolves both sides of Eq. (10) directly, the pairs
// (H I~, H) and ((1-H) I~, 1-H), so that each fit is a ratio of two sums of
// non-negative weights (no difference of large convolved fields enters f2).
// Three launches per iteration: rsf_ta_xy (x/y, four fields), rsf_ta_z (z and
// the fits, FP32), rsf_tb_z (the update, with a unit tap over (f1, f2)).  The
// intermediates are FP32 whatever the context's storage option.
#include "rsf_tiled.cuh"

namespace rsf {
namespace tiled {
namespace {

template <int R>
int &az4_persist() {
    static int n = 152;
    return n;
}

template <int R>
cudaError_t prepare_eq15_r() {
    cudaError_t e;
    constexpr int sm = (int)xy_smem<R, 2>();
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, uint8_t, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
        cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, uint16_t, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
        cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
        cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ta_z4<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)az4_smem<R>())) !=
        cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ta_z4<R>, kAZThreads, az4_smem<R>())) !=
        cudaSuccess) return e;
    az4_persist<R>() = sms * (occ > 0 ? occ : 1);
    return cudaSuccess;
}

template <int R>
cudaError_t launch_eq15_r(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    GroupArgs G{g.bricks, nullptr, g.nb, parity, g.err, g.fault_tx};
    const TapPairs tp = tap_pairs(g.taps);
    {
        ProfScope ps(prof, KID_TA_XY);
        G.starts = g.starts[0];
        constexpr size_t sm = xy_smem<R, 2>();
        switch (g.imgtype) {
            case 0: k_ta_xy<R, uint8_t, 2><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp); break;
            case 1: k_ta_xy<R, uint16_t, 2><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp); break;
            default: k_ta_xy<R, float, 2><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp);
        }
    }
    {
        ProfScope ps(prof, KID_TA_Z);
        G.starts = g.starts[1];
        const unsigned grid = g.ncta[1] < (unsigned)az4_persist<R>() ? g.ncta[1] : (unsigned)az4_persist<R>();
        k_ta_z4<R><<<grid, kAZThreads, az4_smem<R>(), s>>>(G, tp);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tb_z(g, parity, prof, s);
}

}  // namespace
}  // namespace tiled

cudaError_t tiled_prepare_eq15(int R) {
    switch (R) {
        case 2: return tiled::prepare_eq15_r<2>();
        case 3: return tiled::prepare_eq15_r<3>();
        case 4: return tiled::prepare_eq15_r<4>();
        case 5: return tiled::prepare_eq15_r<5>();
        case 6: return tiled::prepare_eq15_r<6>();
        case 8: return tiled::prepare_eq15_r<8>();
        case 10: return tiled::prepare_eq15_r<10>();
        case 12: return tiled::prepare_eq15_r<12>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tiled_launch_eq15(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    switch (g.taps.R) {
        case 2: return tiled::launch_eq15_r<2>(g, parity, prof, s);
        case 3: return tiled::launch_eq15_r<3>(g, parity, prof, s);
        case 4: return tiled::launch_eq15_r<4>(g, parity, prof, s);
        case 5: return tiled::launch_eq15_r<5>(g, parity, prof, s);
        case 6: return tiled::launch_eq15_r<6>(g, parity, prof, s);
        case 8: return tiled::launch_eq15_r<8>(g, parity, prof, s);
        case 10: return tiled::launch_eq15_r<10>(g, parity, prof, s);
        case 12: return tiled::launch_eq15_r<12>(g, parity, prof, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rsf
