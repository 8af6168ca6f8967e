// rsf_tiled_f32.cu -- instantiates the tiled iteration with FP32 storage (see
// rsf_tiled.cuh), the storage-independent update kernel, the q set-up kernel
// and the host-side launch dispatch.
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "rsf_tiled.cuh"

namespace rsf {
namespace tiled {

namespace {
template <int R, class ImgT>
cudaError_t launch_bz_r(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    GroupArgs G{g.bricks, g.starts[3], g.nb, parity, g.err, g.fault_tx};
    ProfScope ps(prof, KID_TB_Z);
    Taps t = g.taps;
    if (R == 0) {  // the Eq. (15) form: one unit tap, no convolution of (a, b)
        t.R = 0;
        t.g[0] = 1.f;
    }
    if (g.dump)
        k_tb_z<R, ImgT, true><<<g.ncta[3], kZThreads, tbz_smem<R>(), s>>>(G, tap_pairs(t));
    else
        k_tb_z<R, ImgT><<<g.ncta[3], kZThreads, tbz_smem<R>(), s>>>(G, tap_pairs(t));
    return cudaGetLastError();
}
template <int R, bool DUMP>
cudaError_t prepare_bz_d() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_tb_z<R, uint8_t, DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tbz_smem<R>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tb_z<R, uint16_t, DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tbz_smem<R>())) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tb_z<R, float, DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tbz_smem<R>());
}
template <int R>
cudaError_t prepare_bz_i() {
    const cudaError_t e = prepare_bz_d<R, false>();
    return e != cudaSuccess ? e : prepare_bz_d<R, true>();
}
template <int R>
cudaError_t launch_bz_i(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    switch (g.imgtype) {
        case 0: return launch_bz_r<R, uint8_t>(g, parity, prof, s);
        case 1: return launch_bz_r<R, uint16_t>(g, parity, prof, s);
        default: return launch_bz_r<R, float>(g, parity, prof, s);
    }
}
__global__ void k_q_init(const float *__restrict__ phi, float *__restrict__ q, long long n, float eps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        q[i] = heaviside_q_fast(__ldg(phi + i), eps);
}
}  // namespace

cudaError_t prepare_tb_z(int R) {
    switch (R) {
        case 0: return prepare_bz_i<0>();
        case 2: return prepare_bz_i<2>();
        case 3: return prepare_bz_i<3>();
        case 4: return prepare_bz_i<4>();
        case 5: return prepare_bz_i<5>();
        case 6: return prepare_bz_i<6>();
        case 8: return prepare_bz_i<8>();
        case 10: return prepare_bz_i<10>();
        case 12: return prepare_bz_i<12>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tb_z(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    switch (g.force ? 0 : g.taps.R) {
        case 0: return launch_bz_i<0>(g, parity, prof, s);
        case 2: return launch_bz_i<2>(g, parity, prof, s);
        case 3: return launch_bz_i<3>(g, parity, prof, s);
        case 4: return launch_bz_i<4>(g, parity, prof, s);
        case 5: return launch_bz_i<5>(g, parity, prof, s);
        case 6: return launch_bz_i<6>(g, parity, prof, s);
        case 8: return launch_bz_i<8>(g, parity, prof, s);
        case 10: return launch_bz_i<10>(g, parity, prof, s);
        case 12: return launch_bz_i<12>(g, parity, prof, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tiled

bool tiled_supports(int R) {
    switch (R) {
        case 2: case 3: case 4: case 5: case 6: case 8: case 10: case 12: return true;
        default: return false;
    }
}

int tiled_pitch(int nx) { return (nx + tiled::kZX - 1) / tiled::kZX * tiled::kZX; }

bool tiled_fits(long long nx, long long ny, long long nz) {
    return (long long)tiled_pitch((int)nx) * ny * nz < (1LL << 32);
}

namespace {
// cuTensorMapEncodeTiled, reached through the runtime's driver entry point (no
// link against the driver library); null if the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The unit's rules for a 3-D tiled map: base 16-byte aligned, row and plane
// strides multiples of 16 bytes, boxes of 1..256 elements per dimension whose
// rows are a multiple of 16 bytes.
bool map_ok(const void *base, unsigned long long row_bytes, int bx, int by, int bz, int esize) {
    return base && reinterpret_cast<uintptr_t>(base) % 16 == 0 && row_bytes % 16 == 0 &&
           ((unsigned long long)bx * esize) % 16 == 0 && bx >= 1 && bx <= 256 && by >= 1 && by <= 256 && bz >= 1 &&
           bz <= 256;
}

// View [nz][ny][c nx] of a field of `type` elements (esize bytes) with c elements per
// voxel and a row pitch of c rx elements, read in boxes of bx x by x bz elements.
// Elements outside the view (columns < 0 or >= c nx, rows and planes likewise)
// arrive as zeros.
cudaError_t encode_typed(CUtensorMap *m, CUtensorMapDataType type, int esize, const void *base, int c, int rx,
                         const BrickDev &b, int bx, int by, int bz) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const unsigned long long row = (unsigned long long)esize * c * rx;
    if (!map_ok(base, row, bx, by, bz, esize)) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)c * b.nx, (cuuint64_t)b.ny, (cuuint64_t)b.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)row, (cuuint64_t)row * b.ny};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t elem[3] = {1u, 1u, 1u};
    const CUresult r = enc(m, type, 3, const_cast<void *>(base), dims, strides, box, elem,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// FP32 view [nz][ny][c nx] of a pitched field (row pitch c px floats).
cudaError_t encode_map(CUtensorMap *m, const void *base, int c, const BrickDev &b, int bx, int by, int bz) {
    return encode_typed(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, c, b.px, b, bx, by, bz);
}

// Group A's x/y staging maps (q[0], q[1], the image) of an even-radius brick when
// its unpitched rows allow them; b.xy_tma says whether they were made.
template <class ImgT>
cudaError_t encode_xy_stage(BrickDev &b, CUtensorMapDataType type, int R) {
    b.xy_tma = 0;
    switch (R) {
        case 2: case 4: case 6: case 8: case 10: case 12: break;
        default: return cudaSuccess;
    }
    // the same box geometry as the kernel's staging (XYStageH)
    const int H = 32 + 2 * R, RQ = (R + 3) / 4 * 4, AI = 16 / (int)sizeof(ImgT), RI = (R + AI - 1) / AI * AI;
    const int WQ = 32 + 2 * RQ, WI = 32 + 2 * RI;
    const unsigned long long qrow = 4ull * b.nx, irow = (unsigned long long)sizeof(ImgT) * b.nx;
    if (!map_ok(b.q[0], qrow, WQ, H, 1, 4) || !map_ok(b.q[1], qrow, WQ, H, 1, 4) ||
        !map_ok(b.img, irow, WI, H, 1, (int)sizeof(ImgT)))
        return cudaSuccess;  // not eligible: the register loaders serve this brick's group
    cudaError_t e = encode_typed(&b.tm_q[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.q[0], 1, b.nx, b, WQ, H, 1);
    if (e == cudaSuccess) e = encode_typed(&b.tm_q[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.q[1], 1, b.nx, b, WQ, H, 1);
    if (e == cudaSuccess)
        e = encode_typed(&b.tm_img, type, (int)sizeof(ImgT), b.img, 1, b.nx, b, WI, H, 1);
    if (e == cudaSuccess) b.xy_tma = 1;
    return e;
}
}  // namespace

cudaError_t tiled_encode_maps(BrickDev &b, int force, int storage, int imgtype, int R) {
    const int rows = tiled::kAZT + 2 * R;
    b.tm_k = CUtensorMap{};
    b.tm_ab = CUtensorMap{};
    b.tm_q[0] = b.tm_q[1] = b.tm_img = CUtensorMap{};
    b.xy_tma = 0;
    if (force == 1)  // the Eq. (15) form: four fields per voxel, no K*I~, no group B
        return encode_map(&b.tm_u, b.u2, 4, b, 128, 1, rows);
    cudaError_t e = encode_map(&b.tm_u, b.u2, 2, b, 64, 1, rows);
    if (e == cudaSuccess) e = encode_map(&b.tm_k, b.ki, 1, b, 32, 1, tiled::kAZT);
    if (e == cudaSuccess && storage == 0 && tiled::tbxy_tma(R))
        e = encode_map(&b.tm_ab, b.ab, 2, b, 2 * tiled_xy_in_pitch(R), 32 + 2 * R, 1);
    if (e == cudaSuccess) {
        switch (imgtype) {
            case 0: e = encode_xy_stage<uint8_t>(b, CU_TENSOR_MAP_DATA_TYPE_UINT8, R); break;
            case 1: e = encode_xy_stage<uint16_t>(b, CU_TENSOR_MAP_DATA_TYPE_UINT16, R); break;
            default: e = encode_xy_stage<float>(b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, R);
        }
    }
    return e;
}

cudaError_t tiled_q_init(const float *phi, float *q, long long n, float eps, cudaStream_t s) {
    tiled::k_q_init<<<1216, 256, 0, s>>>(phi, q, n, eps);
    return cudaGetLastError();
}

cudaError_t tiled_launch_f16(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s);
cudaError_t tiled_launch_bf16(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s);
cudaError_t tiled_prepare_f16(int R);
cudaError_t tiled_prepare_bf16(int R);

cudaError_t tiled_prepare_eq15(int R);
cudaError_t tiled_launch_eq15(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s);

cudaError_t tiled_prepare(int storage, int R, int force) {
    const cudaError_t e = tiled::prepare_tb_z(force ? 0 : R);
    if (e != cudaSuccess) return e;
    if (force) return tiled_prepare_eq15(R);  // FP32 intermediates whatever the storage option
    switch (storage) {
        case 0: return tiled::prepare_group_s<float>(R);
        case 1: return tiled_prepare_bf16(R);
        case 2: return tiled_prepare_f16(R);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tiled_iterate(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    if (g.force) return tiled_launch_eq15(g, parity, prof, s);
    switch (g.storage) {
        case 0: return tiled::launch_group_s<float>(g, parity, prof, s);
        case 1: return tiled_launch_bf16(g, parity, prof, s);
        case 2: return tiled_launch_f16(g, parity, prof, s);
        default: return cudaErrorInvalidValue;
    }
}

void tiled_cta_counts(const BrickDev &b, unsigned counts[4]) {
    const unsigned ntx = (b.nx + tiled::kXYT - 1) / tiled::kXYT, nty = (b.ny + tiled::kXYT - 1) / tiled::kXYT;
    const unsigned nzp = (b.nz + tiled::xy_planes(b) - 1) / tiled::xy_planes(b);
    counts[0] = ntx * nty * nzp;
    counts[1] = (unsigned)((b.nz + tiled::kAZT - 1) / tiled::kAZT) * ((b.nx + 31) / 32) * b.ny;
    counts[2] = counts[0];
    counts[3] = (unsigned)((b.nx + tiled::kZX - 1) / tiled::kZX) * ((b.ny + tiled::kZY - 1) / tiled::kZY) *
                ((b.nz + b.zc - 1) / b.zc);
}

// Per pitched voxel, Li's form: (H I~, H) 8 bytes, (a, b) 2 elements of the
// storage type, x/y-convolved (a, b) 8 bytes, K*I~ 4 bytes (24 or 28 bytes; np
// is even: every view is 8-byte aligned).  The Eq. (15) form: the two
// x/y-convolved pairs 16 bytes, the fits (f1, f2) 8 bytes (24 bytes, within
// the count for every storage type; no (a, b), no K*I~).
size_t tiled_stage_bytes(int storage, long long np) {
    const size_t e = storage == 0 ? 4 : 2;
    return (8 + 2 * e + 8 + 4) * (size_t)np;
}

void tiled_stage_views(int storage, int force, void *base, long long np, float2 **u2, void **ab, float2 **abxy,
                       float **ki) {
    char *p = static_cast<char *>(base);
    *u2 = reinterpret_cast<float2 *>(p);
    if (force) {
        *ab = nullptr;
        *abxy = reinterpret_cast<float2 *>(p + 16 * np);
        *ki = nullptr;
        return;
    }
    const size_t e = storage == 0 ? 4 : 2;
    *ab = p + 8 * np;
    *abxy = reinterpret_cast<float2 *>(p + (8 + 2 * e) * np);
    *ki = reinterpret_cast<float *>(p + (16 + 2 * e) * np);
}

namespace {
template <int R, class ImgT>
cudaError_t ki_init_r(const BrickDev &b, const Taps &taps, cudaStream_t s) {
    static_assert(tiled::XYLayout<R, 1>::bytes <= 48 * 1024, "k_ki_xy needs no shared-memory opt-in");
    const tiled::TapPairs tp = tiled::tap_pairs(taps);
    unsigned counts[4];
    tiled_cta_counts(b, counts);
    tiled::k_ki_xy<R, ImgT><<<counts[0], tiled::kXYThreads, tiled::XYLayout<R, 1>::bytes, s>>>(b, tp);
    tiled::k_ki_z<R><<<counts[1], tiled::kAZThreads, 0, s>>>(b, tp);
    return cudaGetLastError();
}
template <int R>
cudaError_t ki_init_i(const BrickDev &b, int imgtype, const Taps &taps, cudaStream_t s) {
    switch (imgtype) {
        case 0: return ki_init_r<R, uint8_t>(b, taps, s);
        case 1: return ki_init_r<R, uint16_t>(b, taps, s);
        default: return ki_init_r<R, float>(b, taps, s);
    }
}
}  // namespace

cudaError_t tiled_ki_init(const BrickDev &b, int imgtype, const Taps &taps, cudaStream_t s) {
    if (!b.ki) return cudaSuccess;  // the Eq. (15) form convolves the complement directly
    switch (taps.R) {
        case 2: return ki_init_i<2>(b, imgtype, taps, s);
        case 3: return ki_init_i<3>(b, imgtype, taps, s);
        case 4: return ki_init_i<4>(b, imgtype, taps, s);
        case 5: return ki_init_i<5>(b, imgtype, taps, s);
        case 6: return ki_init_i<6>(b, imgtype, taps, s);
        case 8: return ki_init_i<8>(b, imgtype, taps, s);
        case 10: return ki_init_i<10>(b, imgtype, taps, s);
        case 12: return ki_init_i<12>(b, imgtype, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rsf
