// rsf_tiled.cuh -- the tiled four-kernel RSF iteration (arXiv 2404.02813,
// Sec. 3 and 4.2) over a table of bricks.
//
// A launch covers every brick of one group (same kernel radius R and image
// type); a plain volume is a group of one brick.  Each brick is an independent
// volume with its own boundaries, fields and scalars (the sub-volumes of the
// paper's volume-level parallelism, Sec. 4.1).  A CTA finds its brick by a
// binary search over the per-kernel CTA offsets of the group.
//
//   rsf_ta_xy  per z-plane, a 32x32 output tile plus an R halo in shared
//              memory: forms H I~ and H (Eqs. 6, 8-10) from the image
//              (centred on load; four columns per load where alignment
//              allows) and q = +-atan(eps/|phi|)/pi, convolves the pair along
//              x then y (packed f32x2 FMAs) and stores it (FP32).
//   rsf_ta_z   x-z slabs (32 columns x 64 output planes) staged in shared
//              memory by cp.async, two slabs in flight; z convolution over a
//              register window; the local fits f1 = K*(H I~)/K*H and
//              f2 = K*((1-H) I~)/K*(1-H), the latter from the linearity of the
//              convolution as (K*I~ - K*(H I~)) / (K*1 - K*H) with K*I~ fixed
//              for the solve (rsf_ki_xy / rsf_ki_z, once) and K*1 the product of
//              the three 1-D zero-padding profiles; a = l1 f1 - l2 f2,
//              b = l1 f1^2 - l2 f2^2 (stored FP32, FP16 or BF16).
//   rsf_tb_xy  the x/y kernel on (a, b); its output stays FP32 (the data term
//              below is a difference of terms much larger than itself).
//   rsf_tb_z   a z march over a 32x8 column tile: a register ring of (a, b)
//              planes, a phi ring and a unit-normal ring in shared memory
//              (each normal computed once per tile position, not per use);
//              g = s^2 [ (l1 - l2) K1 I~^2 - 2 I~ K*a + K*b ]  (Eqs. 11-12),
//              kappa and the Laplacian (Eqs. 3-4), the update of Eqs. (1),
//              (13), (14), and q of the new phi for the next rsf_ta_xy.
//
// Convolutions use zero padding, taps summed k = -R..R, FP32 accumulation;
// finite differences use reflect-101 for phi and for the normal.  The
// intermediate fields are stored with an x pitch rounded up to 32 columns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "rsf_internal.h"

namespace rsf {
namespace tiled {

constexpr int kXYT = 32;          // x/y kernel: output tile edge (x and y)
constexpr int kXYThreads = 256;   // 8 warps
// z-planes per CTA of the x/y kernel: BrickDev::xyp (tuned per brick group), kDefaultXYPlanes by default
__host__ __device__ __forceinline__ int xy_planes(const BrickDev &B) { return B.xyp > 0 ? B.xyp : kDefaultXYPlanes; }
constexpr int kZX = 32, kZY = 8;  // z march: columns per CTA
constexpr int kZThreads = kZX * kZY;
constexpr int kAZT = 64;          // x-z slab: output planes per CTA
constexpr int kAZThreads = 256;
constexpr int kAZO = kAZT / (kAZThreads / 32);
constexpr int kPFB = 2;           // (a, b) planes loaded ahead in the z march

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The taps of Eq. (7) duplicated into (g_k, g_k) pairs, passed by value: the
// first operand of a packed f32x2 FMA over a field pair, read from the
// kernel's parameter space.
struct TapPairs {
    float2 g[2 * RMAX + 1];
};
inline TapPairs tap_pairs(const Taps &t) {
    TapPairs p{};
    for (int k = 0; k <= 2 * t.R; ++k) p.g[k] = make_float2(t.g[k], t.g[k]);
    return p;
}
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------------- storage

template <class S> struct Store;
template <> struct Store<float> {
    using V4 = float4;
    using V2 = float2;
    __device__ __forceinline__ static V4 pack4(float4 v) { return v; }
    __device__ __forceinline__ static float4 unpack4(V4 v) { return v; }
    __device__ __forceinline__ static V2 pack2(float2 v) { return v; }
    __device__ __forceinline__ static float2 unpack2(V2 v) { return v; }
};
template <> struct Store<__half> {
    using V4 = uint2;
    using V2 = uint32_t;
    __device__ __forceinline__ static uint32_t p(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static float2 u(uint32_t w) { return __half22float2(*reinterpret_cast<__half2 *>(&w)); }
    __device__ __forceinline__ static V4 pack4(float4 v) { return make_uint2(p(v.x, v.y), p(v.z, v.w)); }
    __device__ __forceinline__ static float4 unpack4(V4 v) {
        const float2 a = u(v.x), b = u(v.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static V2 pack2(float2 v) { return p(v.x, v.y); }
    __device__ __forceinline__ static float2 unpack2(V2 v) { return u(v); }
};
template <> struct Store<__nv_bfloat16> {
    using V4 = uint2;
    using V2 = uint32_t;
    __device__ __forceinline__ static uint32_t p(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static float2 u(uint32_t w) {
        return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w));
    }
    __device__ __forceinline__ static V4 pack4(float4 v) { return make_uint2(p(v.x, v.y), p(v.z, v.w)); }
    __device__ __forceinline__ static float4 unpack4(V4 v) {
        const float2 a = u(v.x), b = u(v.y);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static V2 pack2(float2 v) { return p(v.x, v.y); }
    __device__ __forceinline__ static float2 unpack2(V2 v) { return u(v); }
};

// Image value, centred and scaled on load: (I - m) / s = I * (1/s) + (-m/s),
// one rounding (1/s is a power of two), the same value the centring kernel stores.
template <class T>
__device__ __forceinline__ float centred(const T *img, long long p, float inv_s, float nms) {
    return fmaf((float)__ldg(img + p), inv_s, nms);
}

// ------------------------------------------------------------ brick table

__device__ __forceinline__ int find_brick(const int *__restrict__ starts, int nb, int cta) {
    int lo = 0, hi = nb;  // starts[lo] <= cta < starts[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(starts + mid) <= cta) lo = mid; else hi = mid;
    }
    return lo;
}

struct GroupArgs {
    const BrickDev *bricks;
    const int *starts;  // nb + 1 CTA offsets of this kernel within the launch
    int nb;
    int parity;         // launch parity: a brick reads phi[p], q[p] with p = parity ^ flip, writes the other
    int *err;           // the group's error word (bounded waits), may be null
    unsigned fault_tx;  // extra bytes the TMA barriers expect (0; > 0 only in a fault test)
};

// ---- TMA tile copies completing on shared-memory mbarriers (PTX ISA: mbarrier,
// cp.async.bulk.tensor).  One thread arms a barrier with the bytes it expects and
// issues the copies; every thread waits for the phase to complete, for at most
// kWaitNs (then the kernel reports through the group's error word).
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes initialised barriers visible to the other threads and to the copy unit
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// one arrival that also raises the phase's expected transaction count by `bytes`
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// waits for the completion of the barrier's phase of the given parity until the
// global timer passes `deadline`; false if it did not complete by then
__device__ __forceinline__ bool mbar_wait_until(uint64_t *bar, unsigned parity, unsigned long long deadline) {
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() > deadline) return false;
    return true;
}
// the same for at most kWaitNs from the first failed try (the timer is read only then)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_until(bar, parity, globaltimer_ns() + kWaitNs);
}
// orders this thread's earlier generic-proxy accesses to shared memory before
// later copies of the async proxy (the copy unit) into it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// The tensor map at `map` in global memory as it is now (the host rewrites the
// descriptor array between launches, perhaps over maps the copy unit has seen).
__device__ __forceinline__ void fence_tensormap(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}
// 3-D tile load of the box at element coordinates (x, y, z) of `map` into `dst`
// (128-byte aligned), completing `bytes of the box` on `bar`.  x times the
// element size must be a multiple of 16 bytes; y and z may lie outside the
// tensor (those elements arrive as zeros).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
// records an error in the group's error word (mapped host memory), once per CTA
__device__ __forceinline__ void report_error(int *err, int code) {
    if (err && threadIdx.x == 0) {
        *reinterpret_cast<volatile int *>(err) = code;
        __threadfence_system();
    }
}

// ---------------------------------------------------------------- x / y

// A producer of the x/y kernel's input pairs: plane(off) gives the plane at
// element offset `off`, fetch(plane, o) the raw values at offset o within it,
// apply() the NP float2 pairs (zero outside the brick).
template <class ImgT>
struct ProH {  // (H I~, H) from q and the centred image
    const float *q;
    const ImgT *img;
    float inv_s, nms;
    struct Raw { float q, im; };
    struct Plane { const float *q; const ImgT *img; };
    __device__ __forceinline__ Plane plane(long long off) const { return Plane{q + off, img + off}; }
    __device__ __forceinline__ Raw fetch(const Plane &pl, int o) const {
        return Raw{__ldg(pl.q + o), fmaf((float)__ldg(pl.img + o), inv_s, nms)};
    }
    __device__ __forceinline__ Raw zero() const { return Raw{0.f, 0.f}; }
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        const float h = h_of_q(r.q);
        v[0] = inside ? make_float2(h * r.im, h) : make_float2(0.f, 0.f);
    }
};

template <class ImgT>
struct ProH2 : ProH<ImgT> {  // (H I~, H) and ((1-H) I~, 1-H): both sides of Eq. (10) for the Eq. (15) form
    using typename ProH<ImgT>::Raw;
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        const float h = h_of_q(r.q), hc = hc_of_q(r.q);
        v[0] = inside ? make_float2(h * r.im, h) : make_float2(0.f, 0.f);
        v[1] = inside ? make_float2(hc * r.im, hc) : make_float2(0.f, 0.f);
    }
};

template <class ImgT>
struct ProI {  // (I~, 0): the centred image alone, for K*I~
    const ImgT *img;
    float inv_s, nms;
    using Raw = float;
    struct Plane { const ImgT *img; };
    __device__ __forceinline__ Plane plane(long long off) const { return Plane{img + off}; }
    __device__ __forceinline__ Raw fetch(const Plane &pl, int o) const {
        return fmaf((float)__ldg(pl.img + o), inv_s, nms);
    }
    __device__ __forceinline__ Raw zero() const { return 0.f; }
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        v[0] = make_float2(inside ? r : 0.f, 0.f);
    }
};

template <class S>
struct ProAB {  // (a, b) as stored by rsf_ta_z (pitched)
    const typename Store<S>::V2 *ab;
    using Raw = typename Store<S>::V2;
    struct Plane { const typename Store<S>::V2 *ab; };
    __device__ __forceinline__ Plane plane(long long off) const { return Plane{ab + off}; }
    __device__ __forceinline__ Raw fetch(const Plane &pl, int o) const { return __ldg(pl.ab + o); }
    __device__ __forceinline__ Raw zero() const { return Raw{}; }
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        v[0] = inside ? Store<S>::unpack2(r) : make_float2(0.f, 0.f);
    }
};

// Shared-memory layout of the x/y kernel (float2 units): the input tile of NP
// pairs and the x-convolved rows of XCP pairs (NP, or 1 when the pairs pass
// through the x and y convolutions one after the other).
template <int R, int NP, int XCP = NP>
struct XYLayout {
    static constexpr int W = kXYT + 2 * R;              // loaded width
    static constexpr int H = kXYT + 2 * R;              // loaded rows
    // row pitch = 2 (mod 16) float2: rows start 16-byte aligned, and the x pass's
    // 16-byte window reads (an 8-lane phase covers 2 rows x 4 column groups 8 floats
    // apart, or 4 rows x 2 groups 16 floats apart) hit distinct banks
    static constexpr int P = tiled_xy_in_pitch(R);
    static_assert(P == ((W + 15) / 16) * 16 + 2, "input tile pitch");
    static constexpr int IN = NP * H * P;               // input tile
    // x-convolved rows, room for a row pitch of up to 34 (XYCfg)
    static constexpr int XC = XCP * H * (kXYT + 2);
    static constexpr size_t bytes = sizeof(float2) * (IN + XC);
};

// Resident CTAs per SM the x/y kernels are compiled for: 3 (4 for rsf_ta_xy at
// radius <= 6) measured faster than 2 at radii 8-12 in spite of a few spilled words.

// Loads the x/y kernel's input tile of one plane entry by entry (any row
// pitch): entry e of this thread has its offset within the plane (-1 outside
// the brick) and its shared-memory index; entries e < NFULL always lie inside
// the tile.  fetch(z) issues the global loads of plane z into registers,
// store(in) writes the NP pairs into the tile.
template <int R, int NP, class Pro>
struct ScalarLoader {
    using L = XYLayout<R, NP>;
    using Raw = typename Pro::Raw;
    static constexpr int NE = (L::H * L::W + kXYThreads - 1) / kXYThreads;
    static constexpr int NFULL = L::H * L::W / kXYThreads;
    static_assert(NE <= 32, "too many tile entries per thread");
    const Pro &pro;
    long long iplane;
    int eoff[NE], esm[NE];
    Raw raw[NE];
    __device__ __forceinline__ ScalarLoader(const Pro &p, int nx, int ny, int ipx, int x0, int y0)
        : pro(p), iplane((long long)ipx * ny) {
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int i = threadIdx.x + e * kXYThreads;
            const int ii = min(i, L::H * L::W - 1);
            const int ly = ii / L::W, lx = ii - ly * L::W;
            const int gx = x0 + lx - R, gy = y0 + ly - R;
            const bool in_vol = i < L::H * L::W && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
            eoff[e] = in_vol ? gy * ipx + gx : -1;
            esm[e] = i < L::H * L::W ? ly * L::P + lx : -1;
        }
    }
    __device__ __forceinline__ void fetch(int z) {
        const auto pl = pro.plane((long long)z * iplane);
#pragma unroll
        for (int e = 0; e < NE; ++e) raw[e] = eoff[e] >= 0 ? pro.fetch(pl, eoff[e]) : pro.zero();
    }
    __device__ __forceinline__ void store(float2 *in) const {
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            if (e < NFULL || esm[e] >= 0) {
                float2 v[NP];
                pro.apply(raw[e], eoff[e] >= 0, v);
#pragma unroll
                for (int p = 0; p < NP; ++p) in[p * L::H * L::P + esm[e]] = v[p];
            }
        }
    }
};

// The same tile of (H I~, H) loaded four columns at a time: one 16-byte load
// of q and one load of four image values per group, window columns
// [x0 - RA, x0 + 32 + RA) with RA = R rounded up to a multiple of 4.  Needs an
// even R <= 8 (used for R <= 6) and a row pitch (= nx) that is a multiple of 4, so that a group
// lies wholly inside or wholly outside the brick and its pairs of columns are
// 16-byte aligned in the tile (two 16-byte shared stores per group).
template <class T> struct Vec4;
template <> struct Vec4<uint8_t> { using V = uchar4; };
template <> struct Vec4<uint16_t> { using V = ushort4; };
template <> struct Vec4<float> { using V = float4; };

template <int R, class ImgT, int NP = 1>
struct VecLoaderH {  // NP = 1: (H I~, H); NP = 2: also ((1-H) I~, 1-H) (the Eq. (15) form)
    using L = XYLayout<R, NP>;
    static_assert(R % 2 == 0 && R <= 8, "even radius <= 8");
    static constexpr int RA = (R + 3) / 4 * 4;
    static constexpr int NG = (32 + 2 * RA) / 4;                       // groups per row
    static constexpr int NV = (L::H * NG + kXYThreads - 1) / kXYThreads;  // groups per thread
    using V = typename Vec4<ImgT>::V;
    const float *q;
    const ImgT *img;
    float inv_s, nms;
    long long iplane;
    int goff[NV];  // group offset in the plane (-1: outside the brick)
    int sm0[NV];   // tile index of the group's first column (may lie left of the tile)
    int lx0[NV];   // tile column of the group's first column; kNone: no group for this thread
    static constexpr int kNone = -1 << 20;
    float4 rq[NV];
    V ri[NV];
    __device__ __forceinline__ VecLoaderH(const float *q_, const ImgT *img_, float inv_s_, float nms_, int nx, int ny,
                                          int x0, int y0)
        : q(q_), img(img_), inv_s(inv_s_), nms(nms_), iplane((long long)nx * ny) {
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const int i = threadIdx.x + e * kXYThreads;
            const int ii = min(i, L::H * NG - 1);
            const int row = ii / NG, g = ii - row * NG;
            const int gy = y0 + row - R, gx = x0 - RA + 4 * g;
            const bool in_vol = i < L::H * NG && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
            goff[e] = in_vol ? gy * nx + gx : -1;
            sm0[e] = row * L::P + 4 * g - RA + R;
            lx0[e] = i < L::H * NG ? 4 * g - RA + R : kNone;
        }
    }
    __device__ __forceinline__ void fetch(int z) {
        const float *qp = q + (long long)z * iplane;
        const ImgT *ip = img + (long long)z * iplane;
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            if (goff[e] >= 0) {
                rq[e] = __ldg(reinterpret_cast<const float4 *>(qp + goff[e]));
                ri[e] = __ldg(reinterpret_cast<const V *>(ip + goff[e]));
            } else {
                rq[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                ri[e] = V{};
            }
        }
    }
    // two adjacent columns (q, image value) of each input pair into the tile at index c
    __device__ __forceinline__ void put(float2 *in, int c, float qa, float ia, float qb, float ib, bool inside) const {
        const float ha = h_of_q(qa), hb = h_of_q(qb);
        const float xa = fmaf(ia, inv_s, nms), xb = fmaf(ib, inv_s, nms);
        *reinterpret_cast<float4 *>(in + c) =
            inside ? make_float4(ha * xa, ha, hb * xb, hb) : make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (NP == 2) {
            const float ca = hc_of_q(qa), cb = hc_of_q(qb);
            *reinterpret_cast<float4 *>(in + L::H * L::P + c) =
                inside ? make_float4(ca * xa, ca, cb * xb, cb) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __device__ __forceinline__ void store(float2 *in) const {
#pragma unroll
        for (int e = 0; e < NV; ++e) {
            const int c0 = sm0[e], lx = lx0[e];
            const bool inside = goff[e] >= 0;
            if (lx >= 0 && lx + 1 < L::W) put(in, c0, rq[e].x, (float)ri[e].x, rq[e].y, (float)ri[e].y, inside);
            if (lx != kNone && lx + 2 >= 0 && lx + 3 < L::W)
                put(in, c0 + 2, rq[e].z, (float)ri[e].z, rq[e].w, (float)ri[e].w, inside);
        }
    }
};

// The x/y kernel body for one CTA of one brick: planes [za, za + np) of
// tile (x0, y0).  The global loads of plane z+1 are issued right after the
// first barrier of plane z and land in registers while the convolutions run.
// `Out` writes the NP pairs (pitch out.px).
// Two pairs pass through the x and y convolutions one after the other (one
// pair of x-convolved rows in shared memory) where that lets three CTAs share
// an SM: radius >= 10.
template <int R, int NP>
constexpr bool xy_seq() { return NP == 2 && R >= 10; }
template <int R, int NP>
constexpr size_t xy_smem() { return XYLayout<R, NP, xy_seq<R, NP>() ? 1 : NP>::bytes; }

// x phase of the x/y kernel: XT outputs per thread and the row pitch XS of the
// x-convolved rows.  XT = 8: items of 8 rows x 32 columns, each 8-lane phase of
// a 16-byte window read covering 4 rows x 2 column groups, stores of two outputs
// (16 bytes) at pitch 34, so that both fall on distinct banks (37 % fewer
// shared-load wavefronts than XT = 4 at radius 6).  XT = 4 in the single-pair
// (H I~, H) kernel, whose loader keeps more registers live (XT = 8 measured no
// faster there): items of 8 rows x 16 columns, 64-bit stores at pitch 33 (rows
// r..r+3 of a half-warp, four columns apart, on 32 distinct banks; a pitch of 32
// puts 8 rows on one bank set), pitch 32 at radius >= 10 (measured 8 % faster:
// its schedule under the 80-register cap differs).
template <int R, int NP, bool HLOAD>
struct XYCfg {
    static constexpr bool H1 = HLOAD && NP == 1;
    static constexpr int XT = H1 ? 4 : 8;
    static constexpr int XS = XT == 8 ? kXYT + 2 : (R >= 10 ? kXYT : kXYT + 1);
};

// x then y convolution of plane z of the input tile `in` (NP pairs, row pitch
// L::P) through the x-convolved rows `xc`, written by `out`; ends with a barrier
// (both tiles are free again).
template <int R, int NP, class Cfg, class Out>
__device__ __forceinline__ void xy_plane(const float2 *in, float2 *xc, const Out &out, int z, int nx, int ny,
                                         int x0, int y0, const TapPairs &t) {
    constexpr bool SEQ = xy_seq<R, NP>();
    constexpr int NPX = SEQ ? 1 : NP;        // pairs per x/y round
    using L = XYLayout<R, NP, NPX>;
    constexpr int T = 2 * R + 1;
    constexpr int XT = Cfg::XT, XS = Cfg::XS, YT = 4;  // outputs per thread in the x and y phases; pitch
    static_assert((XT == 4 && XS <= kXYT + 1) || (XT == 8 && XS == kXYT + 2), "x phase layout");
    constexpr int NRB = (L::H + 7) / 8;      // 8-row blocks of the x phase
    constexpr int NCB = kXYT / (4 * XT);     // column blocks of an item row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int ps = 0; ps < NP / NPX; ++ps) {  // rounds of NPX pairs (one round unless SEQ)
    {
        const int h = lane >> 4;
        const int r = XT == 8 ? (lane >> 1) & 3 : (lane >> 2) & 3;
        const int g = XT == 8 ? (lane & 1) | ((lane >> 2) & 2) : lane & 3;
        // items (8 rows x 4 XT columns of one pair) dealt to the warps round-robin; at radius
        // <= 6 and for two pairs a warp's items warp + 8 i run in a compile-time number of
        // rounds (measured faster there; slower at radius 8 with one pair)
        constexpr int NITEMS = NPX * NRB * NCB, NW8 = kXYThreads / 32;
        constexpr bool STATIC = R <= 6 || NP == 2;
        constexpr int NROUNDS = STATIC ? (NITEMS + NW8 - 1) / NW8 : 1;
#pragma unroll
        for (int i = 0; i < NROUNDS; ++i)
        for (int item = warp + NW8 * i; item < NITEMS; item += STATIC ? NITEMS : NW8) {
            const int pl = item / (NRB * NCB);  // pair within the round
            const int p = SEQ ? ps : pl;         // pair of the input tile
            const int rem = item - pl * NRB * NCB;
            const int row = (rem / NCB) * 8 + h * 4 + r;
            const int xo = (rem % NCB) * 16 + g * XT;
            if (row < L::H) {
                const float4 *src = reinterpret_cast<const float4 *>(in + (p * L::H + row) * L::P + xo);
                // streamed: each loaded pair feeds the outputs it contributes to
                // (output o takes taps k = 0..T-1 in order, as a window would)
                float2 acc[XT];
#pragma unroll
                for (int o = 0; o < XT; ++o) acc[o] = make_float2(0.f, 0.f);
#pragma unroll
                for (int j2 = 0; j2 < (XT + 2 * R) / 2; ++j2) {
                    const float4 q = src[j2];
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int j = 2 * j2 + h2;
                        const float2 v = h2 ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
#pragma unroll
                        for (int o = 0; o < XT; ++o)
                            if (j - o >= 0 && j - o < T) acc[o] = f2fma(t.g[j - o], v, acc[o]);
                    }
                }
                float2 *dst = xc + (pl * L::H + row) * XS + xo;
                if constexpr (XT == 8) {
#pragma unroll
                    for (int o = 0; o < XT; o += 2)
                        *reinterpret_cast<float4 *>(dst + o) =
                            make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
                } else {
#pragma unroll
                    for (int o = 0; o < XT; ++o) dst[o] = acc[o];
                }
            }
        }
    }
    __syncthreads();
    {
        const int gx = x0 + lane;
        float2 res[NPX][YT];
#pragma unroll
        for (int p = 0; p < NPX; ++p) {
#pragma unroll
            for (int o = 0; o < YT; ++o) res[p][o] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < YT + 2 * R; ++j) {
                const float2 v = xc[(p * L::H + warp * YT + j) * XS + lane];
#pragma unroll
                for (int o = 0; o < YT; ++o)
                    if (j - o >= 0 && j - o < T) res[p][o] = f2fma(t.g[j - o], v, res[p][o]);
            }
        }
        if (gx < nx) {
            const int gy0 = y0 + warp * YT;
            const auto op = out.plane(z);
#pragma unroll
            for (int o = 0; o < YT; ++o) {
                if (gy0 + o < ny) {
                    if constexpr (SEQ)
                        out.half(op, (gy0 + o) * out.px + gx, ps, res[0][o]);
                    else
                        out(op, (gy0 + o) * out.px + gx, res[0][o], res[NPX - 1][o]);
                }
            }
        }
    }
    __syncthreads();  // the next round or plane reuses the tiles
    }
}

template <int R, int NP, class Cfg, class Loader, class Out>
__device__ __forceinline__ void xy_tile(Loader &ld, const Out &out, int nx, int ny, int nz, int x0, int y0, int za,
                                        int np, const TapPairs &t, float2 *sm) {
    using L = XYLayout<R, NP, xy_seq<R, NP>() ? 1 : NP>;
    float2 *in = sm;
    float2 *xc = sm + L::IN;
    const int zb_end = min(za + np, nz);
    ld.fetch(za);
    for (int z = za; z < zb_end; ++z) {
        ld.store(in);
        __syncthreads();
        if (z + 1 < zb_end) ld.fetch(z + 1);
        xy_plane<R, NP, Cfg>(in, xc, out, z, nx, ny, x0, y0, t);
    }
}

// Writers of the x/y kernel's outputs: plane(z) gives plane z, operator()
// stores at offset y * px + x within it.
struct OutF2 {  // one x/y-convolved pair, FP32, pitched
    float2 *u;
    int px;
    long long pplane;
    __device__ __forceinline__ float2 *plane(int z) const { return u + (long long)z * pplane; }
    __device__ __forceinline__ void operator()(float2 *pl, int o, float2 a, float2) const { pl[o] = a; }
};

struct OutF4 {  // two x/y-convolved pairs interleaved per voxel (16 bytes), FP32, pitched
    float4 *u;
    int px;
    long long pplane;
    __device__ __forceinline__ float4 *plane(int z) const { return u + (long long)z * pplane; }
    __device__ __forceinline__ void operator()(float4 *pl, int o, float2 a, float2 b) const {
        pl[o] = make_float4(a.x, a.y, b.x, b.y);
    }
    // pair p alone (the pairs convolved one after the other): its half of the voxel's 16 bytes
    __device__ __forceinline__ void half(float4 *pl, int o, int p, float2 v) const {
        reinterpret_cast<float2 *>(pl + o)[p] = v;
    }
};

// CTA -> (brick, tile) for the x/y kernels: tiles (tx, ty, tz) of 32 x 32 x xy_planes(B).
struct XYTile {
    int b, x0, y0, za;
};
__device__ __forceinline__ XYTile xy_tile_of(const GroupArgs &G, const BrickDev &B, int b) {
    const int local = blockIdx.x - __ldg(G.starts + b);
    const int ntx = (B.nx + kXYT - 1) / kXYT, nty = (B.ny + kXYT - 1) / kXYT;
    const int tx = local % ntx, r = local / ntx;
    return XYTile{b, tx * kXYT, (r % nty) * kXYT, (r / nty) * xy_planes(B)};
}

// NP = 1: (H I~, H) into B.u2 (Li's form); NP = 2: both sides of Eq. (10),
// ((H I~, H), ((1-H) I~, 1-H)) interleaved per voxel into B.u2 read as float4
// (the Eq. (15) form, which convolves the complement directly).
template <int R, class ImgT, int NP = 1>
__global__ void __launch_bounds__(kXYThreads, NP == 1 ? (R <= 6 ? 4 : 3) : (R <= 8 || xy_seq<R, NP>() ? 3 : 2))
    k_ta_xy(GroupArgs G, TapPairs t) {
    extern __shared__ float2 sm[];
    const int b = find_brick(G.starts, G.nb, blockIdx.x);
    const BrickDev B = G.bricks[b];
    const XYTile tl = xy_tile_of(G, B, b);
    const float inv_s = B.cs[1], nms = -B.cs[0] * B.cs[1];
    const float *q = (G.parity ^ B.flip) ? B.q[1] : B.q[0];
    const ImgT *img = reinterpret_cast<const ImgT *>(B.img);
    using Out = typename std::conditional<NP == 1, OutF2, OutF4>::type;
    using OutV = typename std::conditional<NP == 1, float2, float4>::type;
    const Out out{reinterpret_cast<OutV *>(B.u2), B.px, (long long)B.px * B.ny};
    if constexpr (R % 2 == 0 && R <= 6) {
        // four columns per load where the row pitch and both base addresses allow it (uniform per CTA);
        // at radius 8 the second code path cost more registers than the loads saved (measured)
        if (B.nx % 4 == 0 && reinterpret_cast<uintptr_t>(q) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(img) % (4 * sizeof(ImgT)) == 0) {
            VecLoaderH<R, ImgT, NP> ld(q, img, inv_s, nms, B.nx, B.ny, tl.x0, tl.y0);
            xy_tile<R, NP, XYCfg<R, NP, true>>(ld, out, B.nx, B.ny, B.nz, tl.x0, tl.y0, tl.za, xy_planes(B), t, sm);
            return;
        }
    }
    using Pro = typename std::conditional<NP == 1, ProH<ImgT>, ProH2<ImgT>>::type;
    Pro pro{};
    pro.q = q;
    pro.img = img;
    pro.inv_s = inv_s;
    pro.nms = nms;
    ScalarLoader<R, NP, Pro> ld(pro, B.nx, B.ny, B.nx, tl.x0, tl.y0);
    xy_tile<R, NP, XYCfg<R, NP, true>>(ld, out, B.nx, B.ny, B.nz, tl.x0, tl.y0, tl.za, xy_planes(B), t, sm);
}

// Group A's x/y kernel of Li's form with its inputs copied by TMA (even radius;
// used for a brick group whose bricks all have q and image rows of a multiple of
// 16 bytes and aligned bases): per plane one box of q and one of the image land
// in a staging buffer, each starting at the 16-byte aligned column at or left of
// x0 - R; a transform pass writes (H I~, H) of the tile from it, two columns per
// step, zero outside the brick (the copies' zero fill would give H = 1 there),
// with the arithmetic of the register loaders; the next plane's boxes are then in
// flight while the tile is convolved.
template <int R, class ImgT>
struct XYStageH {
    static_assert(R % 2 == 0, "even radius: the staged columns' offsets are even");
    static constexpr int H = kXYT + 2 * R, W = kXYT + 2 * R;
    static constexpr int RQ = (R + 3) / 4 * 4;                              // q: 4 floats per 16 bytes
    static constexpr int AI = 16 / (int)sizeof(ImgT);                       // image values per 16 bytes
    static constexpr int RI = (R + AI - 1) / AI * AI;
    static constexpr int WQ = kXYT + 2 * RQ, WI = kXYT + 2 * RI;            // box widths (elements)
    static constexpr int QB = WQ * H * 4, IB = WI * H * (int)sizeof(ImgT);  // box bytes
    static constexpr int IOFF = (QB + 127) / 128 * 128;                     // image box offset (bytes)
    static constexpr int BYTES = IOFF + (IB + 127) / 128 * 128;             // staging bytes
    using L = XYLayout<R, 1>;
    static constexpr size_t smem = BYTES + sizeof(float2) * (L::IN + L::XC) + sizeof(uint64_t);
};
template <class T> struct Pair2;
template <> struct Pair2<uint8_t> { using V = uchar2; };
template <> struct Pair2<uint16_t> { using V = ushort2; };
template <> struct Pair2<float> { using V = float2; };

template <int R, class ImgT>
__global__ void __launch_bounds__(kXYThreads, R <= 6 ? 4 : 3) k_ta_xy_tma(GroupArgs G, TapPairs t) {
    using S = XYStageH<R, ImgT>;
    using L = XYLayout<R, 1>;
    extern __shared__ __align__(128) unsigned char xsm[];
    const float *sq = reinterpret_cast<const float *>(xsm);
    const ImgT *simg = reinterpret_cast<const ImgT *>(xsm + S::IOFF);
    float2 *tile = reinterpret_cast<float2 *>(xsm + S::BYTES);
    float2 *xc = tile + L::IN;
    uint64_t *bar = reinterpret_cast<uint64_t *>(xc + L::XC);
    const int b = find_brick(G.starts, G.nb, blockIdx.x);
    const BrickDev &B = G.bricks[b];
    const XYTile tl = xy_tile_of(G, B, b);
    const int nx = B.nx, ny = B.ny, nz = B.nz, x0 = tl.x0, y0 = tl.y0, za = tl.za;
    const float inv_s = B.cs[1], nms = -B.cs[0] * B.cs[1];
    const CUtensorMap *mq = (G.parity ^ B.flip) ? &B.tm_q[1] : &B.tm_q[0];
    const CUtensorMap *mi = &B.tm_img;
    const OutF2 out{B.u2, B.px, (long long)B.px * ny};
    const int zb_end = min(za + xy_planes(B), nz);
    if (smem_addr(xsm) % 128u != 0u) {
        report_error(G.err, kErrSmemAlign);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const auto issue = [&](int z) {
        mbar_arrive_expect_tx(bar, (unsigned)(S::QB + S::IB) + G.fault_tx);
        tma_load_3d(xsm, mq, x0 - S::RQ, y0 - R, z, bar);
        tma_load_3d(xsm + S::IOFF, mi, x0 - S::RI, y0 - R, z, bar);
    };
    bool pending = false;
    if (za < zb_end) {
        if (threadIdx.x == 0) {
            fence_tensormap(mq);
            fence_tensormap(mi);
            issue(za);
        }
        pending = true;
    }
    unsigned phase = 0u;
    bool ok = true;
    for (int z = za; z < zb_end; ++z) {
        if (!mbar_wait(bar, phase)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        pending = false;
        constexpr int NPAIRS = S::H * S::W / 2, W2 = S::W / 2;
#pragma unroll
        for (int k = 0; k < (NPAIRS + kXYThreads - 1) / kXYThreads; ++k) {
            const int i = threadIdx.x + k * kXYThreads;
            if (i < NPAIRS) {
                const int row = i / W2, col = 2 * (i - row * W2);
                const float2 qv = *reinterpret_cast<const float2 *>(sq + row * S::WQ + col + (S::RQ - R));
                const typename Pair2<ImgT>::V iv =
                    *reinterpret_cast<const typename Pair2<ImgT>::V *>(simg + row * S::WI + col + (S::RI - R));
                const int gx = x0 - R + col, gy = y0 - R + row;
                const bool iny = (unsigned)gy < (unsigned)ny;
                const bool in0 = iny && (unsigned)gx < (unsigned)nx, in1 = iny && (unsigned)(gx + 1) < (unsigned)nx;
                const float h0 = h_of_q(qv.x), h1 = h_of_q(qv.y);
                const float v0 = fmaf((float)iv.x, inv_s, nms), v1 = fmaf((float)iv.y, inv_s, nms);
                *reinterpret_cast<float4 *>(tile + row * L::P + col) =
                    make_float4(in0 ? h0 * v0 : 0.f, in0 ? h0 : 0.f, in1 ? h1 * v1 : 0.f, in1 ? h1 : 0.f);
            }
        }
        __syncthreads();  // the staging buffer is consumed, the tile complete
        if (z + 1 < zb_end) {
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                issue(z + 1);
            }
            pending = true;
        }
        xy_plane<R, 1, XYCfg<R, 1, true>>(tile, xc, out, z, nx, ny, x0, y0, t);
    }
    if (!ok) {
        report_error(G.err, kErrWaitExpired);
        if (pending) mbar_wait_until(bar, phase, globaltimer_ns() + kWaitNs);
        return;
    }
    if (threadIdx.x == 0) mbar_inval(bar);
}

// Group B's x/y kernel takes its FP32 (a, b) tile from TMA at even radius: the box's
// x origin, 2 (x0 - R) floats, is then 16-byte aligned.
constexpr bool tbxy_tma(int R) { return R % 2 == 0; }

// The single-pair x/y kernel body with the input tile copied by TMA: one box per
// plane, H rows x P pairs of an FP32 pair field from (x0 - R, y0 - R) -- zeros
// outside the brick, exactly the convolutions' padding, and the tile's own row
// pitch, so the x phase reads it as it is.  Two tile stages: plane z + 1 is in
// flight while plane z is convolved.  Shared memory: the stages (each rounded up
// to 128 bytes), the x-convolved rows, two mbarriers.  Waits are bounded as in
// the z pass (expiry reported in the group's error word).
template <int R>
struct XYTma {
    using L = XYLayout<R, 1>;
    static constexpr int STAGE = (L::IN + 15) / 16 * 16;  // float2 units, a multiple of 128 bytes
    static constexpr size_t bytes = sizeof(float2) * (2 * STAGE + L::XC) + 2 * sizeof(uint64_t);
};

template <int R, class Cfg, class Out>
__device__ __forceinline__ void xy_tile_tma(const GroupArgs &G, const CUtensorMap *map, const Out &out, int nx, int ny,
                                            int nz, int x0, int y0, int za, int np, const TapPairs &t, float2 *sm) {
    using L = XYLayout<R, 1>;
    constexpr int STAGE = XYTma<R>::STAGE;
    constexpr unsigned BOX = sizeof(float2) * L::IN;  // bytes of one plane's box
    float2 *xc = sm + 2 * STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(xc + L::XC);
    if (smem_addr(sm) % 128u != 0u) {
        report_error(G.err, kErrSmemAlign);
        return;
    }
    const int zb_end = min(za + np, nz);
    if (threadIdx.x == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const auto issue = [&](int z, int st) {
        mbar_arrive_expect_tx(bars + st, BOX + G.fault_tx);
        tma_load_3d(sm + st * STAGE, map, 2 * (x0 - R), y0 - R, z, bars + st);
    };
    unsigned phase = 0u, pending = 0u;  // bit s: parity of stage s's next phase; stage s awaits its copy
    if (za < zb_end) {
        if (threadIdx.x == 0) {
            fence_tensormap(map);
            issue(za, 0);
        }
        pending = 1u;
    }
    bool ok = true;
    for (int z = za; z < zb_end; ++z) {
        const int st = (z - za) & 1;
        if (z + 1 < zb_end) {  // the other stage was last read by plane z - 1's x phase, before a barrier
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                issue(z + 1, st ^ 1);
            }
            pending |= 1u << (st ^ 1);
        }
        if (!mbar_wait(bars + st, (phase >> st) & 1u)) {
            ok = false;
            break;
        }
        phase ^= 1u << st;
        pending &= ~(1u << st);
        xy_plane<R, 1, Cfg>(sm + st * STAGE, xc, out, z, nx, ny, x0, y0, t);
    }
    if (!ok) {
        report_error(G.err, kErrWaitExpired);
        const unsigned long long deadline = globaltimer_ns() + kWaitNs;
        for (int b = 0; b < 2; ++b)
            if ((pending >> b) & 1u) mbar_wait_until(bars + b, (phase >> b) & 1u, deadline);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_inval(bars);
        mbar_inval(bars + 1);
    }
}

// Dynamic shared memory of group B's x/y kernel for storage S.
template <int R, class S>
constexpr size_t tbxy_smem() {
    return std::is_same<S, float>::value && tbxy_tma(R) ? XYTma<R>::bytes : XYLayout<R, 1>::bytes;
}

template <int R, class S>
__global__ void __launch_bounds__(kXYThreads, 3) k_tb_xy(GroupArgs G, TapPairs t) {
    extern __shared__ __align__(128) float2 sm[];
    const int b = find_brick(G.starts, G.nb, blockIdx.x);
    const BrickDev B = G.bricks[b];
    const XYTile tl = xy_tile_of(G, B, b);
    OutF2 out{B.abxy, B.px, (long long)B.px * B.ny};
    if constexpr (std::is_same<S, float>::value && tbxy_tma(R)) {
        xy_tile_tma<R, XYCfg<R, 1, false>>(G, &G.bricks[b].tm_ab, out, B.nx, B.ny, B.nz, tl.x0, tl.y0, tl.za,
                                           xy_planes(B), t, sm);
    } else {
        ProAB<S> pro{reinterpret_cast<const typename Store<S>::V2 *>(B.ab)};
        ScalarLoader<R, 1, ProAB<S>> ld(pro, B.nx, B.ny, B.px, tl.x0, tl.y0);
        xy_tile<R, 1, XYCfg<R, 1, false>>(ld, out, B.nx, B.ny, B.nz, tl.x0, tl.y0, tl.za, xy_planes(B), t, sm);
    }
}

// ------------------------------------------------------------------ A: z

// x-z slabs: 32 columns of one y row and kAZT output planes (plus the R-plane
// halos) of the x/y-convolved pair (H I~, H), and the kAZT planes of K*I~ the
// slab's outputs use.  A persistent CTA walks the slabs of the launch
// (consecutive slabs are consecutive z ranges of one row, so shared halos hit
// L2) with a two-stage shared-memory buffer: the cp.async copies of the next
// slab are in flight while the current one is convolved.  Rows outside the
// brick are zero-filled by the copy (source size 0).
template <int R>
constexpr int az_stage() { return (kAZT + 2 * R) * 32 + kAZT * 16; }  // float2 units per stage
template <int R>
constexpr size_t az_smem() { return 2 * sizeof(float2) * az_stage<R>() + 2 * sizeof(uint64_t); }  // + barriers

__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }


struct AZSlabId {
    int b, x0, y, z0;
};
// n / d and n % d for n >= 0, d > 0.  Below 2^24 a float quotient, off by at
// most one, corrected once; larger n (very thin bricks only) divide exactly.
__device__ __forceinline__ int divmod24(int n, int d, float inv_d, int &rem) {
    if (n >= (1 << 24)) {
        const int q = n / d;
        rem = n - q * d;
        return q;
    }
    int q = __float2int_rz((float)n * inv_d);
    int r = n - q * d;
    if (r < 0) { --q; r += d; } else if (r >= d) { ++q; r -= d; }
    rem = r;
    return q;
}
__device__ __forceinline__ AZSlabId az_slab_of(const GroupArgs &G, int slab) {
    const int b = find_brick(G.starts, G.nb, slab);
    const BrickDev &B = G.bricks[b];
    const int local = slab - __ldg(G.starts + b);
    const int nzt = (B.nz + kAZT - 1) / kAZT, nxt = (B.nx + 31) / 32;
    int zt, xt;
    const int rest = divmod24(local, nzt, __frcp_rn((float)nzt), zt);
    const int y = divmod24(rest, nxt, __frcp_rn((float)nxt), xt);
    return AZSlabId{b, xt * 32, y, zt * kAZT};
}

// The persistent slab walk of group A's z kernels: each CTA takes the slabs
// blockIdx.x, blockIdx.x + gridDim.x, ... of the launch through two stage
// buffers of STAGE_BYTES in dynamic shared memory, followed by one mbarrier per
// stage.  Thread 0 issues a slab's TMA copies (issue(id, buf, bar)) one slab
// ahead, into the stage the previous slab left; every thread waits for its
// stage's barrier, then body(id, buf) convolves the slab.  The last argument of
// issue asks it to fence the brick's tensor maps (first slab of each brick).  A wait that runs out
// (kWaitNs) is reported in the group's error word; the CTA then gives the copies
// still in flight the same time to land and returns.
template <int STAGE_BYTES, class Issue, class Body>
__device__ __forceinline__ void az_walk(const GroupArgs &G, unsigned char *smem, const Issue &issue,
                                        const Body &body) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * STAGE_BYTES);
    if (smem_addr(smem) % 128u != 0u) {  // the copies' destinations must be 128-byte aligned
        report_error(G.err, kErrSmemAlign);
        return;
    }
    const int total = __ldg(G.starts + G.nb);
    if (threadIdx.x == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned phase = 0u, pending = 0u;  // bit s: parity of stage s's next phase; stage s awaits copies
    AZSlabId next{};
    int last_b = -1;  // thread 0: the brick whose maps it fenced last
    if ((int)blockIdx.x < total) {
        next = az_slab_of(G, blockIdx.x);
        if (threadIdx.x == 0) {
            issue(next, smem, bars, true);
            last_b = next.b;
        }
        pending = 1u;
    }
    int stage = 0;
    bool ok = true;
    for (int sl = blockIdx.x; sl < total; sl += gridDim.x) {
        const AZSlabId id = next;
        if (sl + (int)gridDim.x < total) {
            next = az_slab_of(G, sl + gridDim.x);
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();  // the reads of that stage (before the last barrier) come first
                issue(next, smem + (stage ^ 1) * STAGE_BYTES, bars + (stage ^ 1), next.b != last_b);
                last_b = next.b;
            }
            pending |= 1u << (stage ^ 1);
        }
        if (!mbar_wait(bars + stage, (phase >> stage) & 1u)) {
            ok = false;
            break;
        }
        phase ^= 1u << stage;
        pending &= ~(1u << stage);
        body(id, smem + stage * STAGE_BYTES);
        __syncthreads();  // this stage is refilled by the next iteration's copies
        stage ^= 1;
    }
    if (!ok) {
        report_error(G.err, kErrWaitExpired);
        const unsigned long long deadline = globaltimer_ns() + kWaitNs;
        for (int s = 0; s < 2; ++s)
            if ((pending >> s) & 1u) mbar_wait_until(bars + s, (phase >> s) & 1u, deadline);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_inval(bars);
        mbar_inval(bars + 1);
    }
}

template <int R, class S>
__global__ void __launch_bounds__(kAZThreads, R <= 6 ? 3 : 2) k_ta_z(GroupArgs G, TapPairs t) {
    constexpr int T = 2 * R + 1;
    constexpr int ROWS = kAZT + 2 * R;
    constexpr int WIN = kAZO + 2 * R;
    constexpr int STAGE_BYTES = (int)sizeof(float2) * az_stage<R>();
    using V2 = typename Store<S>::V2;
    // [2 stages]{[ROWS][32] pairs, [kAZT][32] K*I~}, then the two barriers
    extern __shared__ __align__(128) unsigned char az_sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the slab's boxes: ROWS planes of the pair field from plane z0 - R, kAZT planes of K*I~
    // from z0 (planes outside the brick and columns past nx arrive as zeros)
    const auto issue = [&](const AZSlabId &id, unsigned char *buf, uint64_t *bar, bool fence) {
        const BrickDev &B = G.bricks[id.b];
        if (fence) {
            fence_tensormap(&B.tm_u);
            fence_tensormap(&B.tm_k);
        }
        mbar_arrive_expect_tx(bar, (unsigned)STAGE_BYTES + G.fault_tx);
        tma_load_3d(buf, &B.tm_u, 2 * id.x0, id.y, id.z0 - R, bar);
        tma_load_3d(buf + ROWS * 32 * sizeof(float2), &B.tm_k, id.x0, id.y, id.z0, bar);
    };
    const auto body = [&](const AZSlabId &id, const unsigned char *sbuf) {
        const float2 *buf = reinterpret_cast<const float2 *>(sbuf);
        const BrickDev &B = G.bricks[id.b];
        const int x = id.x0 + lane;
        const int zb = warp * kAZO;
        const int bnx = B.nx, bny = B.ny, bnz = B.nz;  // read once: the stores below might alias B
        if (x >= bnx) return;
        const float l1 = B.lambda1, l2 = B.lambda2;
        float2 w[WIN];
#pragma unroll
        for (int j = 0; j < WIN; ++j) w[j] = buf[(zb + j) * 32 + lane];
        const long long pplane = (long long)B.px * bny;
        const long long off = (long long)(id.z0 + zb) * pplane + (long long)id.y * B.px + x;
        V2 *ab = reinterpret_cast<V2 *>(B.ab) + off;
        const float *ki = reinterpret_cast<const float *>(buf + ROWS * 32) + zb * 32 + lane;
        const float kxy = __ldg(B.prof + x) * __ldg(B.prof + bnx + id.y);
        float2 res = make_float2(0.f, 0.f);  // rounding residual carried along z (16-bit storage)
        const float *pz = B.prof + bnx + bny + id.z0 + zb;
        float *const dump = B.dump;
#pragma unroll
        for (int o = 0; o < kAZO; ++o) {
            const int zo = id.z0 + zb + o;
            if (zo < bnz) {
                float2 acc = make_float2(0.f, 0.f);  // (K*(H I~), K*H)
#pragma unroll
                for (int k = 0; k < T; ++k) acc = f2fma(t.g[k], w[o + k], acc);
                const float f1 = __fdividef(acc.x, acc.y);
                // K*(1-H) = K*1 - K*H keeps few significant bits once 1-H < ~1e-6 over the
                // whole window (phi > ~3e5 there, delta < 4e-12); the fit is then taken as
                // f1, the window mean in that limit, so that it stays finite
                const float k1 = kxy * __ldg(pz + o), den = k1 - acc.y;
                const float f2 = den > 0x1p-20f * k1 ? __fdividef(ki[o * 32] - acc.x, den) : f1;
                const float2 v = make_float2(l1 * f1 - l2 * f2, l1 * (f1 * f1) - l2 * (f2 * f2));
                if constexpr (std::is_same<S, float>::value) {
                    *ab = v;
                } else {
                    // 16-bit storage: the rounding residual of each plane is carried into the
                    // next plane of the column before it is rounded (first-order noise
                    // shaping along z), so that the stored field's rounding error is a
                    // difference of neighbours, which the Gaussian of group B averages out
                    const float2 want = make_float2(v.x + res.x, v.y + res.y);
                    const V2 st = Store<S>::pack2(want);
                    const float2 got = Store<S>::unpack2(st);
                    res = make_float2(want.x - got.x, want.y - got.y);
                    *ab = st;
                }
                ab += pplane;
                if (dump) {
                    const long long q = (long long)zo * B.nx * B.ny + (long long)id.y * B.nx + x;
                    const long long n = (long long)B.nx * B.ny * B.nz;
                    dump[q] = f1 * B.cs[3] + B.cs[0];
                    dump[n + q] = f2 * B.cs[3] + B.cs[0];
                }
            }
        }
    };
    az_walk<STAGE_BYTES>(G, az_sm, issue, body);
}

// The z pass of the Eq. (15) form: the same x-z slabs and persistent walk,
// over the four x/y-convolved fields ((H I~, H), ((1-H) I~, 1-H)) staged as
// one float4 per row and column; writes the fits f1 = K*(H I~)/K*H and
// f2 = K*((1-H) I~)/K*(1-H) (Eq. 6, both sides convolved directly) in FP32
// to B.abxy, where the update kernel forms (I~ - f_i)^2 (Eq. 15, sigma_2 = 0).
template <int R>
constexpr int az4_stage() { return (kAZT + 2 * R) * 32; }  // float4 units per stage
template <int R>
constexpr size_t az4_smem() { return 2 * sizeof(float4) * az4_stage<R>() + 2 * sizeof(uint64_t); }  // + barriers

template <int R>
__global__ void __launch_bounds__(kAZThreads, 2) k_ta_z4(GroupArgs G, TapPairs t) {
    constexpr int T = 2 * R + 1;
    constexpr int WIN = kAZO + 2 * R;
    constexpr int STAGE_BYTES = (int)sizeof(float4) * az4_stage<R>();
    extern __shared__ __align__(128) unsigned char az_sm[];  // [2 stages][ROWS][32] float4, then the barriers
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the slab's box: ROWS planes of the four fields from plane z0 - R (planes outside the
    // brick and columns past nx arrive as zeros)
    const auto issue = [&](const AZSlabId &id, unsigned char *buf, uint64_t *bar, bool fence) {
        const CUtensorMap *map = &G.bricks[id.b].tm_u;
        if (fence) fence_tensormap(map);
        mbar_arrive_expect_tx(bar, (unsigned)STAGE_BYTES + G.fault_tx);
        tma_load_3d(buf, map, 4 * id.x0, id.y, id.z0 - R, bar);
    };
    const auto body = [&](const AZSlabId &id, const unsigned char *sbuf) {
        const float4 *buf = reinterpret_cast<const float4 *>(sbuf);
        const BrickDev &B = G.bricks[id.b];
        const int x = id.x0 + lane;
        const int zb = warp * kAZO;
        if (x >= B.nx) return;
        // the two pairs one after the other, each over a window of float2 entries
        // (one float4 window of 8 + 2R entries spills at radius >= 10)
        float2 acc[2][kAZO];  // (K*(H I~), K*H), (K*((1-H) I~), K*(1-H))
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 *b2 = reinterpret_cast<const float2 *>(buf) + p;
            float2 w[WIN];
#pragma unroll
            for (int j = 0; j < WIN; ++j) w[j] = b2[2 * ((zb + j) * 32 + lane)];
#pragma unroll
            for (int o = 0; o < kAZO; ++o) {
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < T; ++k) a = f2fma(t.g[k], w[o + k], a);
                acc[p][o] = a;
            }
        }
        const long long pplane = (long long)B.px * B.ny;
        const long long off = (long long)(id.z0 + zb) * pplane + (long long)id.y * B.px + x;
        float2 *fits = B.abxy + off;
        const int bnz = B.nz;
        float *const dump = B.dump;
#pragma unroll
        for (int o = 0; o < kAZO; ++o) {
            const int zo = id.z0 + zb + o;
            if (zo < bnz) {
                const float f1 = __fdividef(acc[0][o].x, acc[0][o].y), f2 = __fdividef(acc[1][o].x, acc[1][o].y);
                *fits = make_float2(f1, f2);
                fits += pplane;
                if (dump) {
                    const long long q = (long long)zo * B.nx * B.ny + (long long)id.y * B.nx + x;
                    const long long n = (long long)B.nx * B.ny * B.nz;
                    dump[q] = f1 * B.cs[3] + B.cs[0];
                    dump[n + q] = f2 * B.cs[3] + B.cs[0];
                }
            }
        }
    };
    az_walk<STAGE_BYTES>(G, az_sm, issue, body);
}

// ------------------------------------------------------- set-up: K*I~

// K*I~ of one brick, once per solve: the x/y kernel on (I~, 0) into b.abxy,
// then a z convolution of its first component into b.ki.  Launched per brick
// (the descriptor by value), on the x/y kernel's tiles and the slabs of group A.
template <int R, class ImgT>
__global__ void __launch_bounds__(kXYThreads) k_ki_xy(BrickDev B, TapPairs t) {
    extern __shared__ float2 sm[];
    const int ntx = (B.nx + kXYT - 1) / kXYT, nty = (B.ny + kXYT - 1) / kXYT;
    const int tx = blockIdx.x % ntx, r = blockIdx.x / ntx;
    ProI<ImgT> pro{reinterpret_cast<const ImgT *>(B.img), B.cs[1], -B.cs[0] * B.cs[1]};
    OutF2 out{B.abxy, B.px, (long long)B.px * B.ny};
    ScalarLoader<R, 1, ProI<ImgT>> ld(pro, B.nx, B.ny, B.nx, tx * kXYT, (r % nty) * kXYT);
    xy_tile<R, 1, XYCfg<R, 1, false>>(ld, out, B.nx, B.ny, B.nz, tx * kXYT, (r % nty) * kXYT, (r / nty) * xy_planes(B), xy_planes(B), t, sm);
}

template <int R>
__global__ void __launch_bounds__(kAZThreads) k_ki_z(BrickDev B, TapPairs t) {
    constexpr int T = 2 * R + 1;
    constexpr int WIN = kAZO + 2 * R;
    const int nzt = (B.nz + kAZT - 1) / kAZT, nxt = (B.nx + 31) / 32;
    const int zt = blockIdx.x % nzt, rest = blockIdx.x / nzt;
    const int x = (rest % nxt) * 32 + (threadIdx.x & 31), y = rest / nxt;
    const int z0 = zt * kAZT + (threadIdx.x >> 5) * kAZO;
    if (x >= B.nx) return;
    const long long pplane = (long long)B.px * B.ny;
    const float2 *src = B.abxy + (long long)y * B.px + x;
    float w[WIN];
#pragma unroll
    for (int j = 0; j < WIN; ++j) {
        const int zi = z0 - R + j;
        w[j] = (unsigned)zi < (unsigned)B.nz ? __ldg(src + zi * pplane).x : 0.f;
    }
#pragma unroll
    for (int o = 0; o < kAZO; ++o) {
        if (z0 + o < B.nz) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < T; ++k) acc = fmaf(t.g[k].x, w[o + k], acc);
            B.ki[(long long)(z0 + o) * pplane + (long long)y * B.px + x] = acc;
        }
    }
}

// ------------------------------------------------------------------ B: z

// q = +-atan(eps/|u|)/pi (the small side of H, sign of u) with the atan
// argument kept in [0, 1]: atan(m/M) for m = min(|u|, eps), M = max(|u|, eps),
// and for |u| < eps, atan(eps/|u|) = pi/2 - atan(|u|/eps).  atan(x)/pi on
// [0, 1] is x P(x^2), P the degree-8 minimax polynomial of relative error
// (coefficients by Lawson's algorithm, atan_poly.py), 1.5e-7 relative in FP32.
// P's coefficients, highest power first (Horner order).
__device__ constexpr float kAtanPi[9] = {9.071480017e-04f, -5.114803091e-03f, 1.358913258e-02f, -2.388691157e-02f,
                              3.387114406e-02f, -4.521160573e-02f, 6.363848597e-02f, -1.061024666e-01f,
                              3.183098733e-01f};
__device__ __forceinline__ float atan01_pi(float x) {
    const float t = x * x;
    float p = kAtanPi[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) p = fmaf(p, t, kAtanPi[k]);
    return x * p;
}
__device__ __forceinline__ float heaviside_q_fast(float u, float eps) {
    const float a = fabsf(u);
    const float at = atan01_pi(fminf(a, eps) * rcp_approx(fmaxf(a, eps)));
    return copysignf(a >= eps ? at : 0.5f - at, u);
}

// Packed f32x2 arithmetic (IEEE round-to-nearest per lane) for two planes at once.
__device__ __forceinline__ float2 f2v(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// heaviside_q_fast of two values with packed arithmetic: per lane the same
// operations in the same order (the ratio, the polynomial, 1/2 - at), so each
// lane equals the scalar function bit for bit.
__device__ __forceinline__ float2 heaviside_q_fast2(float2 u, float eps) {
    const float ax = fabsf(u.x), ay = fabsf(u.y);
    const float2 x = f2mul(make_float2(fminf(ax, eps), fminf(ay, eps)),
                           make_float2(rcp_approx(fmaxf(ax, eps)), rcp_approx(fmaxf(ay, eps))));
    const float2 t = f2mul(x, x);
    float2 p = f2v(kAtanPi[0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) p = __ffma2_rn(p, t, f2v(kAtanPi[k]));
    const float2 at = f2mul(x, p);
    const float2 lo = f2sub(f2v(0.5f), at);
    return make_float2(copysignf(ax >= eps ? at.x : lo.x, u.x), copysignf(ay >= eps ? at.y : lo.y, u.y));
}

// z march over a 32x8 column tile of one brick, z chunk [z0, z0 + zc), two
// output planes per step.  Planes are numbered relative to the chunk start
// (r = z - z0); ring slots are r mod ring size, so with the step loop unrolled
// over 2 SPB planes every slot index is a compile-time constant.
//
// Step k, outputs zo = z0 + 2k and zo + 1: bring in the planes later steps
// need (below); barrier; unit normals of planes zo+3, zo+4; outputs zo, zo+1,
// which read phi zo-1 .. zo+2 and the normals of zo-1 .. zo+2 (earlier steps).
// Rings: phi 16 planes, normals 8, (a, b) in registers M = 16 or 32 (2R+2
// planes in use plus those of the next step).  Finite differences use the
// logical planes, which hold reflect-101 copies outside the brick; the unit
// normal is itself padded by reflect-101, so the normal of plane -1 is that of
// plane 1 and the normal of plane nz that of plane nz-2 (the prologue and the
// step loop copy them).
//
// Two schedules by radius (measured per radius):
//   R <= 6: three CTAs per SM at 80 registers.  Step k loads the (a, b) planes
//     of the next step (zo+R+2, zo+R+3) into the register ring, stores phi
//     planes zo+4, zo+5 (loaded one step earlier) into the phi ring and loads
//     zo+6, zo+7, and loads the image and p_z of planes zo+2, zo+3.
//   R >= 8 (a 32-plane register ring): two CTAs per SM at up to 128
//     registers, so the loads run two steps ahead to cover the HBM latency at
//     16 warps per SM.  Step k copies (cp.async) phi planes zo+8, zo+9 straight
//     into the phi ring and this thread's (a, b) of planes zo+R+6, zo+R+7 into
//     an 8-plane staging ring, waits for the copies of two steps ago, moves
//     (a, b) planes zo+R+2, zo+R+3 from the staging ring into the register
//     ring, and loads the image and p_z of planes zo+4, zo+5.  Offsets within a
//     field are 32-bit (bricks of fewer than 2^32 pitched voxels).
template <int R>
constexpr bool tbz_deep() { return R > 6; }
template <int R>
constexpr int tbz_ring() { return 2 * R + 4 <= 4 ? 4 : (2 * R + 4 <= 8 ? 8 : (2 * R + 4 <= 16 ? 16 : 32)); }

constexpr int kZPhiRing = 16, kZNrmRing = 8, kZAbRing = 8;
constexpr int kZPW = kZX + 4, kZPH = kZY + 4;  // phi tile, halo 2
constexpr int kZNW = kZX + 2, kZNH = kZY + 2;  // normal tile, halo 1
template <int R>
constexpr size_t tbz_smem() {
    return sizeof(float) * (kZPhiRing * kZPH * kZPW + kZNrmRing * 3 * kZNH * kZNW) +
           (tbz_deep<R>() ? sizeof(float2) * kZAbRing * kZThreads : 0);
}

__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// DUMP: also write g, kappa and L of every output to B.dump (rsf_step_stages); a
// separate instantiation keeps the iteration's kernel free of it.
template <int R, class ImgT, bool DUMP = false>
__global__ void __launch_bounds__(kZThreads, tbz_deep<R>() ? 2 : 3) k_tb_z(GroupArgs G, TapPairs t) {
    constexpr bool DEEP = tbz_deep<R>();
    constexpr bool PHI_ASYNC = DEEP;  // phi planes copied into the ring two steps ahead (cp.async)
    using Off = typename std::conditional<DEEP, unsigned, long long>::type;  // offsets within a field
    constexpr int NIV = DEEP ? 4 : 2;  // image and p_z registers: planes zo .. zo + NIV - 1
    constexpr int T = 2 * R + 1;
    constexpr int M = tbz_ring<R>();
    constexpr int SPB = (M < kZPhiRing ? kZPhiRing : M) / 2;  // steps per unrolled body: 2 SPB planes, a multiple
                                                              // of every ring size and of NIV
    constexpr int PW = kZPW, PH = kZPH, NW = kZNW, NH = kZNH;
    constexpr int PPL = PH * PW, NPL = 3 * NH * NW;
    constexpr int NPE = (PH * PW + kZThreads - 1) / kZThreads;
    constexpr int NNE = (NH * NW + kZThreads - 1) / kZThreads;
    extern __shared__ float zsm[];
    float *const sphi = zsm;                                                 // [kZPhiRing][PH * PW]
    float *const snrm = zsm + kZPhiRing * PPL;                               // [kZNrmRing][3][NH * NW]
    float2 *const sab = reinterpret_cast<float2 *>(snrm + kZNrmRing * NPL);  // DEEP: [kZAbRing][kZThreads]

    const int bi = find_brick(G.starts, G.nb, blockIdx.x);
    const BrickDev B = G.bricks[bi];
    const int local = blockIdx.x - __ldg(G.starts + bi);
    const int nbx = (B.nx + kZX - 1) / kZX, nby = (B.ny + kZY - 1) / kZY;
    const int bx = local % nbx, rr = local / nbx;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const Off plane = (Off)nx * (Off)ny;

    const int tx = threadIdx.x & (kZX - 1), ty = threadIdx.x / kZX;
    const int x0 = bx * kZX, y0 = (rr % nby) * kZY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < nx && y < ny;
    const int z0 = (rr / nby) * B.zc;
    const int z1 = min(z0 + B.zc, nz);
    const int nout = z1 - z0;
    const int nplanes = nout + 2 * R;  // (a, b) planes of the chunk, r = -R .. nout + R - 1
    const long long col = (long long)min(y, ny - 1) * nx + min(x, nx - 1);
    // this thread's column: in its pointers (R <= 6) or in its 32-bit offsets, from warp-uniform
    // field bases (R >= 8)
    const long long colp = DEEP ? 0 : col;
    const Off colo = DEEP ? (Off)col : (Off)0;
    const int px = B.px;
    const Off pplane = (Off)px * (Off)ny;
    const int par = G.parity ^ B.flip;
    const float *phi = par ? B.phi[1] : B.phi[0];

    int poff[NPE], noff[NNE];
#pragma unroll
    for (int e = 0; e < NPE; ++e) {
        const int i = min((int)threadIdx.x + e * kZThreads, PH * PW - 1);
        const int ly = i / PW, lx = i - ly * PW;
        const int gx = refl101(clampi(x0 + lx - 2, -2, nx + 1), nx);
        const int gy = refl101(clampi(y0 + ly - 2, -2, ny + 1), ny);
        poff[e] = gy * nx + gx;
    }
#pragma unroll
    for (int e = 0; e < NNE; ++e) {
        const int i = min((int)threadIdx.x + e * kZThreads, NH * NW - 1);
        const int ly = i / NW, lx = i - ly * NW;
        const int qx = refl101(clampi(x0 + lx - 1, -1, nx), nx);
        const int qy = refl101(clampi(y0 + ly - 1, -1, ny), ny);
        noff[e] = clampi(qy - y0 + 2, 1, PH - 2) * PW + clampi(qx - x0 + 2, 1, PW - 2);
    }
    auto phi_at = [&](int r) { return sphi + ((r + kZPhiRing) & (kZPhiRing - 1)) * PPL; };
    auto nrm_at = [&](int r) { return snrm + ((r + kZNrmRing) & (kZNrmRing - 1)) * NPL; };
    auto ab_at = [&](int s) { return sab + (s & (kZAbRing - 1)) * kZThreads; };
    // phi plane z (logical, -2 .. nz+1 hold reflect-101 copies; planes past nz+1, never read, are
    // clamped): into registers and then the ring (R <= 6), or copied into the ring (R >= 8)
    auto phi_plane = [&](int z) { return phi + (Off)refl101(clampi(z, -2, nz + 1), nz) * plane; };
    auto fetch_phi = [&](int z, float *v) {
        const float *src = phi_plane(z);
#pragma unroll
        for (int e = 0; e < NPE; ++e) v[e] = __ldg(src + poff[e]);
    };
    auto store_phi = [&](float *dst, const float *v) {
#pragma unroll
        for (int e = 0; e < NPE; ++e)
            if ((int)threadIdx.x + e * kZThreads < PH * PW) dst[threadIdx.x + e * kZThreads] = v[e];
    };
    auto issue_phi = [&](int z, float *dst) {
        const Off zb = (Off)refl101(clampi(z, -2, nz + 1), nz) * plane;
#pragma unroll
        for (int e = 0; e < NPE; ++e)
            if ((int)threadIdx.x + e * kZThreads < PH * PW)
                cp_async4(dst + threadIdx.x + e * kZThreads, phi + (zb + (Off)poff[e]), true);
    };
    // (a, b) plane s of the chunk (z = z0 - R + s) at this thread's column; zero outside the
    // brick and past the chunk: a load (R <= 6) or a copy into a staging slot (R >= 8)
    const long long cab = (long long)min(y, ny - 1) * px + min(x, nx - 1);
    const float2 *src = B.abxy + (DEEP ? 0 : cab);
    const Off cabo = DEEP ? (Off)cab : (Off)0;
    auto ab_ok = [&](int s) { return active && s < nplanes && (unsigned)(z0 - R + s) < (unsigned)nz; };
    auto load_ab = [&](int s) -> float2 {
        return ab_ok(s) ? __ldg(src + (cabo + (Off)(z0 - R + s) * pplane)) : make_float2(0.f, 0.f);
    };
    auto issue_ab = [&](int s, float2 *slot) {
        const bool ok = ab_ok(s);
        cp_async8(slot + threadIdx.x, src + (ok ? cabo + (Off)(z0 - R + s) * pplane : (Off)0), ok);
    };
    // unit normals of one plane from phi planes pm, pc, pp of the ring; the
    // central differences' factor 1/2 cancels: d / (|d| + 2e-10) = (d/2) / (|d/2| + 1e-10)
    auto normals = [&](const float *pm, const float *pc, const float *pp, float *dst) {
#pragma unroll
        for (int e = 0; e < NNE; ++e) {
            const int i = threadIdx.x + e * kZThreads;
            if (i < NH * NW) {
                const int o = noff[e];
                const float gx = pc[o + 1] - pc[o - 1];
                const float gy = pc[o + PW] - pc[o - PW];
                const float gz = pp[o] - pm[o];
                const float inv = rcp_approx(sqrt_approx(gx * gx + gy * gy + gz * gz) + 2e-10f);
                dst[i] = gx * inv;
                dst[NH * NW + i] = gy * inv;
                dst[2 * NH * NW + i] = gz * inv;
            }
        }
    };
    // unit normals of two consecutive planes c, c + 1 from phi planes c - 1 .. c + 2, with
    // packed arithmetic (per lane the operations of normals(), bit for bit)
    auto normals2 = [&](const float *pm, const float *pc, const float *pp, const float *pq, float *dc, float *dp) {
#pragma unroll
        for (int e = 0; e < NNE; ++e) {
            const int i = threadIdx.x + e * kZThreads;
            if (i < NH * NW) {
                const int o = noff[e];
                const float2 gx = f2sub(make_float2(pc[o + 1], pp[o + 1]), make_float2(pc[o - 1], pp[o - 1]));
                const float2 gy = f2sub(make_float2(pc[o + PW], pp[o + PW]), make_float2(pc[o - PW], pp[o - PW]));
                const float2 gz = f2sub(make_float2(pp[o], pq[o]), make_float2(pm[o], pc[o]));
                const float2 ss = __ffma2_rn(gz, gz, __ffma2_rn(gy, gy, f2mul(gx, gx)));
                const float2 r = f2add(make_float2(sqrt_approx(ss.x), sqrt_approx(ss.y)), f2v(2e-10f));
                const float2 inv = make_float2(rcp_approx(r.x), rcp_approx(r.y));
                const float2 nx2 = f2mul(gx, inv), ny2 = f2mul(gy, inv), nz2 = f2mul(gz, inv);
                dc[i] = nx2.x;
                dc[NH * NW + i] = ny2.x;
                dc[2 * NH * NW + i] = nz2.x;
                dp[i] = nx2.y;
                dp[NH * NW + i] = ny2.y;
                dp[2 * NH * NW + i] = nz2.y;
            }
        }
    };
    auto copy_normals = [&](const float *from, float *dst) {
#pragma unroll
        for (int e = 0; e < NNE; ++e) {
            const int i = threadIdx.x + e * kZThreads;
            if (i < NH * NW) {
                dst[i] = from[i];
                dst[NH * NW + i] = from[NH * NW + i];
                dst[2 * NH * NW + i] = from[2 * NH * NW + i];
            }
        }
    };

    // K*1 = p_x p_y p_z; with R = 0 (the Eq. (15) form, sigma_2 = 0) the data terms
    // take no convolution and K*1 is 1
    const float pxy = R == 0 ? 1.f : (active ? __ldg(B.prof + x) * __ldg(B.prof + nx + y) : 0.f);
    const float *profz = B.prof + nx + ny + z0;
    const float l1 = B.lambda1, l2 = B.lambda2, s2 = B.cs[2];
    // the data term's constants folded: s^2 (l1 - l2) p_x p_y (times p_z per plane), -2 s^2, and
    // for the Eq. (15) form s^2 l1, s^2 l2
    const float cK = s2 * (l1 - l2) * pxy, m2s2 = -2.f * s2, s2l1 = s2 * l1, s2l2 = s2 * l2;
    const float inv_s = B.cs[1], nms = -B.cs[0] * B.cs[1];
    const float eps = B.eps, eps2 = eps * eps;
    const float nu = B.nu, dt_mu = B.dt * B.mu, dt_eps_pi = B.dt * (eps * INV_PI);
    const ImgT *img = reinterpret_cast<const ImgT *>(B.img) + colp;
    float *phi_out = (par ? B.phi[0] : B.phi[1]) + colp;
    float *q_out = (par ? B.q[0] : B.q[1]) + colp;
    float *const dump = DUMP ? B.dump : nullptr;
    const long long n = (long long)plane * nz;
    // the centred image and p_z at output plane r (unused values past the chunk: 0 and 1)
    auto img_at = [&](int r) -> float {
        return (active && r < nout) ? centred(img, (long long)(colo + (Off)(z0 + r) * plane), inv_s, nms) : 0.f;
    };
    auto pz_at = [&](int r) -> float { return (R == 0 || r >= nout) ? 1.f : __ldg(profz + r); };

    // prologue: phi planes z0-2 .. z0+3 (R <= 6; z0+4, z0+5 in registers) or z0-2 .. z0+7 and
    // (a, b) planes s = 2R+2 .. 2R+5 (R >= 8, copies); the register ring's planes s = 0 .. 2R+1
    // and the image of planes z0 .. z0+NIV-1
    float pva[NPE], pvb[NPE];
    if constexpr (PHI_ASYNC) {
#pragma unroll 1
        for (int r = -2; r <= 7; ++r) issue_phi(z0 + r, phi_at(r));
    }
    if constexpr (DEEP) {
#pragma unroll
        for (int j = 2 * R + 2; j < 2 * R + 6; ++j) issue_ab(j, ab_at(j));
    }
    if constexpr (PHI_ASYNC || DEEP) {
        cp_async_commit();
    } else {
#pragma unroll 1
        for (int r = -2; r <= 3; ++r) {
            fetch_phi(z0 + r, pva);
            store_phi(phi_at(r), pva);
        }
    }
    float2 ring[M];
#pragma unroll
    for (int s = 0; s < 2 * R + 2; ++s) ring[s] = load_ab(s);
    float iv[NIV], kz[NIV];
#pragma unroll
    for (int j = 0; j < NIV; ++j) {
        iv[j] = img_at(j);
        kz[j] = pz_at(j);
    }
    if constexpr (PHI_ASYNC || DEEP) cp_async_wait0();
    __syncthreads();
#pragma unroll 1
    for (int r = -1; r <= 2; ++r) {
        const int q = refl101(clampi(z0 + r, -1, nz), nz) - z0;  // physical plane, relative
        normals(phi_at(q - 1), phi_at(q), phi_at(q + 1), nrm_at(r));
    }
    if constexpr (!PHI_ASYNC) {
        fetch_phi(z0 + 4, pva);
        fetch_phi(z0 + 5, pvb);
    }

    Off zoff = colo + (Off)z0 * plane;            // offset of the step's first output plane
    Off aoff = (Off)(z0 + R + 2) * pplane;        // offset of the next step's first (a, b) plane (R <= 6)
    for (int base = 0; 2 * base < nout; base += SPB) {
#pragma unroll
        for (int kk = 0; kk < SPB; ++kk) {
            const int k = base + kk;
            const int r0 = 2 * k;  // relative output plane
            if (r0 < nout) {
                const int zo = z0 + r0;
                // the next step's (a, b) planes s = r0 + 2R + 2, + 3 (z = zo + R + 2, + 3) and phi
                if constexpr (PHI_ASYNC) {
                    issue_phi(zo + 8, phi_at(2 * kk + 8));
                    issue_phi(zo + 9, phi_at(2 * kk + 9));
                }
                if constexpr (DEEP) {
                    issue_ab(r0 + 2 * R + 6, ab_at(2 * kk + 2 * R + 6));
                    issue_ab(r0 + 2 * R + 7, ab_at(2 * kk + 2 * R + 7));
                }
                if constexpr (PHI_ASYNC || DEEP) {
                    cp_async_commit();
                    cp_async_wait2();  // this thread's copies of two steps ago have landed
                }
                if constexpr (DEEP) {
                    ring[(2 * kk + 2 * R + 2) % M] = ab_at(2 * kk + 2 * R + 2)[threadIdx.x];
                    ring[(2 * kk + 2 * R + 3) % M] = ab_at(2 * kk + 2 * R + 3)[threadIdx.x];
                } else {
                    const bool in2 = active && r0 + 2 < nout && zo + R + 2 < nz;
                    const bool in3 = active && r0 + 3 < nout && zo + R + 3 < nz;
                    ring[(2 * kk + 2 * R + 2) % M] = in2 ? __ldg(src + aoff) : make_float2(0.f, 0.f);
                    ring[(2 * kk + 2 * R + 3) % M] = in3 ? __ldg(src + aoff + pplane) : make_float2(0.f, 0.f);
                    aoff += 2 * pplane;
                }
                if constexpr (!PHI_ASYNC) {
                    store_phi(phi_at(2 * kk + 4), pva);
                    store_phi(phi_at(2 * kk + 5), pvb);
                    fetch_phi(zo + 6, pva);
                    fetch_phi(zo + 7, pvb);
                }
                const float im0 = iv[(2 * kk) % NIV], im1 = iv[(2 * kk + 1) % NIV];
                const float pz0 = kz[(2 * kk) % NIV], pz1 = kz[(2 * kk + 1) % NIV];
                iv[(2 * kk) % NIV] = img_at(r0 + NIV);
                iv[(2 * kk + 1) % NIV] = img_at(r0 + NIV + 1);
                kz[(2 * kk) % NIV] = pz_at(r0 + NIV);
                kz[(2 * kk + 1) % NIV] = pz_at(r0 + NIV + 1);
                __syncthreads();
                if (zo + 4 < nz) {
                    normals2(phi_at(2 * kk + 2), phi_at(2 * kk + 3), phi_at(2 * kk + 4), phi_at(2 * kk + 5),
                             nrm_at(2 * kk + 3), nrm_at(2 * kk + 4));
                } else {
#pragma unroll
                    for (int c = 3; c <= 4; ++c) {
                        if (zo + c < nz)
                            normals(phi_at(2 * kk + c - 1), phi_at(2 * kk + c), phi_at(2 * kk + c + 1),
                                    nrm_at(2 * kk + c));
                        else if (zo + c == nz)
                            copy_normals(nrm_at(2 * kk + c - 2), nrm_at(2 * kk + c));
                    }
                }
                if (active) {
                    // outputs zo and zo + 1 together: lane c of every float2 below is plane zo + c
                    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int kt = 0; kt < T; ++kt) {
                        a0 = f2fma(t.g[kt], ring[(2 * kk + kt) % M], a0);
                        a1 = f2fma(t.g[kt], ring[(2 * kk + 1 + kt) % M], a1);
                    }
                    const float2 im = make_float2(im0, im1);
                    float2 g;
                    if constexpr (R == 0) {  // Eq. (15), sigma_2 = 0: the ring holds (f1, f2)
                        const float2 d1 = f2sub(im, make_float2(a0.x, a1.x)), d2 = f2sub(im, make_float2(a0.y, a1.y));
                        g = __ffma2_rn(f2v(s2l1), f2mul(d1, d1), f2mul(f2v(-s2l2), f2mul(d2, d2)));
                    } else {  // Li's data terms from K*a, K*b: s^2 [(l1 - l2) K1 I~^2 - 2 I~ K*a + K*b]
                        const float2 t1 = f2mul(f2mul(f2v(cK), make_float2(pz0, pz1)), f2mul(im, im));
                        const float2 t2 = __ffma2_rn(f2mul(f2v(m2s2), im), make_float2(a0.x, a1.x), t1);
                        g = __ffma2_rn(f2v(s2), make_float2(a0.y, a1.y), t2);
                    }
                    const int pc0 = (ty + 2) * PW + tx + 2;
                    const float *pm = phi_at(2 * kk - 1), *p0 = phi_at(2 * kk), *p1 = phi_at(2 * kk + 1),
                                *pp = phi_at(2 * kk + 2);
                    const float2 ph = make_float2(p0[pc0], p1[pc0]);
                    const float2 m2ph = f2mul(f2v(-2.f), ph);
                    const float2 lap =
                        f2add(f2add(f2add(f2add(make_float2(p0[pc0 + 1], p1[pc0 + 1]), make_float2(p0[pc0 - 1], p1[pc0 - 1])), m2ph),
                                    f2add(f2add(make_float2(p0[pc0 + PW], p1[pc0 + PW]), make_float2(p0[pc0 - PW], p1[pc0 - PW])), m2ph)),
                              f2add(f2add(make_float2(p1[pc0], pp[pc0]), make_float2(pm[pc0], p0[pc0])), m2ph));
                    const int nc0 = (ty + 1) * NW + tx + 1;
                    const float *nm = nrm_at(2 * kk - 1), *n0 = nrm_at(2 * kk), *n1 = nrm_at(2 * kk + 1),
                                *np1 = nrm_at(2 * kk + 2);
                    constexpr int NZ = 2 * NH * NW;
                    const float2 kap = f2mul(
                        f2add(f2add(f2sub(make_float2(n0[nc0 + 1], n1[nc0 + 1]), make_float2(n0[nc0 - 1], n1[nc0 - 1])),
                                    f2sub(make_float2(n0[NH * NW + nc0 + NW], n1[NH * NW + nc0 + NW]),
                                          make_float2(n0[NH * NW + nc0 - NW], n1[NH * NW + nc0 - NW]))),
                              f2sub(make_float2(n1[NZ + nc0], np1[NZ + nc0]), make_float2(nm[NZ + nc0], n0[NZ + nc0]))),
                        f2v(0.5f));
                    const float2 den = __ffma2_rn(ph, ph, f2v(eps2));
                    // dt delta (Eq. 14), then phi + dt mu (L - kappa) + dt delta (nu kappa - g) (Eqs. 1, 13)
                    const float2 dtdel = f2mul(f2v(dt_eps_pi), make_float2(rcp_approx(den.x), rcp_approx(den.y)));
                    const float2 pn = __ffma2_rn(f2v(dt_mu), f2sub(lap, kap),
                                                 __ffma2_rn(dtdel, __ffma2_rn(f2v(nu), kap, make_float2(-g.x, -g.y)), ph));
                    const float2 qn = heaviside_q_fast2(pn, eps);
                    phi_out[zoff] = pn.x;
                    q_out[zoff] = qn.x;
                    if (r0 + 1 < nout) {
                        phi_out[zoff + plane] = pn.y;
                        q_out[zoff + plane] = qn.y;
                    }
                    if constexpr (DUMP) {
                        const long long q0 = colp + (long long)zoff, q1 = q0 + (long long)plane;
                        dump[2 * n + q0] = g.x;
                        dump[3 * n + q0] = kap.x;
                        dump[4 * n + q0] = lap.x;
                        if (r0 + 1 < nout) {
                            dump[2 * n + q1] = g.y;
                            dump[3 * n + q1] = kap.y;
                            dump[4 * n + q1] = lap.y;
                        }
                    }
                }
                zoff += 2 * plane;
            }
        }
    }
    if constexpr (PHI_ASYNC || DEEP) cp_async_wait0();  // no copy into this CTA's shared memory outlives it
}

// ------------------------------------------------------------ launchers

// The update kernel (storage independent; defined in rsf_tiled_f32.cu).
cudaError_t launch_tb_z(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s);
cudaError_t prepare_tb_z(int R);

// Resident CTAs of the persistent z kernel of group A (set by prepare_storage).
template <int R, class S>
int &az_persist() {
    static int n = 152;
    return n;
}

template <int R, class S>
cudaError_t prepare_storage() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)XYLayout<R, 1>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)XYLayout<R, 1>::bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ta_xy<R, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)XYLayout<R, 1>::bytes)) != cudaSuccess) return e;
    if constexpr (R % 2 == 0) {
        if ((e = cudaFuncSetAttribute(k_ta_xy_tma<R, uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)XYStageH<R, uint8_t>::smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_ta_xy_tma<R, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)XYStageH<R, uint16_t>::smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_ta_xy_tma<R, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)XYStageH<R, float>::smem)) != cudaSuccess) return e;
    }
    if ((e = cudaFuncSetAttribute(k_ta_z<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)az_smem<R>())) !=
        cudaSuccess) return e;
    {
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ta_z<R, S>, kAZThreads, az_smem<R>())) !=
            cudaSuccess) return e;
        az_persist<R, S>() = sms * (occ > 0 ? occ : 1);
    }
    return cudaFuncSetAttribute(k_tb_xy<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tbxy_smem<R, S>());
}

// One iteration of Li's form (group A, group B, update) for radius R and storage S.
template <int R, class S>
cudaError_t launch_storage(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    GroupArgs G{g.bricks, nullptr, g.nb, parity, g.err, g.fault_tx};
    const TapPairs tp = tap_pairs(g.taps);
    {
        ProfScope ps(prof, KID_TA_XY);
        G.starts = g.starts[0];
        constexpr size_t sm = XYLayout<R, 1>::bytes;
        bool staged = false;  // inputs by TMA (every brick's rows allow the copies)
        if constexpr (R % 2 == 0) {
            if (g.xy_tma) {
                staged = true;
                switch (g.imgtype) {
                    case 0: k_ta_xy_tma<R, uint8_t><<<g.ncta[0], kXYThreads, XYStageH<R, uint8_t>::smem, s>>>(G, tp); break;
                    case 1: k_ta_xy_tma<R, uint16_t><<<g.ncta[0], kXYThreads, XYStageH<R, uint16_t>::smem, s>>>(G, tp); break;
                    default: k_ta_xy_tma<R, float><<<g.ncta[0], kXYThreads, XYStageH<R, float>::smem, s>>>(G, tp);
                }
            }
        }
        if (!staged) {
            switch (g.imgtype) {
                case 0: k_ta_xy<R, uint8_t><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp); break;
                case 1: k_ta_xy<R, uint16_t><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp); break;
                default: k_ta_xy<R, float><<<g.ncta[0], kXYThreads, sm, s>>>(G, tp);
            }
        }
    }
    {
        ProfScope ps(prof, KID_TA_Z);
        G.starts = g.starts[1];
        const unsigned grid = g.ncta[1] < (unsigned)az_persist<R, S>() ? g.ncta[1] : (unsigned)az_persist<R, S>();
        k_ta_z<R, S><<<grid, kAZThreads, az_smem<R>(), s>>>(G, tp);
    }
    {
        ProfScope ps(prof, KID_TB_XY);
        G.starts = g.starts[2];
        k_tb_xy<R, S><<<g.ncta[2], kXYThreads, tbxy_smem<R, S>(), s>>>(G, tp);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tb_z(g, parity, prof, s);
}

template <class S>
cudaError_t prepare_group_s(int R) {
    switch (R) {
        case 2: return prepare_storage<2, S>();
        case 3: return prepare_storage<3, S>();
        case 4: return prepare_storage<4, S>();
        case 5: return prepare_storage<5, S>();
        case 6: return prepare_storage<6, S>();
        case 8: return prepare_storage<8, S>();
        case 10: return prepare_storage<10, S>();
        case 12: return prepare_storage<12, S>();
        default: return cudaErrorInvalidValue;
    }
}

template <class S>
cudaError_t launch_group_s(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s) {
    switch (g.taps.R) {
        case 2: return launch_storage<2, S>(g, parity, prof, s);
        case 3: return launch_storage<3, S>(g, parity, prof, s);
        case 4: return launch_storage<4, S>(g, parity, prof, s);
        case 5: return launch_storage<5, S>(g, parity, prof, s);
        case 6: return launch_storage<6, S>(g, parity, prof, s);
        case 8: return launch_storage<8, S>(g, parity, prof, s);
        case 10: return launch_storage<10, S>(g, parity, prof, s);
        case 12: return launch_storage<12, S>(g, parity, prof, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tiled
}  // namespace rsf
