// rsf_tiled.cu -- the tiled four-kernel RSF iteration (arXiv 2404.02813,
// Sec. 3 and 4.2), the library's default path for kernel radii 2..6, 8, 10, 12.
//
//   rsf_ta_xy  per z-plane, a 32x32 output tile plus an R halo in shared
//              memory: forms H I~, H, (1-H) I~, 1-H (Eqs. 6, 8-10) from the
//              centred image and q = +-atan(eps/|phi|)/pi, convolves them
//              along x then y (field pairs share packed f32x2 FMAs) and stores
//              one float4 per voxel.
//   rsf_ta_z   x-z slabs (32 columns x 64 output planes) loaded into shared
//              memory all at once; z convolution over a register window; the
//              local fits f1 = K*(H I)/K*H, f2 = K*((1-H) I)/K*(1-H), and
//              a = l1 f1 - l2 f2, b = l1 f1^2 - l2 f2^2 (one float2 per voxel).
//   rsf_tb_xy  the x/y kernel on the (a, b) pair.
//   rsf_tb_z   a z march over a 32x8 column tile: a register ring of (a, b)
//              planes (loaded two planes ahead), a phi ring and a unit-normal
//              ring in shared memory (each normal computed once per voxel);
//              g = s^2 [ (l1 - l2) K1 I~^2 - 2 I~ K*a + K*b ]  (Eqs. 11-12),
//              kappa, the Laplacian (Eqs. 3-4), the update of Eqs. (1), (13),
//              (14), and q of the new phi for the next rsf_ta_xy.
//
// Convolutions use zero padding, taps summed k = -R..R, FP32 accumulation;
// finite differences use reflect-101 for phi and for the normal.  The three
// intermediate fields are stored with an x pitch rounded up to 32 columns.
// Compulsory traffic: 24 + 24 + 16 + 24 = 88 bytes per voxel and iteration.
#include <cuda_runtime.h>

#include <cstdint>

#include "rsf_internal.h"

namespace rsf {
namespace {

constexpr int kXYT = 32;          // x/y kernel: output tile edge (x and y)
constexpr int kXYThreads = 256;   // 8 warps
constexpr int kZX = 32, kZY = 8;  // z kernels: columns per CTA
constexpr int kZThreads = kZX * kZY;

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ----------------------------------------------------------------- x / y

struct ProHP {  // (H I~, H), ((1-H) I~, 1-H) from q = +-atan(eps/|phi|)/pi and the centred image
    const float *q, *I;
    struct Raw { float q, im; };
    __device__ __forceinline__ Raw fetch(long long p) const { return Raw{__ldg(q + p), __ldg(I + p)}; }
    __device__ __forceinline__ Raw zero() const { return Raw{0.f, 0.f}; }
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        if (inside) {
            const float h = h_of_q(r.q), hc = hc_of_q(r.q);
            v[0] = make_float2(h * r.im, h);
            v[1] = make_float2(hc * r.im, hc);
        } else {
            v[0] = v[1] = make_float2(0.f, 0.f);
        }
    }
};

struct ProAB {  // (a, b) as stored by rsf_ta_z (pitched)
    const float2 *ab;
    using Raw = float2;
    __device__ __forceinline__ Raw fetch(long long p) const { return __ldg(ab + p); }
    __device__ __forceinline__ Raw zero() const { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ void apply(const Raw &r, bool inside, float2 *v) const {
        v[0] = inside ? r : make_float2(0.f, 0.f);
    }
};

// Shared-memory layout of the x/y kernel (float2 units).
template <int R, int NP>
struct XYLayout {
    static constexpr int W = kXYT + 2 * R;              // loaded width
    static constexpr int H = kXYT + 2 * R;              // loaded rows
    static constexpr int P = ((W + 15) / 16) * 16 + 1;  // row pitch = 1 (mod 16): conflict-free float2 reads
    static constexpr int IN = NP * H * P;               // input tile
    static constexpr int XC = NP * H * kXYT;            // x-convolved rows
    static constexpr size_t bytes = sizeof(float2) * (IN + XC);
};

constexpr int kXYPlanes = 8;  // z-planes per CTA of the x/y kernel

// grid: (ceil(nx/32), ceil(ny/32), ceil(nz/kXYPlanes)).  Each CTA walks its
// planes; the global loads of plane z+1 are issued right after the first
// barrier of plane z and land in registers while the convolutions run.
// Input row pitch `ipx` (nx for q and I, the pitch for (a, b)); output pitch `opx`.
template <int R, int NP, class Pro>
__global__ void __launch_bounds__(kXYThreads, ((NP == 2 && R <= 6) || (NP == 1 && R <= 5)) ? 3 : 2)
    k_xy(Pro pro, float2 *__restrict__ out, Dims d, int ipx, int opx, Taps t) {
    using L = XYLayout<R, NP>;
    using Raw = typename Pro::Raw;
    constexpr int T = 2 * R + 1;
    constexpr int XT = 4, YT = 4;            // outputs per thread in the x and y phases
    constexpr int NRB = (L::H + 7) / 8;      // 8-row blocks of the x phase
    constexpr int NE = (L::H * L::W + kXYThreads - 1) / kXYThreads;  // tile entries per thread
    static_assert(NE <= 32, "tile entries per thread exceed the mask");
    extern __shared__ float2 sm[];
    float2 *in = sm;
    float2 *xc = sm + L::IN;
    float2 gg[T];
#pragma unroll
    for (int k = 0; k < T; ++k) gg[k] = make_float2(t.g[k], t.g[k]);

    const int x0 = blockIdx.x * kXYT, y0 = blockIdx.y * kXYT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int za = blockIdx.z * kXYPlanes, zb_end = min(za + kXYPlanes, d.nz);
    const long long iplane = (long long)ipx * d.ny, oplane = (long long)opx * d.ny;

    // z-invariant part of the tile entries this thread loads
    int eoff[NE], esm[NE];
    unsigned inside = 0;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int i = threadIdx.x + e * kXYThreads;
        const int ii = min(i, L::H * L::W - 1);
        const int ly = ii / L::W, lx = ii - ly * L::W;
        const int gx = x0 + lx - R, gy = y0 + ly - R;
        const bool in_vol = i < L::H * L::W && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
        eoff[e] = in_vol ? gy * ipx + gx : 0;
        esm[e] = i < L::H * L::W ? ly * L::P + lx : -1;
        inside |= (in_vol ? 1u : 0u) << e;
    }
    Raw raw[NE];
    auto fetch = [&](int z) {
        const long long zb = (long long)z * iplane;
#pragma unroll
        for (int e = 0; e < NE; ++e) raw[e] = ((inside >> e) & 1u) ? pro.fetch(zb + eoff[e]) : pro.zero();
    };
    fetch(za);
    for (int z = za; z < zb_end; ++z) {
        // phase 1: prologue on the fetched tile (zero outside the volume)
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            if (esm[e] >= 0) {
                float2 v[NP];
                pro.apply(raw[e], (inside >> e) & 1u, v);
#pragma unroll
                for (int p = 0; p < NP; ++p) in[p * L::H * L::P + esm[e]] = v[p];
            }
        }
        __syncthreads();
        if (z + 1 < zb_end) fetch(z + 1);
        // phase 2: x convolution.  A warp covers 8 rows x 16 outputs; lane -> (row, group of 4 outputs)
        {
            const int h = lane >> 4, r = (lane >> 2) & 3, g = lane & 3;
            for (int item = warp; item < NP * NRB * 2; item += kXYThreads / 32) {
                const int p = item / (NRB * 2);
                const int rem = item - p * NRB * 2;
                const int row = (rem >> 1) * 8 + h * 4 + r;
                const int xo = (rem & 1) * 16 + g * XT;
                if (row < L::H) {
                    const float2 *src = in + (p * L::H + row) * L::P + xo;
                    float2 w[XT + 2 * R];
#pragma unroll
                    for (int j = 0; j < XT + 2 * R; ++j) w[j] = src[j];
#pragma unroll
                    for (int o = 0; o < XT; ++o) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < T; ++k) acc = f2fma(gg[k], w[o + k], acc);
                        xc[(p * L::H + row) * kXYT + xo + o] = acc;
                    }
                }
            }
        }
        __syncthreads();
        // phase 3: y convolution; thread -> (x = lane, 4 rows starting at 4*warp)
        {
            const int gx = x0 + lane;
            float2 res[NP][YT];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 w[YT + 2 * R];
#pragma unroll
                for (int j = 0; j < YT + 2 * R; ++j) w[j] = xc[(p * L::H + warp * YT + j) * kXYT + lane];
#pragma unroll
                for (int o = 0; o < YT; ++o) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < T; ++k) acc = f2fma(gg[k], w[o + k], acc);
                    res[p][o] = acc;
                }
            }
            if (gx < d.nx) {
                const int gy0 = y0 + warp * YT;
                const long long q0 = (long long)z * oplane + (long long)gy0 * opx + gx;
#pragma unroll
                for (int o = 0; o < YT; ++o) {
                    if (gy0 + o < d.ny) {
                        const long long q = q0 + (long long)o * opx;
                        if (NP == 2) {
                            reinterpret_cast<float4 *>(out)[q] =
                                make_float4(res[0][o].x, res[0][o].y, res[NP - 1][o].x, res[NP - 1][o].y);
                        } else {
                            out[q] = res[0][o];
                        }
                    }
                }
            }
        }
        __syncthreads();  // the next plane reuses the tiles
    }
}

// ---------------------------------------------------------------- A: z

// Group A z pass over x-z slabs: a CTA takes 32 columns of one y row and kAZT
// consecutive output planes, loads the kAZT + 2R input planes of that slab into
// shared memory with every load in flight at once (no marching state), then
// each lane convolves its column over a register window.  The slab is stored
// as two float2 arrays (the (H I, H) and ((1-H) I, 1-H) pairs) so that the
// window reads are conflict-free.  Consecutive CTAs take consecutive z slabs of
// the same row, so the 2R halo planes they share are mostly L2 hits.
constexpr int kAZT = 64;        // output planes per CTA
constexpr int kAZThreads = 256; // 8 warps x 8 output planes each
constexpr int kAZO = kAZT / (kAZThreads / 32);

// grid: (ceil(nz/kAZT) * ceil(nx/32) * ny); block kAZThreads; dynamic smem 2 * (kAZT+2R) * 32 float2.
template <int R>
__global__ void __launch_bounds__(kAZThreads)
    k_az(const float4 *__restrict__ u, float2 *__restrict__ ab, Dims d, int px, Taps t, float l1, float l2,
         const float *__restrict__ cs, float *__restrict__ dump_f1, float *__restrict__ dump_f2) {
    constexpr int T = 2 * R + 1;
    constexpr int ROWS = kAZT + 2 * R;
    constexpr int WIN = kAZO + 2 * R;
    extern __shared__ float2 slab[];  // [2][ROWS][32]
    const int nzt = (d.nz + kAZT - 1) / kAZT, nxt = (d.nx + 31) / 32;
    const int id = blockIdx.x;
    const int zt = id % nzt;
    const int rest = id / nzt;
    const int xt = rest % nxt, y = rest / nxt;
    const int x0 = xt * 32, z0 = zt * kAZT;
    const long long pplane = (long long)px * d.ny;
    const float4 *src = u + (long long)y * px + x0;

    // every load of the slab in flight at once; planes outside the volume are zero
    for (int i = threadIdx.x; i < ROWS * 32; i += kAZThreads) {
        const int row = i >> 5, col = i & 31;
        const int zi = z0 - R + row;
        const float4 v = ((unsigned)zi < (unsigned)d.nz) ? __ldg(src + (long long)zi * pplane + col)
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        slab[row * 32 + col] = make_float2(v.x, v.y);
        slab[(ROWS + row) * 32 + col] = make_float2(v.z, v.w);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = x0 + lane;
    const int zb = warp * kAZO;  // first output plane of this warp, relative to z0
    if (x >= d.nx) return;
    float f1[kAZO];
    {
        float2 w[WIN];
#pragma unroll
        for (int j = 0; j < WIN; ++j) w[j] = slab[(zb + j) * 32 + lane];
#pragma unroll
        for (int o = 0; o < kAZO; ++o) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < T; ++k) acc = f2fma(make_float2(t.g[k], t.g[k]), w[o + k], acc);
            f1[o] = __fdividef(acc.x, acc.y);
        }
    }
    float2 w[WIN];
#pragma unroll
    for (int j = 0; j < WIN; ++j) w[j] = slab[(ROWS + zb + j) * 32 + lane];
#pragma unroll
    for (int o = 0; o < kAZO; ++o) {
        const int zo = z0 + zb + o;
        if (zo < d.nz) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < T; ++k) acc = f2fma(make_float2(t.g[k], t.g[k]), w[o + k], acc);
            const float f2 = __fdividef(acc.x, acc.y);
            ab[(long long)zo * pplane + (long long)y * px + x] =
                make_float2(l1 * f1[o] - l2 * f2, l1 * (f1[o] * f1[o]) - l2 * (f2 * f2));
            if (dump_f1) {
                const long long q = (long long)zo * d.plane + (long long)y * d.nx + x;
                dump_f1[q] = f1[o] * cs[3] + cs[0];
                dump_f2[q] = f2 * cs[3] + cs[0];
            }
        }
    }
}

template <int R>
constexpr size_t az_smem() { return sizeof(float2) * 2 * (kAZT + 2 * R) * 32; }

// ---------------------------------------------------------------- B: z

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

struct BZArgs {
    const float2 *abxy;       // pitched
    const float *phi, *I, *prof, *cs;
    float *phi_out, *q_out;   // phi_{n+1} and its small-side Heaviside value
    float *dump_g, *dump_k, *dump_l;
};

// q = +-atan(eps/|u|)/pi (the small side of H, sign of u), with the atan
// argument kept in [0, 1]: for |u| < eps, atan(eps/|u|) = pi/2 - atan(|u|/eps).
__device__ __forceinline__ float heaviside_q_fast(float u, float eps) {
    const float a = fabsf(u);
    const float r = a >= eps ? atanf(__fdividef(eps, a)) * INV_PI : 0.5f - atanf(__fdividef(a, eps)) * INV_PI;
    return copysignf(r, u);
}

constexpr int kPFB = 2;  // (a, b) planes loaded ahead in registers

// grid: (ceil(nx/32), ceil(ny/8), ceil(nz/zc)); 256 threads, one barrier per output plane.
//
// Output step zo:  store phi plane zo+3 (loaded into registers one step earlier)
//                  and issue the loads of plane zo+4;  barrier;
//                  normals of plane zo+2;  output of plane zo, which reads the
//                  normals of zo-1, zo, zo+1 written in earlier steps.
// Rings (logical plane p in slot p & (size-1)): phi 8 planes (zo-2 .. zo+3 live),
// normals 4 planes (zo-1 .. zo+2 live).  The reflected tile offsets do not
// depend on z and are computed once.  The (a, b) window is a register ring of
// 2R+1+kPFB slots (plane s in slot s mod (2R+1+kPFB)); the load of plane
// s+kPFB goes straight into its slot, so the body unrolled over the ring has
// static indices.
template <int R>
__global__ void __launch_bounds__(kZThreads, R <= 8 ? 3 : 2) k_bz(BZArgs A, Dims d, int px, Taps t, Coeffs c, int zc) {
    constexpr int T = 2 * R + 1;
    constexpr int M = T + kPFB;
    constexpr int PW = kZX + 4, PH = kZY + 4;  // phi tile: halo 2
    constexpr int NW = kZX + 2, NH = kZY + 2;  // normal tile: halo 1
    constexpr int NPE = (PH * PW + kZThreads - 1) / kZThreads;  // phi tile entries per thread
    constexpr int NNE = (NH * NW + kZThreads - 1) / kZThreads;  // normal tile entries per thread
    __shared__ float sphi[8][PH * PW];
    __shared__ float snrm[4][3][NH * NW];

    const int tx = threadIdx.x & (kZX - 1), ty = threadIdx.x / kZX;
    const int x0 = blockIdx.x * kZX, y0 = blockIdx.y * kZY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < d.nx && y < d.ny;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, d.nz);
    const int nsteps = (z1 - z0) + 2 * R;
    const long long col = (long long)min(y, d.ny - 1) * d.nx + min(x, d.nx - 1);
    const long long pplane = (long long)px * d.ny;

    int poff[NPE], noff[NNE];
#pragma unroll
    for (int e = 0; e < NPE; ++e) {
        const int i = min((int)threadIdx.x + e * kZThreads, PH * PW - 1);
        const int ly = i / PW, lx = i - ly * PW;
        const int gx = refl101(clampi(x0 + lx - 2, -2, d.nx + 1), d.nx);
        const int gy = refl101(clampi(y0 + ly - 2, -2, d.ny + 1), d.ny);
        poff[e] = gy * d.nx + gx;
    }
#pragma unroll
    for (int e = 0; e < NNE; ++e) {
        const int i = min((int)threadIdx.x + e * kZThreads, NH * NW - 1);
        const int ly = i / NW, lx = i - ly * NW;
        const int qx = refl101(clampi(x0 + lx - 1, -1, d.nx), d.nx);
        const int qy = refl101(clampi(y0 + ly - 1, -1, d.ny), d.ny);
        noff[e] = clampi(qy - y0 + 2, 1, PH - 2) * PW + clampi(qx - x0 + 2, 1, PW - 2);
    }
    auto fetch_phi = [&](int lz, float *v) {
        const float *src = A.phi + (long long)refl101(clampi(lz, -2, d.nz + 1), d.nz) * d.plane;
#pragma unroll
        for (int e = 0; e < NPE; ++e) v[e] = __ldg(src + poff[e]);
    };
    auto store_phi = [&](int lz, const float *v) {
        float *dst = sphi[lz & 7];
#pragma unroll
        for (int e = 0; e < NPE; ++e)
            if ((int)threadIdx.x + e * kZThreads < PH * PW) dst[threadIdx.x + e * kZThreads] = v[e];
    };
    // unit normals of logical plane lz, each evaluated at the reflected position
    auto normals = [&](int lz) {
        const int q = refl101(clampi(lz, -1, d.nz), d.nz);  // physical plane; q-1..q+1 are in the phi ring
        const float *pm = sphi[(q - 1) & 7], *pc = sphi[q & 7], *pp = sphi[(q + 1) & 7];
        float *n0 = snrm[lz & 3][0], *n1 = snrm[lz & 3][1], *n2 = snrm[lz & 3][2];
#pragma unroll
        for (int e = 0; e < NNE; ++e) {
            const int i = threadIdx.x + e * kZThreads;
            if (i < NH * NW) {
                const int o = noff[e];
                const float gx = (pc[o + 1] - pc[o - 1]) * 0.5f;
                const float gy = (pc[o + PW] - pc[o - PW]) * 0.5f;
                const float gz = (pp[o] - pm[o]) * 0.5f;
                const float inv = rcp_approx(sqrt_approx(gx * gx + gy * gy + gz * gz) + 1e-10f);
                n0[i] = gx * inv;
                n1[i] = gy * inv;
                n2[i] = gz * inv;
            }
        }
    };

    // warm-up: phi planes z0-2 .. z0+3, normals of z0-1 .. z0+1
    float pv[NPE];
    for (int lz = z0 - 2; lz <= z0 + 3; ++lz) {
        fetch_phi(lz, pv);
        store_phi(lz, pv);
    }
    __syncthreads();
    normals(z0 - 1);
    normals(z0);
    normals(z0 + 1);
    fetch_phi(z0 + 3, pv);  // the first output step stores plane z0+3 again, from registers

    const float pxy = active ? __ldg(A.prof + x) * __ldg(A.prof + d.nx + y) : 0.f;
    const float *profz = A.prof + d.nx + d.ny;
    const float l12 = c.lambda1 - c.lambda2, s2 = A.cs[2];
    const float eps_pi = c.eps * INV_PI, eps2 = c.eps * c.eps;
    const float *Iz = A.I + (long long)z0 * d.plane + col;
    float *Oz = A.phi_out + (long long)z0 * d.plane + col;
    float *Qz = A.q_out + (long long)z0 * d.plane + col;
    const int pc0 = (ty + 2) * PW + tx + 2;  // this thread's voxel in the phi tile
    const int nc0 = (ty + 1) * NW + tx + 1;  // and in the normal tile

    const float2 *src = A.abxy + (long long)min(y, d.ny - 1) * px + min(x, d.nx - 1);
    auto load = [&](int s) -> float2 {
        const int zi = z0 - R + s;
        return (active && s < nsteps && (unsigned)zi < (unsigned)d.nz) ? __ldg(src + (long long)zi * pplane)
                                                                        : make_float2(0.f, 0.f);
    };
    float2 r[M];
#pragma unroll
    for (int i = 0; i < kPFB; ++i) r[i] = load(i);
    float iv = active ? __ldg(Iz) : 0.f;
    for (int base = 0; base < nsteps; base += M) {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int s = base + j;
            if (s < nsteps) {
                r[(j + kPFB) % M] = load(s + kPFB);
                if (s >= 2 * R) {
                    const int zo = z0 + s - 2 * R;
                    store_phi(zo + 3, pv);
                    fetch_phi(zo + 4, pv);
                    const float im = iv;
                    if (active && zo + 1 < z1) iv = __ldg(Iz + d.plane);
                    __syncthreads();
                    normals(zo + 2);
                    if (active) {
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < T; ++k)
                            acc = f2fma(make_float2(t.g[k], t.g[k]), r[(j - 2 * R + k + 2 * M) % M], acc);
                        const float K1 = pxy * __ldg(profz + zo);
                        const float g = s2 * (l12 * K1 * (im * im) - 2.f * im * acc.x + acc.y);
                        const float *p0 = sphi[zo & 7];
                        const float ph = p0[pc0];
                        const float lap = (p0[pc0 + 1] + p0[pc0 - 1] - 2.f * ph) + (p0[pc0 + PW] + p0[pc0 - PW] - 2.f * ph) +
                                          (sphi[(zo + 1) & 7][pc0] + sphi[(zo - 1) & 7][pc0] - 2.f * ph);
                        const float *n0 = snrm[zo & 3][0], *n1 = snrm[zo & 3][1];
                        const float kap = (n0[nc0 + 1] - n0[nc0 - 1]) * 0.5f + (n1[nc0 + NW] - n1[nc0 - NW]) * 0.5f +
                                          (snrm[(zo + 1) & 3][2][nc0] - snrm[(zo - 1) & 3][2][nc0]) * 0.5f;
                        const float del = eps_pi * rcp_approx(eps2 + ph * ph);  // Eq. (14)
                        const float pn = ph + c.dt * (c.mu * (lap - kap) + del * (c.nu * kap - g));
                        *Oz = pn;
                        *Qz = heaviside_q_fast(pn, c.eps);
                        if (A.dump_g) {
                            const long long q = Oz - A.phi_out;
                            A.dump_g[q] = g;
                            A.dump_k[q] = kap;
                            A.dump_l[q] = lap;
                        }
                    }
                    Iz += d.plane;
                    Oz += d.plane;
                    Qz += d.plane;
                }
            }
        }
    }
}

// ------------------------------------------------------------- launchers

template <int R>
cudaError_t iterate_r(const Taps &t, const Coeffs &c, Fields &f, const float *phi_in, const float *q_in, float *phi_out,
                      float *q_out, float *dump, Profiler *prof, cudaStream_t s, int zc) {
    const Dims &d = f.d;
    const long long n = d.n;
    const int px = f.px;
    const long long np = (long long)px * d.ny * d.nz;
    float4 *u = reinterpret_cast<float4 *>(f.t[0]);             // 4 np floats
    float2 *ab = reinterpret_cast<float2 *>(f.t[0] + 4 * np);   // 2 np floats
    float2 *abxy = reinterpret_cast<float2 *>(f.t[0] + 6 * np); // 2 np floats
    const dim3 gxy((d.nx + kXYT - 1) / kXYT, (d.ny + kXYT - 1) / kXYT, (d.nz + kXYPlanes - 1) / kXYPlanes);
    const dim3 gz((d.nx + kZX - 1) / kZX, (d.ny + kZY - 1) / kZY, (d.nz + zc - 1) / zc);
    {
        ProfScope ps(prof, KID_TA_XY);
        constexpr size_t sm = XYLayout<R, 2>::bytes;
        k_xy<R, 2, ProHP><<<gxy, kXYThreads, sm, s>>>(ProHP{q_in, f.I}, reinterpret_cast<float2 *>(u), d, d.nx, px, t);
    }
    {
        ProfScope ps(prof, KID_TA_Z);
        const long long nb = (long long)((d.nz + kAZT - 1) / kAZT) * ((d.nx + 31) / 32) * d.ny;
        k_az<R><<<(unsigned)nb, kAZThreads, az_smem<R>(), s>>>(u, ab, d, px, t, c.lambda1, c.lambda2, f.cs,
                                                               dump ? dump : nullptr, dump ? dump + n : nullptr);
    }
    {
        ProfScope ps(prof, KID_TB_XY);
        constexpr size_t sm = XYLayout<R, 1>::bytes;
        k_xy<R, 1, ProAB><<<gxy, kXYThreads, sm, s>>>(ProAB{ab}, abxy, d, px, px, t);
    }
    {
        ProfScope ps(prof, KID_TB_Z);
        BZArgs A{abxy, phi_in, f.I, f.prof, f.cs, phi_out, q_out, dump ? dump + 2 * n : nullptr,
                 dump ? dump + 3 * n : nullptr, dump ? dump + 4 * n : nullptr};
        k_bz<R><<<gz, kZThreads, 0, s>>>(A, d, px, t, c, zc);
    }
    return cudaGetLastError();
}

template <int R>
cudaError_t prepare_r() {
    cudaError_t e = cudaFuncSetAttribute(k_az<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)az_smem<R>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_xy<R, 2, ProHP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)XYLayout<R, 2>::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_xy<R, 1, ProAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)XYLayout<R, 1>::bytes);
}

__global__ void k_q_init(const float *__restrict__ phi, float *__restrict__ q, long long n, float eps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        q[i] = heaviside_q_fast(__ldg(phi + i), eps);
}

}  // namespace

bool tiled_supports(int R) {
    switch (R) {
        case 2: case 3: case 4: case 5: case 6: case 8: case 10: case 12: return true;
        default: return false;
    }
}

int tiled_pitch(int nx) { return (nx + kZX - 1) / kZX * kZX; }

cudaError_t tiled_prepare(int R) {
    switch (R) {
        case 2: return prepare_r<2>();
        case 3: return prepare_r<3>();
        case 4: return prepare_r<4>();
        case 5: return prepare_r<5>();
        case 6: return prepare_r<6>();
        case 8: return prepare_r<8>();
        case 10: return prepare_r<10>();
        case 12: return prepare_r<12>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t tiled_q_init(const float *phi, float *q, long long n, float eps, cudaStream_t s) {
    k_q_init<<<1216, 256, 0, s>>>(phi, q, n, eps);
    return cudaGetLastError();
}

cudaError_t iterate_tiled(const Taps &t, const Coeffs &c, Fields &f, const float *phi_in, const float *q_in,
                          float *phi_out, float *q_out, float *stages, Profiler *prof, cudaStream_t s, int zc) {
    switch (t.R) {
        case 2: return iterate_r<2>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 3: return iterate_r<3>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 4: return iterate_r<4>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 5: return iterate_r<5>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 6: return iterate_r<6>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 8: return iterate_r<8>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 10: return iterate_r<10>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        case 12: return iterate_r<12>(t, c, f, phi_in, q_in, phi_out, q_out, stages, prof, s, zc);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rsf
