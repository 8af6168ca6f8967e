// rsf_passes.cu -- set-up kernels and the separable six-pass path of one RSF
// iteration (arXiv 2404.02813, Sec. 3 and 4.2).
//
// One iteration is two groups of three 1-D Gaussian passes (x, y, z; zero
// padding outside the volume; taps summed k = -R..R in FP32):
//   group A  convolves u1 = H I, v1 = H, u2 = (1-H) I, v2 = 1-H   (Eqs. 6, 8-10)
//            the x pass forms the four products from phi and I on load; the z
//            pass divides into the local fits f1 = K*u1 / K*v1 and
//            f2 = K*u2 / K*v2 and stores a = l1 f1 - l2 f2, b = l1 f1^2 - l2 f2^2
//   group B  convolves a and b; the z pass forms
//            g = l1 e1 - l2 e2 = s^2 [ (l1 - l2) K1 I^2 - 2 I K*a + K*b ]
//            (linearity of K applied to the data terms of Eqs. 11-12), the
//            curvature and Laplacian of phi (Eqs. 3-4) and the update of
//            Eqs. (1), (13), (14).
// I is centred and scaled, I~ = (I - m)/s with s a power of two, before the
// iteration; the data terms are invariant to the shift and scale by s^2, so the
// epilogue multiplies g by s^2.  This keeps the cancellation in e_i small.
#include <cmath>

#include "rsf_internal.h"

namespace rsf {

// ------------------------------------------------------------------ set-up

template <typename T>
__global__ void k_stats(const T *__restrict__ vol, long long n, float *__restrict__ part) {
    __shared__ float ss[256], smn[256], smx[256];
    float s = 0.f, mn = INFINITY, mx = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = (float)vol[i];
        s += v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    ss[threadIdx.x] = s;
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            smn[threadIdx.x] = fminf(smn[threadIdx.x], smn[threadIdx.x + w]);
            smx[threadIdx.x] = fmaxf(smx[threadIdx.x], smx[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ss[0];
        part[kStatBlocks + blockIdx.x] = smn[0];
        part[2 * kStatBlocks + blockIdx.x] = smx[0];
    }
}

// One block of kStatBlocks threads: m = mean, s = 2^ceil(log2(max |I - m|)).
__global__ void k_stats_final(const float *__restrict__ part, long long n, float *__restrict__ cs) {
    __shared__ float ss[kStatBlocks], smn[kStatBlocks], smx[kStatBlocks];
    int t = threadIdx.x;
    ss[t] = part[t];
    smn[t] = part[kStatBlocks + t];
    smx[t] = part[2 * kStatBlocks + t];
    __syncthreads();
    for (int w = kStatBlocks / 2; w > 0; w >>= 1) {
        if (t < w) {
            ss[t] += ss[t + w];
            smn[t] = fminf(smn[t], smn[t + w]);
            smx[t] = fmaxf(smx[t], smx[t + w]);
        }
        __syncthreads();
    }
    if (t == 0) {
        float m = ss[0] / (float)n;
        float r = fmaxf(fmaxf(smx[0] - m, m - smn[0]), 1.f);
        int e;
        float fr = frexpf(r, &e);          // r = fr * 2^e, fr in [0.5, 1)
        if (fr == 0.5f) e -= 1;            // exact power of two: keep it
        float s = ldexpf(1.f, e);
        cs[0] = m;
        cs[1] = 1.f / s;
        cs[2] = s * s;
        cs[3] = s;
    }
}

template <typename T>
__global__ void k_center(const T *__restrict__ vol, long long n, const float *__restrict__ cs,
                         float *__restrict__ out) {
    const float m = cs[0], inv_s = cs[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = ((float)vol[i] - m) * inv_s;
}

// ------------------------------------------------------------ x pass

struct LoadH4 {   // u1 = H I, v1 = H, u2 = (1-H) I, v2 = 1-H from phi and the centred image
    const float *phi, *I;
    float eps;
    __device__ void operator()(long long p, float *v) const {
        float ph = __ldg(phi + p), im = __ldg(I + p);
        float h = heaviside(ph, eps), hc = heaviside_c(ph, eps);
        v[0] = h * im;
        v[1] = h;
        v[2] = hc * im;
        v[3] = hc;
    }
};

template <int NF>
struct LoadN {
    const float *a[NF];
    __device__ void operator()(long long p, float *v) const {
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = __ldg(a[f] + p);
    }
};

template <int NF>
struct Outs { float *o[NF]; };

constexpr int kXThreads = 128;

// grid: x = rows (y + z*ny), y = x chunks of kXThreads.
template <int NF, class Load>
__global__ void __launch_bounds__(kXThreads) k_xpass(Load load, Outs<NF> out, Dims d, Taps t) {
    extern __shared__ float sm[];
    const int W = kXThreads + 2 * t.R;
    const long long base = (long long)blockIdx.x * d.nx;
    const int x0 = blockIdx.y * kXThreads;
    for (int i = threadIdx.x; i < W; i += kXThreads) {
        int x = x0 - t.R + i;
        float v[NF];
        if (x >= 0 && x < d.nx) {
            load(base + x, v);
        } else {
#pragma unroll
            for (int f = 0; f < NF; ++f) v[f] = 0.f;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) sm[f * W + i] = v[f];
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= d.nx) return;
    const int T = 2 * t.R + 1;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        float acc = 0.f;
        for (int k = 0; k < T; ++k) acc = fmaf(t.g[k], sm[f * W + threadIdx.x + k], acc);
        out.o[f][base + x] = acc;
    }
}

// ------------------------------------------------------ y / z passes

template <int NF>
struct StoreEpi {
    Outs<NF> out;
    __device__ void operator()(long long p, int, int, int, const float *acc) const {
#pragma unroll
        for (int f = 0; f < NF; ++f) out.o[f][p] = acc[f];
    }
};

// K*1 at (x, y, z) as the product of the three zero-padding profiles.
__device__ __forceinline__ float k_one(const float *prof, const Dims &d, int x, int y, int z) {
    return __ldg(prof + x) * __ldg(prof + d.nx + y) * __ldg(prof + d.nx + d.ny + z);
}

struct FitsEpi {  // group A z epilogue: local fits -> a, b
    float *a, *b;
    float l1, l2;
    float *dump_f1, *dump_f2;  // optional, uncentred fits
    const float *cs;
    __device__ void operator()(long long p, int, int, int, const float *acc) const {
        float f1 = acc[0] / acc[1];
        float f2 = acc[2] / acc[3];
        a[p] = l1 * f1 - l2 * f2;
        b[p] = l1 * (f1 * f1) - l2 * (f2 * f2);
        if (dump_f1) {
            dump_f1[p] = f1 * cs[3] + cs[0];
            dump_f2[p] = f2 * cs[3] + cs[0];
        }
    }
};

// Curvature div(grad phi / (|grad phi| + 1e-10)) and 7-point Laplacian at (x, y, z),
// central differences, reflect-101 boundaries for phi and for the normal.
struct PhiAt {
    const float *phi;
    Dims d;
    __device__ __forceinline__ float operator()(int x, int y, int z) const {
        return __ldg(phi + ((long long)refl101(z, d.nz) * d.ny + refl101(y, d.ny)) * d.nx + refl101(x, d.nx));
    }
};

__device__ __forceinline__ float normal_comp(const PhiAt &at, int qx, int qy, int qz, int axis) {
    qx = refl101(qx, at.d.nx);
    qy = refl101(qy, at.d.ny);
    qz = refl101(qz, at.d.nz);
    float gx = (at(qx + 1, qy, qz) - at(qx - 1, qy, qz)) * 0.5f;
    float gy = (at(qx, qy + 1, qz) - at(qx, qy - 1, qz)) * 0.5f;
    float gz = (at(qx, qy, qz + 1) - at(qx, qy, qz - 1)) * 0.5f;
    float m = sqrtf(gx * gx + gy * gy + gz * gz) + 1e-10f;
    return (axis == 0 ? gx : (axis == 1 ? gy : gz)) / m;
}

struct UpdateEpi {  // group B z epilogue: data term, curvature, Laplacian, update
    const float *phi_in, *I, *prof, *cs;
    float *phi_out;
    Coeffs c;
    Dims d;
    float *dump_g, *dump_k, *dump_l;
    __device__ void operator()(long long p, int x, int y, int z, const float *acc) const {
        const float im = __ldg(I + p);
        const float K1 = k_one(prof, d, x, y, z);
        const float g = cs[2] * ((c.lambda1 - c.lambda2) * K1 * (im * im) - 2.f * im * acc[0] + acc[1]);
        PhiAt at{phi_in, d};
        const float ph = at(x, y, z);
        const float lap = (at(x + 1, y, z) + at(x - 1, y, z) - 2.f * ph) + (at(x, y + 1, z) + at(x, y - 1, z) - 2.f * ph) +
                          (at(x, y, z + 1) + at(x, y, z - 1) - 2.f * ph);
        const float kap = (normal_comp(at, x + 1, y, z, 0) - normal_comp(at, x - 1, y, z, 0)) * 0.5f +
                          (normal_comp(at, x, y + 1, z, 1) - normal_comp(at, x, y - 1, z, 1)) * 0.5f +
                          (normal_comp(at, x, y, z + 1, 2) - normal_comp(at, x, y, z - 1, 2)) * 0.5f;
        const float del = dirac(ph, c.eps);
        phi_out[p] = ph + c.dt * (c.mu * (lap - kap) + del * (c.nu * kap - g));
        if (dump_g) {
            dump_g[p] = g;
            dump_k[p] = kap;
            dump_l[p] = lap;
        }
    }
};

constexpr int kSX = 32, kSY = 8;

// grid: x = ceil(nx/32), y = min(ceil(ny/8), 65535), z = min(nz, 65535); loops cover the rest.
template <int NF, class Epi>
__global__ void __launch_bounds__(kSX * kSY) k_spass(Outs<NF> in, Epi epi, Dims d, Taps t, int axis) {
    const int x = blockIdx.x * kSX + threadIdx.x;
    if (x >= d.nx) return;
    const int na = axis == 1 ? d.ny : d.nz;
    const long long st = axis == 1 ? (long long)d.nx : d.plane;
    for (int z = blockIdx.z; z < d.nz; z += gridDim.z)
        for (int y = blockIdx.y * kSY + threadIdx.y; y < d.ny; y += gridDim.y * kSY) {
            const long long p = (long long)z * d.plane + (long long)y * d.nx + x;
            const int ia = axis == 1 ? y : z;
            float acc[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = 0.f;
            for (int k = -t.R; k <= t.R; ++k) {
                const int j = ia + k;
                if (j < 0 || j >= na) continue;
                const long long q = p + (long long)k * st;
                const float w = t.g[k + t.R];
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] = fmaf(w, __ldg(in.o[f] + q), acc[f]);
            }
            epi(p, x, y, z, acc);
        }
}

// ------------------------------------------------------------- launchers

template <int NF, class Load>
static void launch_x(Load load, Outs<NF> out, const Dims &d, const Taps &t, cudaStream_t s) {
    dim3 grid((unsigned)((long long)d.ny * d.nz), (unsigned)((d.nx + kXThreads - 1) / kXThreads));
    size_t smem = sizeof(float) * NF * (kXThreads + 2 * t.R);
    k_xpass<NF, Load><<<grid, kXThreads, smem, s>>>(load, out, d, t);
}

template <int NF, class Epi>
static void launch_s(Outs<NF> in, Epi epi, const Dims &d, const Taps &t, int axis, cudaStream_t s) {
    dim3 grid((unsigned)((d.nx + kSX - 1) / kSX), (unsigned)std::min((d.ny + kSY - 1) / kSY, 65535),
              (unsigned)std::min(d.nz, 65535));
    k_spass<NF, Epi><<<grid, dim3(kSX, kSY), 0, s>>>(in, epi, d, t, axis);
}

void zero_padding_profiles(const Taps &taps, int nx, int ny, int nz, float *out) {
    // p_a(i) = sum_{k: 0 <= i+k < n_a} g[k], summed in double: K*1 = p_x p_y p_z
    const int n3[3] = {nx, ny, nz};
    size_t o = 0;
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < n3[a]; ++i) {
            double acc = 0.0;
            for (int k = -taps.R; k <= taps.R; ++k)
                if (i + k >= 0 && i + k < n3[a]) acc += (double)taps.g[k + taps.R];
            out[o++] = (float)acc;
        }
}

cudaError_t image_stats(const void *vol, int vt, Fields &f, cudaStream_t s) {
    const Dims &d = f.d;
    switch (vt) {
        case 0: k_stats<uint8_t><<<kStatBlocks, 256, 0, s>>>((const uint8_t *)vol, d.n, f.partials); break;
        case 1: k_stats<uint16_t><<<kStatBlocks, 256, 0, s>>>((const uint16_t *)vol, d.n, f.partials); break;
        default: k_stats<float><<<kStatBlocks, 256, 0, s>>>((const float *)vol, d.n, f.partials);
    }
    k_stats_final<<<1, kStatBlocks, 0, s>>>(f.partials, d.n, f.cs);
    return cudaGetLastError();
}

cudaError_t setup_image(const void *vol, int vt, const Taps &taps, Fields &f, cudaStream_t s, bool centre) {
    const Dims &d = f.d;
    const int eb = 1184;  // elementwise grid: a multiple of the SM count, grid-stride beyond
    switch (vt) {
        case 0:
            k_stats<uint8_t><<<kStatBlocks, 256, 0, s>>>((const uint8_t *)vol, d.n, f.partials);
            break;
        case 1:
            k_stats<uint16_t><<<kStatBlocks, 256, 0, s>>>((const uint16_t *)vol, d.n, f.partials);
            break;
        default:
            k_stats<float><<<kStatBlocks, 256, 0, s>>>((const float *)vol, d.n, f.partials);
    }
    k_stats_final<<<1, kStatBlocks, 0, s>>>(f.partials, d.n, f.cs);
    if (centre) {
        switch (vt) {
            case 0: k_center<uint8_t><<<eb, 256, 0, s>>>((const uint8_t *)vol, d.n, f.cs, f.I); break;
            case 1: k_center<uint16_t><<<eb, 256, 0, s>>>((const uint16_t *)vol, d.n, f.cs, f.I); break;
            default: k_center<float><<<eb, 256, 0, s>>>((const float *)vol, d.n, f.cs, f.I);
        }
    }
    std::vector<float> prof((size_t)d.nx + d.ny + d.nz);
    zero_padding_profiles(taps, d.nx, d.ny, d.nz, prof.data());
    cudaError_t e = cudaMemcpyAsync(f.prof, prof.data(), sizeof(float) * prof.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // the pageable source must stay alive until the copy has been consumed
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t centre_image(const void *vol, int vt, Fields &f, cudaStream_t s) {
    const Dims &d = f.d;
    const int eb = 1184;
    switch (vt) {
        case 0: k_stats<uint8_t><<<kStatBlocks, 256, 0, s>>>((const uint8_t *)vol, d.n, f.partials); break;
        case 1: k_stats<uint16_t><<<kStatBlocks, 256, 0, s>>>((const uint16_t *)vol, d.n, f.partials); break;
        default: k_stats<float><<<kStatBlocks, 256, 0, s>>>((const float *)vol, d.n, f.partials);
    }
    k_stats_final<<<1, kStatBlocks, 0, s>>>(f.partials, d.n, f.cs);
    switch (vt) {
        case 0: k_center<uint8_t><<<eb, 256, 0, s>>>((const uint8_t *)vol, d.n, f.cs, f.I); break;
        case 1: k_center<uint16_t><<<eb, 256, 0, s>>>((const uint16_t *)vol, d.n, f.cs, f.I); break;
        default: k_center<float><<<eb, 256, 0, s>>>((const float *)vol, d.n, f.cs, f.I);
    }
    return cudaGetLastError();
}

cudaError_t iterate_passes(const Taps &t, const Coeffs &c, Fields &f, const float *phi_in, float *phi_out,
                           float *stages, Profiler *prof, cudaStream_t s) {
    const Dims &d = f.d;
    float **T = f.t;
    float *dump = stages;
    const long long n = d.n;
    {
        ProfScope ps(prof, KID_AX);
        launch_x<4>(LoadH4{phi_in, f.I, c.eps}, Outs<4>{{T[0], T[1], T[2], T[3]}}, d, t, s);
    }
    {
        ProfScope ps(prof, KID_AY);
        launch_s<4>(Outs<4>{{T[0], T[1], T[2], T[3]}}, StoreEpi<4>{{{T[4], T[5], T[6], T[7]}}}, d, t, 1, s);
    }
    {
        ProfScope ps(prof, KID_AZ);
        FitsEpi e{T[0], T[1], c.lambda1, c.lambda2, dump ? dump : nullptr, dump ? dump + n : nullptr, f.cs};
        launch_s<4>(Outs<4>{{T[4], T[5], T[6], T[7]}}, e, d, t, 2, s);
    }
    {
        ProfScope ps(prof, KID_BX);
        launch_x<2>(LoadN<2>{{T[0], T[1]}}, Outs<2>{{T[2], T[3]}}, d, t, s);
    }
    {
        ProfScope ps(prof, KID_BY);
        launch_s<2>(Outs<2>{{T[2], T[3]}}, StoreEpi<2>{{{T[4], T[5]}}}, d, t, 1, s);
    }
    {
        ProfScope ps(prof, KID_BZ);
        UpdateEpi e{phi_in, f.I, f.prof, f.cs, phi_out, c, d,
                    dump ? dump + 2 * n : nullptr, dump ? dump + 3 * n : nullptr, dump ? dump + 4 * n : nullptr};
        launch_s<2>(Outs<2>{{T[4], T[5]}}, e, d, t, 2, s);
    }
    return cudaGetLastError();
}

}  // namespace rsf
