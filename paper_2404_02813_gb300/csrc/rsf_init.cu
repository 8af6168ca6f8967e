// rsf_init.cu -- rsf_init_phi0: the seed initialisation of arXiv 2404.02813,
// Sec. 4.3.  Blob seeds come from the determinant of the Hessian in every z
// slice; phi0 is r0 minus the Euclidean distance to the nearest seed (the
// distance the paper's fast sweeping approximates, here exact).
//
//   taps       g_k = exp(-k^2/2s^2)/sum, g'_k = -(k/s^2) g_k,
//              g''_k = (k^2/s^4 - 1/s^2) g_k, k = -R..R, R = round(3 s)
//   filters    in-slice correlation with zero padding: I_xx = (g'' in x, g in y),
//              I_yy = (g in x, g'' in y), I_xy = (g' in x, g' in y)
//   response   D = s^4 (I_xx I_yy - I_xy^2) where I_xx + I_yy < 0, else -inf
//   seeds      D > t * (maximum of D over the slice), that maximum > 0, and D
//              above D at each existing in-slice neighbour (3 x 3)
//   phi0       r0 - sqrt(min over seeds of the squared distance); the squared
//              distances are integers below 2^24, exact in FP32, built by one
//              pass per axis: d_a(i) = min_j (d_{a-1}(j) + (i - j)^2) along the line.
// This is one-time set-up, not the per-iteration path: the kernels are plain
// one-thread-per-voxel loops over taps or lines.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "rsf.h"
#include "rsf_ctx.h"

namespace {

constexpr int kMaxR = 16;

struct DerivTaps {
    int R;
    float g[2 * kMaxR + 1], g1[2 * kMaxR + 1], g2[2 * kMaxR + 1];
};

DerivTaps make_deriv_taps(float s) {
    DerivTaps t{};
    t.R = (int)std::floor(3.0 * s + 0.5);
    double w[2 * kMaxR + 1], sum = 0.0;
    for (int k = -t.R; k <= t.R; ++k) sum += (w[k + t.R] = std::exp(-(double)k * k / (2.0 * s * s)));
    for (int k = -t.R; k <= t.R; ++k) {
        const double g = w[k + t.R] / sum;
        t.g[k + t.R] = (float)g;
        t.g1[k + t.R] = (float)(-(k / ((double)s * s)) * g);
        t.g2[k + t.R] = (float)(((double)k * k / std::pow((double)s, 4) - 1.0 / ((double)s * s)) * g);
    }
    return t;
}

template <class T>
__global__ void k_hx(const T *__restrict__ img, float *__restrict__ t0, float *__restrict__ t1,
                     float *__restrict__ t2, int nx, long long n, DerivTaps tp) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        float a = 0.f, b = 0.f, c = 0.f;
        for (int k = -tp.R; k <= tp.R; ++k) {
            const int xx = x + k;
            if (xx < 0 || xx >= nx) continue;
            const float v = (float)img[i + k];
            a = fmaf(tp.g[k + tp.R], v, a);
            b = fmaf(tp.g1[k + tp.R], v, b);
            c = fmaf(tp.g2[k + tp.R], v, c);
        }
        t0[i] = a;
        t1[i] = b;
        t2[i] = c;
    }
}

__global__ void k_hy(const float *__restrict__ t0, const float *__restrict__ t1, const float *__restrict__ t2,
                     float *__restrict__ D, int nx, int ny, long long n, DerivTaps tp, float s4) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)((i / nx) % ny);
        float ixx = 0.f, iyy = 0.f, ixy = 0.f;
        for (int k = -tp.R; k <= tp.R; ++k) {
            const int yy = y + k;
            if (yy < 0 || yy >= ny) continue;
            const long long j = i + (long long)k * nx;
            ixx = fmaf(tp.g[k + tp.R], t2[j], ixx);
            iyy = fmaf(tp.g2[k + tp.R], t0[j], iyy);
            ixy = fmaf(tp.g1[k + tp.R], t1[j], ixy);
        }
        D[i] = ixx + iyy < 0.f ? s4 * (ixx * iyy - ixy * ixy) : -INFINITY;
    }
}

__global__ void k_slice_max(const float *__restrict__ D, float *__restrict__ smax, long long plane) {
    __shared__ float red[256];
    const float *p = D + (long long)blockIdx.x * plane;
    float m = -INFINITY;
    for (long long i = threadIdx.x; i < plane; i += blockDim.x) m = fmaxf(m, p[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) smax[blockIdx.x] = red[0];
}

__global__ void k_seeds(const float *__restrict__ D, const float *__restrict__ smax, uint8_t *__restrict__ mask,
                        float *__restrict__ d2, unsigned long long *__restrict__ count, int nx, int ny, long long n,
                        float t) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const float v = D[i], m = smax[z];
        bool seed = m > 0.f && v > t * m;
        for (int dy = -1; dy <= 1 && seed; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int xx = x + dx, yy = y + dy;
                if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
                if (!(v > D[i + (long long)dy * nx + dx])) {
                    seed = false;
                    break;
                }
            }
        mask[i] = seed ? 1 : 0;
        d2[i] = seed ? 0.f : INFINITY;
        if (seed) atomicAdd(count, 1ULL);
    }
}

// One axis of the squared distance transform: out(i) = min_j in(j) + (i - j)^2
// along the line through i (stride `stride`, length `len`).
__global__ void k_edt_axis(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int axis,
                           long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const int pos = axis == 0 ? x : (axis == 1 ? y : z);
        const long long stride = axis == 0 ? 1 : (axis == 1 ? (long long)nx : (long long)nx * ny);
        const int len = axis == 0 ? nx : (axis == 1 ? ny : (int)(n / ((long long)nx * ny)));
        const float *line = in + (i - (long long)pos * stride);
        float best = INFINITY;
        for (int j = 0; j < len; ++j) {
            const float d = (float)(pos - j);
            best = fminf(best, line[(long long)j * stride] + d * d);
        }
        out[i] = best;
    }
}

__global__ void k_phi0(const float *__restrict__ d2, float *__restrict__ phi, long long n, float r0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        phi[i] = r0 - sqrtf(d2[i]);
}

}  // namespace

extern "C" rsf_status rsf_init_phi0(rsf_ctx *c, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                                    float blob_sigma, float rel_threshold, float r0, float *phi0_out,
                                    int64_t *nseeds, uint8_t *seeds_out, float *response_out) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!volume || !phi0_out || !nseeds) return fail(RSF_E_INVAL, "null volume, phi0_out or nseeds pointer");
    if (vt != RSF_U8 && vt != RSF_U16 && vt != RSF_F32) return fail(RSF_E_INVAL, "unknown volume dtype %d", (int)vt);
    if (nx < 4 || ny < 4 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
        return fail(RSF_E_INVAL, "dimensions must lie in [4, 2^20] (x, y) and [1, 2^20] (z)");
    if ((double)nx * ny * nz > 17179869184.0) return fail(RSF_E_INVAL, "nx*ny*nz exceeds 2^34");
    if ((double)(nx - 1) * (nx - 1) + (double)(ny - 1) * (ny - 1) + (double)(nz - 1) * (nz - 1) >= 16777216.0)
        return fail(RSF_E_INVAL, "squared distances would exceed 2^24 (exact FP32 range)");
    if (!(blob_sigma > 0.f) || std::floor(3.0 * blob_sigma + 0.5) > kMaxR)
        return fail(RSF_E_INVAL, "blob sigma must be positive with round(3 sigma) <= %d", kMaxR);
    if (!(rel_threshold >= 0.f && rel_threshold < 1.f)) return fail(RSF_E_INVAL, "relative threshold must lie in [0, 1)");
    if (!(r0 > 0.f) || !std::isfinite(r0)) return fail(RSF_E_INVAL, "r0 must be positive and finite");

    const long long n = nx * ny * nz, plane = nx * ny;
    const size_t es = dtype_size(vt);
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    const bool host_vol = !on_device(volume), host_phi = !on_device(phi0_out);
    size_t bytes = 4 * align(sizeof(float) * n) + align(n) + align(sizeof(float) * nz) + 256;
    if (host_vol) bytes += align(es * n);
    void *mem = nullptr;
    rsf_status st = dev_alloc(c, &mem, bytes);
    if (st) return st;
    struct Release {
        rsf_ctx *c;
        void *p;
        size_t b;
        ~Release() { dev_free(c, p, b); }
    } release{c, mem, bytes};
    char *p = static_cast<char *>(mem);
    auto take = [&](size_t b) {
        char *q = p;
        p += align(b);
        return q;
    };
    float *t0 = reinterpret_cast<float *>(take(sizeof(float) * n));
    float *t1 = reinterpret_cast<float *>(take(sizeof(float) * n));
    float *t2 = reinterpret_cast<float *>(take(sizeof(float) * n));
    float *D = reinterpret_cast<float *>(take(sizeof(float) * n));
    uint8_t *mask = reinterpret_cast<uint8_t *>(take(n));
    float *smax = reinterpret_cast<float *>(take(sizeof(float) * nz));
    unsigned long long *count = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));

    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const void *img = volume;
    if (host_vol) {
        void *d = take(es * n);
        RSF_CUDA(xfer(d, volume, es * n, s));
        img = d;
    }
    const DerivTaps tp = make_deriv_taps(blob_sigma);
    const int grid = (int)std::min<long long>(4864, (n + 255) / 256);
    switch (vt) {
        case RSF_U8: k_hx<<<grid, 256, 0, s>>>(static_cast<const uint8_t *>(img), t0, t1, t2, (int)nx, n, tp); break;
        case RSF_U16: k_hx<<<grid, 256, 0, s>>>(static_cast<const uint16_t *>(img), t0, t1, t2, (int)nx, n, tp); break;
        default: k_hx<<<grid, 256, 0, s>>>(static_cast<const float *>(img), t0, t1, t2, (int)nx, n, tp);
    }
    const float s2 = blob_sigma * blob_sigma;
    k_hy<<<grid, 256, 0, s>>>(t0, t1, t2, D, (int)nx, (int)ny, n, tp, s2 * s2);
    k_slice_max<<<(unsigned)nz, 256, 0, s>>>(D, smax, plane);
    RSF_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    k_seeds<<<grid, 256, 0, s>>>(D, smax, mask, t0, count, (int)nx, (int)ny, n, rel_threshold);
    k_edt_axis<<<grid, 256, 0, s>>>(t0, t1, (int)nx, (int)ny, 0, n);
    k_edt_axis<<<grid, 256, 0, s>>>(t1, t2, (int)nx, (int)ny, 1, n);
    k_edt_axis<<<grid, 256, 0, s>>>(t2, t0, (int)nx, (int)ny, 2, n);
    RSF_CUDA(cudaGetLastError());
    unsigned long long found = 0;
    RSF_CUDA(cudaMemcpyAsync(&found, count, sizeof(found), cudaMemcpyDeviceToHost, s));
    RSF_CUDA(cudaStreamSynchronize(s));
    *nseeds = (int64_t)found;
    if (response_out) RSF_CUDA(xfer(response_out, D, sizeof(float) * n, s));
    if (seeds_out) RSF_CUDA(xfer(seeds_out, mask, n, s));
    if (found == 0) {
        RSF_CUDA(cudaStreamSynchronize(s));
        return fail(RSF_E_INVAL, "no seed found (relative threshold %g)", (double)rel_threshold);
    }
    float *phi = host_phi ? t1 : phi0_out;
    k_phi0<<<grid, 256, 0, s>>>(t0, phi, n, r0);
    RSF_CUDA(cudaGetLastError());
    if (host_phi) RSF_CUDA(xfer(phi0_out, phi, sizeof(float) * n, s));
    RSF_CUDA(cudaStreamSynchronize(s));
    return RSF_OK;
}

// ------------------------------------------------------------ validation

namespace {

// Counts |phi > 0|, |truth != 0| and their intersection (warp sums, one atomic
// per warp per count).
__global__ void k_overlap(const float *__restrict__ phi, const uint8_t *__restrict__ truth, long long n,
                          unsigned long long *__restrict__ out) {
    unsigned long long a = 0, b = 0, c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const bool s = phi[i] > 0.f, t = truth[i] != 0;
        a += s;
        b += t;
        c += s && t;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 0, a);
        atomicAdd(out + 1, b);
        atomicAdd(out + 2, c);
    }
}

}  // namespace

extern "C" rsf_status rsf_overlap(rsf_ctx *c, const float *phi, const uint8_t *truth, int64_t n, int64_t counts[3]) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!phi || !truth || !counts) return fail(RSF_E_INVAL, "null phi, truth or counts pointer");
    if (n < 0 || n > (int64_t)1 << 34) return fail(RSF_E_INVAL, "n must lie in [0, 2^34]");
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    const bool host_phi = !on_device(phi), host_truth = !on_device(truth);
    size_t bytes = 256 + (host_phi ? align(sizeof(float) * n) : 0) + (host_truth ? align(n) : 0);
    void *mem = nullptr;
    rsf_status st = dev_alloc(c, &mem, bytes);
    if (st) return st;
    struct Release {
        rsf_ctx *c;
        void *p;
        size_t b;
        ~Release() { dev_free(c, p, b); }
    } release{c, mem, bytes};
    char *p = static_cast<char *>(mem);
    unsigned long long *out = reinterpret_cast<unsigned long long *>(p);
    p += 256;
    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    if (host_phi) {
        RSF_CUDA(xfer(p, phi, sizeof(float) * n, s));
        phi = reinterpret_cast<const float *>(p);
        p += align(sizeof(float) * n);
    }
    if (host_truth) {
        RSF_CUDA(xfer(p, truth, n, s));
        truth = reinterpret_cast<const uint8_t *>(p);
    }
    RSF_CUDA(cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), s));
    if (n > 0) {
        k_overlap<<<(int)std::min<long long>(1216, (n + 255) / 256), 256, 0, s>>>(phi, truth, n, out);
        RSF_CUDA(cudaGetLastError());
    }
    unsigned long long h[3];
    RSF_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    RSF_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) counts[k] = (int64_t)h[k];
    return RSF_OK;
}
