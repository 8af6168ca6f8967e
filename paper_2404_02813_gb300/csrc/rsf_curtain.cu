// rsf_curtain.cu -- rsf_evolve_curtain: the volume-level parallelism of
// arXiv 2404.02813, Sec. 4.1.  The volume is divided into overlapping
// sub-volumes, every sub-volume is evolved as a volume of its own (all of them
// together, through rsf_evolve_batch), and neighbouring results are merged by
// linear interpolation across the overlap (the curtain).
//
// Layout along each axis of length n: sub-volumes of `edge` voxels start at
// multiples of edge - curtain and the last one is moved to end at n (a single
// sub-volume when edge >= n).  Sub-volume b carries the weight
// w_b(x) = prod over axes of h_b(x_a), with h = 1 inside, rising linearly
// over the `curtain` voxels next to each face interior to the volume:
// h = min(1, (x - s + 1/2) / curtain) after a start face s > 0 and
// min(1, (e - x - 1/2) / curtain) before an end face e < n.  The merged phi is
// sum_b w_b phi_b / sum_b w_b; across an overlap of exactly `curtain` voxels
// this is the linear interpolation between the two neighbours.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "rsf.h"
#include "rsf_ctx.h"

namespace {

constexpr int kMaxCover = 4;  // sub-volumes covering one coordinate of an axis (at most 3 when curtain <= edge/2)

std::vector<int> starts_of(int n, int edge, int curtain) {
    std::vector<int> s;
    if (edge >= n) {
        s.push_back(0);
        return s;
    }
    for (int a = 0; a < n - edge; a += edge - curtain) s.push_back(a);
    s.push_back(n - edge);
    return s;
}

// Per coordinate of one axis: the covering sub-volumes, the coordinate local to
// each and the axis factor h of its weight.
struct AxisTable {
    std::vector<int> count, box, local;
    std::vector<float> weight;
};

bool axis_table(int n, int edge, int curtain, const std::vector<int> &starts, AxisTable *t) {
    t->count.assign(n, 0);
    t->box.assign((size_t)n * kMaxCover, 0);
    t->local.assign((size_t)n * kMaxCover, 0);
    t->weight.assign((size_t)n * kMaxCover, 0.f);
    for (int k = 0; k < (int)starts.size(); ++k) {
        const int s = starts[k], e = std::min(s + edge, n);
        for (int x = s; x < e; ++x) {
            double h = 1.0;
            if (s > 0) h = std::min(h, (x - s + 0.5) / curtain);
            if (e < n) h = std::min(h, (e - x - 0.5) / curtain);
            const int c = t->count[x]++;
            if (c >= kMaxCover) return false;
            t->box[(size_t)x * kMaxCover + c] = k;
            t->local[(size_t)x * kMaxCover + c] = x - s;
            t->weight[(size_t)x * kMaxCover + c] = (float)std::max(h, 0.0);
        }
    }
    return true;
}

template <class T>
__global__ void k_gather(const T *__restrict__ src, T *__restrict__ dst, int nx, int ny, int x0, int y0, int z0,
                         int bx, int by, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % bx);
        const long long r = i / bx;
        const int y = (int)(r % by), z = (int)(r / by);
        dst[i] = src[((long long)(z0 + z) * ny + (y0 + y)) * nx + x0 + x];
    }
}

struct MergeArgs {
    const float *const *phi;  // per sub-volume (bz, by, bx) in z-major order, its evolved phi
    const int *ext[3];        // sub-volume extent per axis index (x, y, z)
    const int *count[3], *box[3], *local[3];
    const float *weight[3];
    int n[3], nb[3];
};

__global__ void k_merge(MergeArgs a, float *__restrict__ out) {
    const long long total = (long long)a.n[0] * a.n[1] * a.n[2];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.n[0]);
        const long long r = i / a.n[0];
        const int y = (int)(r % a.n[1]), z = (int)(r / a.n[1]);
        float num = 0.f, den = 0.f;
        const int cz = a.count[2][z], cy = a.count[1][y], cx = a.count[0][x];
        for (int iz = 0; iz < cz; ++iz) {
            const int kz = a.box[2][z * kMaxCover + iz], lz = a.local[2][z * kMaxCover + iz];
            const float wz = a.weight[2][z * kMaxCover + iz];
            for (int iy = 0; iy < cy; ++iy) {
                const int ky = a.box[1][y * kMaxCover + iy], ly = a.local[1][y * kMaxCover + iy];
                const float wzy = wz * a.weight[1][y * kMaxCover + iy];
                const int ey = a.ext[1][ky];
                for (int ix = 0; ix < cx; ++ix) {
                    const int kx = a.box[0][x * kMaxCover + ix], lx = a.local[0][x * kMaxCover + ix];
                    const float w = wzy * a.weight[0][x * kMaxCover + ix];
                    const float *p = a.phi[((long long)kz * a.nb[1] + ky) * a.nb[0] + kx];
                    num = fmaf(w, p[((long long)lz * ey + ly) * a.ext[0][kx] + lx], num);
                    den += w;
                }
            }
        }
        out[i] = num / den;
    }
}

}  // namespace

extern "C" rsf_status rsf_evolve_curtain(rsf_ctx *c, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny,
                                         int64_t nz, const float *phi0, float *phi_out, float sigma, float eps,
                                         float lambda1, float lambda2, float nu, float mu, float dt, int32_t iters,
                                         int32_t edge, int32_t curtain) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    rsf_status st = check_args(volume, vt, nx, ny, nz, phi0, phi_out, sigma, eps, dt, iters);
    if (st) return st;
    if (edge < 4) return fail(RSF_E_INVAL, "sub-volume edge %d is below 4", (int)edge);
    if (curtain < 1 || 2 * curtain > edge)
        return fail(RSF_E_INVAL, "curtain %d must lie in [1, edge/2] (edge %d)", (int)curtain, (int)edge);
    const int n[3] = {(int)nx, (int)ny, (int)nz};
    std::vector<int> starts[3];
    AxisTable tab[3];
    for (int a = 0; a < 3; ++a) {
        starts[a] = starts_of(n[a], edge, curtain);
        if (!axis_table(n[a], edge, curtain, starts[a], &tab[a]))
            return fail(RSF_E_INVAL, "more than %d sub-volumes cover one coordinate", kMaxCover);
    }
    const int nb[3] = {(int)starts[0].size(), (int)starts[1].size(), (int)starts[2].size()};
    const long long nbox = (long long)nb[0] * nb[1] * nb[2];
    const size_t es = dtype_size(vt);
    const long long nvox = (long long)nx * ny * nz;

    // device memory: sub-volume images and phi, staging of host inputs and output, tables
    std::vector<long long> bvox(nbox);
    size_t bytes = 0;
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    for (int kz = 0; kz < nb[2]; ++kz)
        for (int ky = 0; ky < nb[1]; ++ky)
            for (int kx = 0; kx < nb[0]; ++kx) {
                const long long v = (long long)std::min(edge, n[0]) * std::min(edge, n[1]) * std::min(edge, n[2]);
                bvox[((long long)kz * nb[1] + ky) * nb[0] + kx] = v;
                bytes += align(es * v) + align(sizeof(float) * v);
            }
    const bool host_vol = !on_device(volume), host_phi = !on_device(phi0), host_out = !on_device(phi_out);
    if (host_vol) bytes += align(es * nvox);
    if (host_phi) bytes += align(sizeof(float) * nvox);
    if (host_out) bytes += align(sizeof(float) * nvox);
    size_t tab_bytes = sizeof(float *) * nbox;
    for (int a = 0; a < 3; ++a)
        tab_bytes += sizeof(int) * (nb[a] + n[a] * (1 + 2 * kMaxCover)) + sizeof(float) * n[a] * kMaxCover;
    bytes += align(tab_bytes) + 1024;
    void *mem = nullptr;
    if ((st = dev_alloc(c, &mem, bytes))) return st;
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

    std::vector<rsf_brick> bricks(nbox);
    std::vector<const float *> phis(nbox);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        RSF_CUDA(cudaSetDevice(c->device));
        const void *vol = volume;
        const float *ph0 = phi0;
        if (host_vol) {
            void *d = take(es * nvox);
            RSF_CUDA(xfer(d, volume, es * nvox, c->stream));
            vol = d;
        }
        if (host_phi) {
            float *d = reinterpret_cast<float *>(take(sizeof(float) * nvox));
            RSF_CUDA(xfer(d, phi0, sizeof(float) * nvox, c->stream));
            ph0 = d;
        }
        for (int kz = 0; kz < nb[2]; ++kz)
            for (int ky = 0; ky < nb[1]; ++ky)
                for (int kx = 0; kx < nb[0]; ++kx) {
                    const long long id = ((long long)kz * nb[1] + ky) * nb[0] + kx;
                    const int bx = std::min(edge, n[0]), by = std::min(edge, n[1]), bz = std::min(edge, n[2]);
                    const int x0 = starts[0][kx], y0 = starts[1][ky], z0 = starts[2][kz];
                    void *img = take(es * bvox[id]);
                    float *ph = reinterpret_cast<float *>(take(sizeof(float) * bvox[id]));
                    const int grid = (int)std::min<long long>(1216, (bvox[id] + 255) / 256);
                    switch (vt) {
                        case RSF_U8:
                            k_gather<<<grid, 256, 0, c->stream>>>(static_cast<const uint8_t *>(vol),
                                                                  static_cast<uint8_t *>(img), n[0], n[1], x0, y0,
                                                                  z0, bx, by, bvox[id]);
                            break;
                        case RSF_U16:
                            k_gather<<<grid, 256, 0, c->stream>>>(static_cast<const uint16_t *>(vol),
                                                                  static_cast<uint16_t *>(img), n[0], n[1], x0, y0,
                                                                  z0, bx, by, bvox[id]);
                            break;
                        default:
                            k_gather<<<grid, 256, 0, c->stream>>>(static_cast<const float *>(vol),
                                                                  static_cast<float *>(img), n[0], n[1], x0, y0, z0,
                                                                  bx, by, bvox[id]);
                    }
                    k_gather<<<grid, 256, 0, c->stream>>>(ph0, ph, n[0], n[1], x0, y0, z0, bx, by, bvox[id]);
                    RSF_CUDA(cudaGetLastError());
                    bricks[id] = rsf_brick{img, vt, bx, by, bz, ph, ph, sigma, eps, lambda1, lambda2, nu, mu, dt,
                                           iters};
                    phis[id] = ph;
                }
    }
    // every sub-volume evolved as its own volume, all together (same stream, so
    // the gathers above are ordered before the batch's first launch)
    if ((st = rsf_evolve_batch(c, bricks.data(), (int32_t)nbox))) return st;

    std::lock_guard<std::mutex> lk(c->mu);
    float *out = host_out ? reinterpret_cast<float *>(take(sizeof(float) * nvox)) : phi_out;
    char *tb = take(tab_bytes);
    std::vector<char> host_tab(tab_bytes);
    size_t off = 0;
    auto put = [&](const void *src, size_t b) {
        memcpy(host_tab.data() + off, src, b);
        const char *d = tb + off;
        off += b;
        return d;
    };
    MergeArgs m{};
    m.phi = reinterpret_cast<const float *const *>(put(phis.data(), sizeof(float *) * nbox));
    for (int a = 0; a < 3; ++a) {
        std::vector<int> ext(nb[a], std::min(edge, n[a]));
        m.ext[a] = reinterpret_cast<const int *>(put(ext.data(), sizeof(int) * nb[a]));
        m.count[a] = reinterpret_cast<const int *>(put(tab[a].count.data(), sizeof(int) * n[a]));
        m.box[a] = reinterpret_cast<const int *>(put(tab[a].box.data(), sizeof(int) * n[a] * kMaxCover));
        m.local[a] = reinterpret_cast<const int *>(put(tab[a].local.data(), sizeof(int) * n[a] * kMaxCover));
        m.weight[a] = reinterpret_cast<const float *>(put(tab[a].weight.data(), sizeof(float) * n[a] * kMaxCover));
        m.n[a] = n[a];
        m.nb[a] = nb[a];
    }
    RSF_CUDA(cudaMemcpyAsync(tb, host_tab.data(), off, cudaMemcpyHostToDevice, c->stream));
    k_merge<<<(int)std::min<long long>(4864, (nvox + 255) / 256), 256, 0, c->stream>>>(m, out);
    RSF_CUDA(cudaGetLastError());
    if (host_out) RSF_CUDA(xfer(phi_out, out, sizeof(float) * nvox, c->stream));
    RSF_CUDA(cudaStreamSynchronize(c->stream));
    return RSF_OK;
}
