// rsf_iso.cu -- rsf_isosurface: the phi = iso surface as triangles (the
// surfaces the paper renders, Figs. 8-9), by marching tetrahedra.
//
// Every voxel cube (x..x+1, y..y+1, z..z+1) is split into six tetrahedra along
// its main diagonal, one per order (a, b, c) of the axes: corners 0, e_a,
// e_a + e_b, (1,1,1).  In a tetrahedron with k corners where phi > iso: k = 0
// or 4, no triangle; k = 1 or 3, one triangle on the three edges joining the
// odd corner to the others; k = 2, two triangles on the four crossed edges
// (the quadrilateral p0 p1 q1 q0 split along p0-q1, with a = the inside
// corners, b = the outside ones, p_j the crossing of (a0, b_j), q_j that of
// (a1, b_j)).  An edge is crossed at p + t (q - p), t = (iso - phi_p) /
// (phi_q - phi_p), with p the corner of smaller grid index, so an edge shared
// by several tetrahedra gives one point.  The normal (v1 - v0) x (v2 - v0)
// points from phi > iso towards phi < iso (v1, v2 swapped otherwise).  Each
// triangle carries the key (cube index) * 12 + (tetrahedron) * 2 + (triangle),
// cube index (z * (ny-1) + y) * (nx-1) + x: the set of triangles is unique,
// their order in the output is not.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "rsf.h"
#include "rsf_ctx.h"

namespace {

// corner c of a cube is (c & 1, (c >> 1) & 1, c >> 2); tetrahedron t's corners
// for the axis orders (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x)
__constant__ int kTetra[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

struct Emit {
    float *tri;            // 9 floats per triangle, or null (count only)
    long long *keys;       // or null
    long long cap;
};

__device__ __forceinline__ float3 corner_pos(int x, int y, int z, int c) {
    return make_float3((float)(x + (c & 1)), (float)(y + ((c >> 1) & 1)), (float)(z + (c >> 2)));
}

// crossing of edge (i, j), from the corner of smaller index (= smaller grid index)
__device__ __forceinline__ float3 cut(const float *v, int x, int y, int z, int i, int j, float iso) {
    if (i > j) {
        const int s = i;
        i = j;
        j = s;
    }
    const float t = (iso - v[i]) / (v[j] - v[i]);
    const float3 p = corner_pos(x, y, z, i), q = corner_pos(x, y, z, j);
    return make_float3(fmaf(t, q.x - p.x, p.x), fmaf(t, q.y - p.y, p.y), fmaf(t, q.z - p.z, p.z));
}

__device__ __forceinline__ void put(const Emit &e, long long slot, long long key, float3 a, float3 b, float3 c,
                                    float3 out_dir) {
    const float3 u = make_float3(b.x - a.x, b.y - a.y, b.z - a.z), w = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    const float3 n = make_float3(u.y * w.z - u.z * w.y, u.z * w.x - u.x * w.z, u.x * w.y - u.y * w.x);
    if (n.x * out_dir.x + n.y * out_dir.y + n.z * out_dir.z < 0.f) {
        const float3 s = b;
        b = c;
        c = s;
    }
    if (slot >= e.cap) return;
    float *o = e.tri + slot * 9;
    o[0] = a.x; o[1] = a.y; o[2] = a.z;
    o[3] = b.x; o[4] = b.y; o[5] = b.z;
    o[6] = c.x; o[7] = c.y; o[8] = c.z;
    if (e.keys) e.keys[slot] = key;
}

__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

// Triangles of cube (x, y, z): counted, or written from `slot` on.
__device__ int cube(const float *v, int x, int y, int z, float iso, long long key0, const Emit *e, long long slot) {
    int n = 0;
    for (int t = 0; t < 6; ++t) {
        const int *c = kTetra[t];
        int mask = 0;
        for (int k = 0; k < 4; ++k) mask |= (v[c[k]] > iso ? 1 : 0) << k;
        const int k = __popc(mask);
        if (k == 0 || k == 4) continue;
        if (k == 1 || k == 3) {
            if (e) {
                int odd = 0;
                for (int q = 0; q < 4; ++q)
                    if (((mask >> q) & 1) == (k == 1 ? 1 : 0)) odd = q;
                int o[3], m = 0;
                for (int q = 0; q < 4; ++q)
                    if (q != odd) o[m++] = q;
                const float3 a = cut(v, x, y, z, c[odd], c[o[0]], iso), b = cut(v, x, y, z, c[odd], c[o[1]], iso),
                             d = cut(v, x, y, z, c[odd], c[o[2]], iso);
                const float3 po = corner_pos(x, y, z, c[odd]);
                put(*e, slot + n, key0 + 2 * t, a, b, d, k == 1 ? sub(a, po) : sub(po, a));
            }
            n += 1;
        } else {
            if (e) {
                int ia[2], ib[2], na = 0, nb = 0;
                for (int q = 0; q < 4; ++q) {
                    if ((mask >> q) & 1) ia[na++] = q;
                    else ib[nb++] = q;
                }
                const float3 p0 = cut(v, x, y, z, c[ia[0]], c[ib[0]], iso), p1 = cut(v, x, y, z, c[ia[0]], c[ib[1]], iso);
                const float3 q0 = cut(v, x, y, z, c[ia[1]], c[ib[0]], iso), q1 = cut(v, x, y, z, c[ia[1]], c[ib[1]], iso);
                const float3 a0 = corner_pos(x, y, z, c[ia[0]]), a1 = corner_pos(x, y, z, c[ia[1]]);
                const float3 b0 = corner_pos(x, y, z, c[ib[0]]), b1 = corner_pos(x, y, z, c[ib[1]]);
                const float3 dir = make_float3(0.5f * (b0.x + b1.x - a0.x - a1.x), 0.5f * (b0.y + b1.y - a0.y - a1.y),
                                               0.5f * (b0.z + b1.z - a0.z - a1.z));
                put(*e, slot + n, key0 + 2 * t, p0, p1, q1, dir);
                put(*e, slot + n + 1, key0 + 2 * t + 1, p0, q1, q0, dir);
            }
            n += 2;
        }
    }
    return n;
}

// One thread per cube: count, reserve slots with one atomic per warp, emit.
__global__ void k_iso(const float *__restrict__ phi, int nx, int ny, int nz, float iso, Emit e,
                      unsigned long long *__restrict__ total) {
    const long long ncube = (long long)(nx - 1) * (ny - 1) * (nz - 1);
    const long long span = (ncube + 31) / 32 * 32;  // every lane of a warp runs the same trips
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < span; i += (long long)gridDim.x * blockDim.x) {
        float v[8];
        int x = 0, y = 0, z = 0, n = 0;
        if (i < ncube) {
            x = (int)(i % (nx - 1));
            const long long r = i / (nx - 1);
            y = (int)(r % (ny - 1));
            z = (int)(r / (ny - 1));
            for (int c = 0; c < 8; ++c)
                v[c] = phi[((long long)(z + (c >> 2)) * ny + (y + ((c >> 1) & 1))) * nx + x + (c & 1)];
            n = cube(v, x, y, z, iso, i * 12, nullptr, 0);
        }
        const int lane = threadIdx.x & 31;
        int incl = n;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(total, (unsigned long long)incl);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (n > 0 && e.tri) cube(v, x, y, z, iso, i * 12, &e, (long long)base + incl - n);
    }
}

}  // namespace

extern "C" rsf_status rsf_isosurface(rsf_ctx *c, const float *phi, int64_t nx, int64_t ny, int64_t nz, float iso,
                                     float *triangles, int64_t *keys, int64_t capacity, int64_t *ntriangles) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!phi || !ntriangles) return fail(RSF_E_INVAL, "null phi or ntriangles pointer");
    if (nx < 2 || ny < 2 || nz < 2 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
        return fail(RSF_E_INVAL, "dimensions must lie in [2, 2^20]");
    if ((double)nx * ny * nz > 17179869184.0) return fail(RSF_E_INVAL, "nx*ny*nz exceeds 2^34");
    if (capacity < 0 || (capacity > 0 && !triangles)) return fail(RSF_E_INVAL, "capacity without a triangle buffer");
    if (!std::isfinite(iso)) return fail(RSF_E_INVAL, "iso must be finite");
    const long long n = nx * ny * nz;
    auto align = [](size_t b) { return (b + 255) & ~size_t(255); };
    const bool host_phi = !on_device(phi);
    const bool host_tri = capacity > 0 && !on_device(triangles);
    const bool host_keys = capacity > 0 && keys && !on_device(keys);
    size_t bytes = 256;
    if (host_phi) bytes += align(sizeof(float) * n);
    if (host_tri) bytes += align(sizeof(float) * 9 * (size_t)capacity);
    if (host_keys) bytes += align(sizeof(long long) * (size_t)capacity);
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
    unsigned long long *total = reinterpret_cast<unsigned long long *>(p);
    p += 256;
    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const float *ph = phi;
    if (host_phi) {
        RSF_CUDA(xfer(p, phi, sizeof(float) * n, s));
        ph = reinterpret_cast<const float *>(p);
        p += align(sizeof(float) * n);
    }
    Emit e{nullptr, nullptr, capacity};
    if (capacity > 0) {
        e.tri = host_tri ? reinterpret_cast<float *>(p) : triangles;
        if (host_tri) p += align(sizeof(float) * 9 * (size_t)capacity);
        e.keys = keys ? (host_keys ? reinterpret_cast<long long *>(p) : reinterpret_cast<long long *>(keys)) : nullptr;
    }
    RSF_CUDA(cudaMemsetAsync(total, 0, sizeof(unsigned long long), s));
    const long long ncube = (nx - 1) * (ny - 1) * (nz - 1);
    k_iso<<<(int)std::min<long long>(4864, (ncube + 255) / 256), 256, 0, s>>>(ph, (int)nx, (int)ny, (int)nz, iso, e,
                                                                              total);
    RSF_CUDA(cudaGetLastError());
    unsigned long long count = 0;
    RSF_CUDA(cudaMemcpyAsync(&count, total, sizeof(count), cudaMemcpyDeviceToHost, s));
    RSF_CUDA(cudaStreamSynchronize(s));
    *ntriangles = (int64_t)count;
    const long long written = std::min<long long>((long long)count, capacity);
    if (host_tri && written > 0)
        RSF_CUDA(xfer(triangles, e.tri, sizeof(float) * 9 * written, s));
    if (host_keys && written > 0)
        RSF_CUDA(xfer(keys, e.keys, sizeof(long long) * written, s));
    RSF_CUDA(cudaStreamSynchronize(s));
    return RSF_OK;
}
