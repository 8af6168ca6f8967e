// rsf_noalloc.cu -- rsf_evolve_noalloc: the level-set evolution of rsf_evolve
// for small volumes, with every working field held in one file-scope device
// array instead of memory the library allocates.
//
// Who needs it: code that may not allocate GPU memory while it runs -- a
// plug-in whose host application owns all device memory through its own pool,
// a real-time or streaming thread that cannot accept the device-wide
// synchronisation a cudaMalloc / cudaFree can imply, or a service whose
// memory was sized once at start-up.  Those callers bring their own input and
// output buffers and a stream; this entry point touches only them and the
// static array below.
//
// The static array is part of the library image: every GPU that loads
// librsf.so holds it (about 10.5 MB) until the process exits.  All calls on a
// device share it and it keeps the contents of the last call; calls whose
// work overlaps on the GPU (several streams, several host threads) race on it
// and must be serialised by the caller.  No part of it needs to start at zero:
// every field is written in full before it is read.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "rsf.h"
#include "rsf_ctx.h"
#include "rsf_internal.h"

namespace {

constexpr long long kMaxVoxels = 1LL << 18;              // 262,144 voxels (for example 64^3)
constexpr long long kMaxProfile = kMaxVoxels / 16 + 8;   // nx+ny+nz when every side is >= 4
constexpr long long kOffI = 0;                           // centred image
constexpr long long kOffPhi = kOffI + kMaxVoxels;        // one phi buffer (phi_out is the other)
constexpr long long kOffT = kOffPhi + kMaxVoxels;        // eight stage buffers
constexpr long long kOffProf = kOffT + 8 * kMaxVoxels;   // K*1 profiles
constexpr long long kOffCs = kOffProf + ((kMaxProfile + 63) / 64) * 64;
constexpr long long kOffPart = kOffCs + 64;              // reduction partials
constexpr long long kScratchFloats = kOffPart + 3 * rsf::kStatBlocks;
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

namespace {

std::mutex g_mu;
float *g_scratch_dev[kMaxDevices] = {};

rsf_status err(rsf_status st, const char *msg) {
    rsf::set_last_error(msg);
    return st;
}

// Device address of the static array on the current device, looked up once per
// device (with that device current).  The name g_noalloc_scratch is only a
// host-side stand-in; kernels must be given this address.
rsf_status scratch_on_current_device(float **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(RSF_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(RSF_E_CUDA, "device index out of range for rsf_evolve_noalloc");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return err(RSF_E_CUDA, buf);
        }
        g_scratch_dev[dev] = (float *)p;
    }
    *out = g_scratch_dev[dev];
    return RSF_OK;
}

// Memory the kernels of device `dev` may read and write in place: device memory
// of that device, or managed memory.  (Device memory of another GPU is refused:
// without peer access a kernel here would fault on it.)
bool is_device_ptr(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// Values written into the static array through kernel parameters, so that no
// host staging buffer and no allocation is involved (24 KB per launch).
constexpr int kParamChunk = 6144;
struct ParamChunk {
    int offset, count;
    float v[kParamChunk];
};

__global__ void k_noalloc_put(ParamChunk c, float *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.count; i += gridDim.x * blockDim.x)
        dst[c.offset + i] = c.v[i];
}

}  // namespace

extern "C" rsf_status rsf_evolve_noalloc(const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                                         const float *phi0, float *phi_out, float sigma, float eps, float lambda1,
                                         float lambda2, float nu, float mu, float dt, int32_t iters, void *stream) {
    if (!volume || !phi0 || !phi_out) return err(RSF_E_INVAL, "null volume, phi0 or phi_out pointer");
    if (vt != RSF_U8 && vt != RSF_U16 && vt != RSF_F32) return err(RSF_E_INVAL, "unknown volume dtype");
    if (nx < 4 || ny < 4 || nz < 4) return err(RSF_E_INVAL, "each dimension must be >= 4");
    if ((double)nx * (double)ny * (double)nz > (double)kMaxVoxels) {
        char buf[200];
        snprintf(buf, sizeof buf, "rsf_evolve_noalloc: %lld voxels exceed its static limit of %lld voxels",
                 (long long)nx * ny * nz, kMaxVoxels);
        return err(RSF_E_INVAL, buf);
    }
    if (!(sigma > 0.f) || !std::isfinite(sigma)) return err(RSF_E_INVAL, "sigma must be positive and finite");
    const int R = (int)std::floor(2.0 * (double)sigma + 0.5);
    if (R > rsf::RMAX) return err(RSF_E_INVAL, "kernel radius round(2 sigma) exceeds 16");
    if (!(eps > 0.f) || !std::isfinite(eps)) return err(RSF_E_INVAL, "eps must be positive and finite");
    if (!(dt > 0.f) || !std::isfinite(dt)) return err(RSF_E_INVAL, "dt must be positive and finite");
    if (iters < 0) return err(RSF_E_INVAL, "iters must be >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(RSF_E_CUDA, cudaGetErrorString(e));
    if (!is_device_ptr(volume, dev) || !is_device_ptr(phi0, dev) || !is_device_ptr(phi_out, dev))
        return err(RSF_E_INVAL, "rsf_evolve_noalloc takes device pointers of the current device only");

    float *base = nullptr;
    rsf_status st = scratch_on_current_device(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;

    rsf::Fields f;
    f.d = rsf::Dims{(int)nx, (int)ny, (int)nz, (long long)nx * ny, (long long)nx * ny * nz};
    f.I = base + kOffI;
    for (int i = 0; i < 8; ++i) f.t[i] = base + kOffT + i * kMaxVoxels;
    f.prof = base + kOffProf;
    f.cs = base + kOffCs;
    f.partials = base + kOffPart;
    float *scratch_phi = base + kOffPhi;
    const long long n = f.d.n;

    const rsf::Taps taps = make_taps(sigma);
    const rsf::Coeffs co{eps, lambda1, lambda2, nu, mu, dt};

    if (iters == 0) {
        if (phi_out != phi0) e = cudaMemcpyAsync(phi_out, phi0, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
        else e = cudaSuccess;
        return e == cudaSuccess ? RSF_OK : err(RSF_E_CUDA, cudaGetErrorString(e));
    }
    if ((e = rsf::centre_image(volume, (int)vt, f, s)) != cudaSuccess) return err(RSF_E_CUDA, cudaGetErrorString(e));
    // zero-padding profiles (K*1 = p_x p_y p_z), by the same host routine as rsf_evolve's;
    // nx + ny + nz <= kMaxProfile within the voxel limit
    float prof[kMaxProfile];
    const int np = (int)(nx + ny + nz);
    rsf::zero_padding_profiles(taps, (int)nx, (int)ny, (int)nz, prof);
    for (int o = 0; o < np; o += kParamChunk) {
        ParamChunk c;
        c.offset = o;
        c.count = np - o < kParamChunk ? np - o : kParamChunk;
        for (int i = 0; i < c.count; ++i) c.v[i] = prof[o + i];
        k_noalloc_put<<<(c.count + 255) / 256, 256, 0, s>>>(c, f.prof);
    }
    // phi0 is copied first so that phi_out may alias it; the iterations then
    // alternate between the static buffer and phi_out
    if ((e = cudaMemcpyAsync(scratch_phi, phi0, sizeof(float) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return err(RSF_E_CUDA, cudaGetErrorString(e));
    const float *in = scratch_phi;
    float *out = phi_out;
    for (int it = 0; it < iters; ++it) {
        if ((e = rsf::iterate_passes(taps, co, f, in, out, nullptr, nullptr, s)) != cudaSuccess)
            return err(RSF_E_CUDA, cudaGetErrorString(e));
        float *nxt = (out == phi_out) ? scratch_phi : phi_out;
        in = out;
        out = nxt;
    }
    if (in != phi_out) {
        if ((e = cudaMemcpyAsync(phi_out, in, sizeof(float) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return err(RSF_E_CUDA, cudaGetErrorString(e));
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? RSF_OK : err(RSF_E_CUDA, cudaGetErrorString(e));
}
