// rsf_api.cu -- the extern "C" boundary of librsf.so (declared in include/rsf.h):
// contexts, the HBM-budgeted workspace, host/device pointer handling, the
// blocking evolve call of Eq. (1) iterated, stage dumps and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rsf.h"
#include "rsf_ctx.h"
#include "rsf_internal.h"

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

rsf_status fail(rsf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

rsf_status cuda_fail(cudaError_t e, const char *what) {
    return fail(RSF_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int device_error_code(const rsf_ctx *c) { return c->h_err ? *(volatile const int *)c->h_err : 0; }

rsf_status device_error(const rsf_ctx *c) {
    const int code = device_error_code(c);
    if (code == 0) return RSF_OK;
    return fail(RSF_E_CUDA, "%s (device error word %d); results since are unreliable: destroy the context",
                code == rsf::kErrWaitExpired ? "a kernel's bounded wait for its TMA copies expired"
                                             : "a TMA destination in shared memory was misaligned",
                code);
}



extern "C" const char *rsf_last_error(void) { return g_last_error.c_str(); }

namespace rsf {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace rsf

// ---------------------------------------------------------------- profiler

namespace rsf {

const char *kernel_name(int id) {
    static const char *names[KID_COUNT] = {"rsf_a_x",  "rsf_a_y",    "rsf_a_z",  "rsf_b_x",   "rsf_b_y",
                                           "rsf_b_z",  "rsf_ta_xy",  "rsf_ta_z", "rsf_tb_xy", "rsf_tb_z"};
    return (id >= 0 && id < KID_COUNT) ? names[id] : nullptr;
}

cudaEvent_t Profiler::take() {
    if (used == pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    return pool[used++];
}

void Profiler::begin(int id) {
    open_id = id;
    open_a = take();
    if (open_a) cudaEventRecord(open_a, stream);
}

void Profiler::end() {
    cudaEvent_t b = take();
    if (open_a && b) {
        cudaEventRecord(b, stream);
        recs.push_back({open_id, open_a, b});
    }
    open_a = nullptr;
}

void Profiler::reset() {
    recs.clear();
    used = 0;
}

void Profiler::release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    recs.clear();
    used = 0;
}

}  // namespace rsf

// ----------------------------------------------------------------- context





rsf_status dev_alloc(rsf_ctx *c, void **p, size_t bytes) {
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    if (c->used + bytes > c->budget)
        return fail(RSF_E_NOMEM, "allocation of %zu bytes exceeds the HBM budget (%llu of %llu bytes in use)", bytes,
                    (unsigned long long)c->used, (unsigned long long)c->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(RSF_E_NOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    return RSF_OK;
}

void dev_free(rsf_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    cudaFree(p);
    c->used -= std::min<uint64_t>(c->used, bytes);
}


// Copy the brick descriptors of several launch groups and their per-kernel
// CTA offsets to the device in one upload, and describe each group.
void free_desc(rsf_ctx *c, DescBuffers &buf) {
    dev_free(c, buf.d_bricks, sizeof(rsf::BrickDev) * (size_t)buf.cap_bricks);
    dev_free(c, buf.d_starts, sizeof(int) * (size_t)buf.cap_starts);
    buf = DescBuffers{};
}

rsf_status upload_groups(rsf_ctx *c, DescBuffers &buf, cudaStream_t stream, const std::vector<GroupSpec> &specs,
                         std::vector<rsf::TiledGroup> *out) {
    int total = 0;
    for (const GroupSpec &g : specs) total += (int)g.bricks.size();
    const int need_starts = 4 * (total + (int)specs.size());
    if (total > buf.cap_bricks || need_starts > buf.cap_starts) {
        free_desc(c, buf);
        const int cap = std::max(total, 16), capst = std::max(need_starts, 4 * 32);
        rsf_status st = dev_alloc(c, (void **)&buf.d_bricks, sizeof(rsf::BrickDev) * (size_t)cap);
        if (st) return st;
        st = dev_alloc(c, (void **)&buf.d_starts, sizeof(int) * (size_t)capst);
        if (st) return st;
        buf.cap_bricks = cap;
        buf.cap_starts = capst;
    }
    std::vector<rsf::BrickDev> all;
    std::vector<int> starts;
    all.reserve(total);
    starts.reserve(need_starts);
    out->clear();
    for (const GroupSpec &gs : specs) {
        const int nb = (int)gs.bricks.size();
        rsf::TiledGroup g{};
        g.storage = gs.storage;
        g.force = gs.force;
        g.imgtype = gs.imgtype;
        g.taps = gs.taps;
        g.bricks = buf.d_bricks + all.size();
        g.nb = nb;
        g.dump = 0;
        for (const rsf::BrickDev &b : gs.bricks) g.dump |= b.dump != nullptr;
        g.err = c->d_err;
        g.fault_tx = c->opt_fault_wait ? 16u : 0u;
        g.xy_tma = 1;
        const size_t s0 = starts.size();
        starts.resize(s0 + 4 * (size_t)(nb + 1));
        unsigned long long tot[4] = {0, 0, 0, 0};
        for (int i = 0; i < nb; ++i) {
            unsigned cnt[4];
            rsf::tiled_cta_counts(gs.bricks[i], cnt);
            for (int k = 0; k < 4; ++k) {
                starts[s0 + (size_t)k * (nb + 1) + i] = (int)tot[k];
                tot[k] += cnt[k];
            }
        }
        for (int k = 0; k < 4; ++k) {
            if (tot[k] >= (1ull << 31)) return fail(RSF_E_INVAL, "launch group too large (%llu CTAs)", tot[k]);
            starts[s0 + (size_t)k * (nb + 1) + nb] = (int)tot[k];
            g.starts[k] = buf.d_starts + s0 + (size_t)k * (nb + 1);
            g.ncta[k] = (unsigned)tot[k];
        }
        for (rsf::BrickDev b : gs.bricks) {
            const cudaError_t e = rsf::tiled_encode_maps(b, gs.force, gs.storage, gs.imgtype, gs.taps.R);
            if (e != cudaSuccess) return fail(RSF_E_CUDA, "TMA descriptor of a %dx%dx%d brick: %s", b.nx, b.ny, b.nz,
                                              cudaGetErrorString(e));
            g.xy_tma &= b.xy_tma;
            all.push_back(b);
        }
        out->push_back(g);
    }
    RSF_CUDA(cudaMemcpyAsync(buf.d_bricks, all.data(), sizeof(rsf::BrickDev) * all.size(), cudaMemcpyHostToDevice,
                             stream));
    RSF_CUDA(cudaMemcpyAsync(buf.d_starts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice,
                             stream));
    return RSF_OK;
}

static void free_fields(rsf_ctx *c) {
    size_t fb = sizeof(float) * (size_t)c->cap_n;
    dev_free(c, c->f.I, fb);
    for (float *&p : c->f.phi) { dev_free(c, p, fb); p = nullptr; }
    for (float *&p : c->f.q) { dev_free(c, p, fb); p = nullptr; }
    dev_free(c, c->f.t[0], sizeof(float) * 8 * (size_t)c->cap_np);
    for (float *&p : c->f.t) p = nullptr;
    c->f.I = nullptr;
    c->cap_n = 0;
    c->cap_np = 0;
    dev_free(c, c->f.prof, sizeof(float) * (size_t)c->cap_prof);
    c->f.prof = nullptr;
    c->cap_prof = 0;
}

rsf_status ensure_fields(rsf_ctx *c, int nx, int ny, int nz) {
    rsf::Dims d{nx, ny, nz, (long long)nx * ny, (long long)nx * ny * nz};
    const int px = rsf::tiled_pitch(nx);
    const long long np = (long long)px * ny * nz;  // >= n: also holds the pass path's fields
    if (d.n > c->cap_n || np > c->cap_np) {
        free_fields(c);
        const size_t fb = sizeof(float) * (size_t)d.n;
        const size_t need = 5 * fb + sizeof(float) * 8 * (size_t)np;
        if (need + c->used > c->budget)
            return fail(RSF_E_NOMEM, "volume of %lld voxels needs %llu bytes of working fields; budget %llu, in use %llu",
                        d.n, (unsigned long long)need, (unsigned long long)c->budget, (unsigned long long)c->used);
        rsf_status st;
        if ((st = dev_alloc(c, (void **)&c->f.I, fb))) return st;
        for (float *&p : c->f.phi)
            if ((st = dev_alloc(c, (void **)&p, fb))) return st;
        for (float *&p : c->f.q)
            if ((st = dev_alloc(c, (void **)&p, fb))) return st;
        if ((st = dev_alloc(c, (void **)&c->f.t[0], sizeof(float) * 8 * (size_t)np))) return st;
        for (int i = 1; i < 8; ++i) c->f.t[i] = c->f.t[0] + (size_t)i * np;
        c->cap_n = d.n;
        c->cap_np = np;
    } else {
        for (int i = 1; i < 8; ++i) c->f.t[i] = c->f.t[0] + (size_t)i * c->cap_np;
    }
    long long npf = (long long)nx + ny + nz;
    if (npf > c->cap_prof) {
        dev_free(c, c->f.prof, sizeof(float) * (size_t)c->cap_prof);
        c->f.prof = nullptr;
        rsf_status st = dev_alloc(c, (void **)&c->f.prof, sizeof(float) * npf);
        if (st) return st;
        c->cap_prof = npf;
    }
    if (!c->f.cs) {
        rsf_status st = dev_alloc(c, (void **)&c->f.cs, sizeof(float) * 4);
        if (st) return st;
        st = dev_alloc(c, (void **)&c->f.partials, sizeof(float) * 3 * rsf::kStatBlocks);
        if (st) return st;
    }
    c->f.d = d;
    c->f.px = px;
    return RSF_OK;
}

// True when p is memory the device can use in place (device or managed).
bool on_device(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t dtype_size(rsf_dtype vt) { return vt == RSF_U8 ? 1 : (vt == RSF_U16 ? 2 : 4); }

namespace {
__global__ void k_copy16(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void k_copy4(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void k_copy1(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
// 0 device or managed, 1 pinned host (allocated or registered with CUDA, with its
// device address), 2 any other host memory (pageable, also where the device can
// reach it through the address translation of the host)
int mem_kind(const void *p, const void **dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *dev = p;
        return 0;
    }
    unsigned flags = 0;
    if (a.type == cudaMemoryTypeHost && a.devicePointer && cudaHostGetFlags(&flags, const_cast<void *>(p)) == cudaSuccess) {
        *dev = a.devicePointer;
        return 1;
    }
    cudaGetLastError();
    return 2;
}
}  // namespace

cudaError_t xfer(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const void *ds = nullptr, *dd = nullptr;
    const int ks = mem_kind(src, &ds), kd = mem_kind(dst, &dd);
    if (ks == 2 || kd == 2 || (ks == 0 && kd == 0)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    // pinned host on at least one side: the SMs copy through the device mapping, which keeps its
    // full rate after long device work (the copy engine's rate drops there)
    const uintptr_t a = reinterpret_cast<uintptr_t>(ds) | reinterpret_cast<uintptr_t>(dd);
    if ((a & 15) == 0 && bytes % 16 == 0) {
        const size_t n = bytes / 16;
        k_copy16<<<(unsigned)std::min<size_t>(1216, (n + 511) / 512), 512, 0, s>>>(static_cast<const uint4 *>(ds),
                                                                                  static_cast<uint4 *>(const_cast<void *>(dd)), n);
    } else if ((a & 3) == 0 && bytes % 4 == 0) {
        const size_t n = bytes / 4;
        k_copy4<<<(unsigned)std::min<size_t>(1216, (n + 511) / 512), 512, 0, s>>>(
            static_cast<const uint32_t *>(ds), static_cast<uint32_t *>(const_cast<void *>(dd)), n);
    } else {
        k_copy1<<<(unsigned)std::min<size_t>(1216, (bytes + 511) / 512), 512, 0, s>>>(
            static_cast<const uint8_t *>(ds), static_cast<uint8_t *>(const_cast<void *>(dd)), bytes);
    }
    return cudaGetLastError();
}

// Device-resident copy of the volume (the caller's own pointer when it already is one).
static rsf_status device_volume(rsf_ctx *c, const void *volume, rsf_dtype vt, long long n, const void **out) {
    if (on_device(volume)) {
        *out = volume;
        return RSF_OK;
    }
    size_t bytes = dtype_size(vt) * (size_t)n;
    if (bytes > c->staging_cap) {
        dev_free(c, c->staging, c->staging_cap);
        c->staging = nullptr;
        c->staging_cap = 0;
        rsf_status st = dev_alloc(c, &c->staging, bytes);
        if (st) return st;
        c->staging_cap = bytes;
    }
    RSF_CUDA(xfer(c->staging, volume, bytes, c->stream));
    *out = c->staging;
    return RSF_OK;
}

rsf_status check_args(const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz, const void *phi0,
                             const void *phi_out, float sigma, float eps, float dt, int32_t iters) {
    if (!volume || !phi0 || !phi_out) return fail(RSF_E_INVAL, "null volume, phi0 or phi_out pointer");
    if (vt != RSF_U8 && vt != RSF_U16 && vt != RSF_F32) return fail(RSF_E_INVAL, "unknown volume dtype %d", (int)vt);
    const int64_t lim = 1 << 20;
    if (nx < 4 || ny < 4 || nz < 4 || nx > lim || ny > lim || nz > lim)
        return fail(RSF_E_INVAL, "each dimension must lie in [4, 2^20]; got %lld x %lld x %lld", (long long)nx,
                    (long long)ny, (long long)nz);
    if ((double)nx * (double)ny * (double)nz > 17179869184.0)
        return fail(RSF_E_INVAL, "nx*ny*nz exceeds 2^34");
    if ((double)ny * (double)nz >= 2147483648.0) return fail(RSF_E_INVAL, "ny*nz must be below 2^31");
    if (!(sigma > 0.f) || !std::isfinite(sigma)) return fail(RSF_E_INVAL, "sigma must be positive and finite");
    if ((int)std::floor(2.0 * sigma + 0.5) > rsf::RMAX)
        return fail(RSF_E_INVAL, "kernel radius round(2 sigma) = %d exceeds %d", (int)std::floor(2.0 * sigma + 0.5),
                    rsf::RMAX);
    if (!(eps > 0.f) || !std::isfinite(eps)) return fail(RSF_E_INVAL, "eps must be positive and finite");
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(RSF_E_INVAL, "dt must be positive and finite");
    if (iters < 0) return fail(RSF_E_INVAL, "iters must be >= 0");
    return RSF_OK;
}

// Normalised taps of Eq. (7): exp(-k^2/(2 sigma^2)) / sum, R = round(2 sigma).
rsf::Taps make_taps(float sigma) {
    rsf::Taps t{};
    t.R = (int)std::floor(2.0 * (double)sigma + 0.5);
    double w[2 * rsf::RMAX + 1], s = 0.0;
    for (int k = -t.R; k <= t.R; ++k) {
        w[k + t.R] = std::exp(-(double)k * k / (2.0 * (double)sigma * (double)sigma));
        s += w[k + t.R];
    }
    for (int k = 0; k < 2 * t.R + 1; ++k) t.g[k] = (float)(w[k] / s);
    return t;
}

extern "C" rsf_status rsf_create(rsf_ctx **out, int device, uint64_t hbm_budget_bytes, uint32_t flags) {
    if (!out) return fail(RSF_E_INVAL, "out is null");
    *out = nullptr;
    if (flags != 0) return fail(RSF_E_INVAL, "flags must be 0");
    int n = 0;
    RSF_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(RSF_E_CUDA, "no CUDA device %d (%d present)", device, n);
    RSF_CUDA(cudaSetDevice(device));
    size_t fr = 0, tot = 0;
    RSF_CUDA(cudaMemGetInfo(&fr, &tot));
    rsf_ctx *c = new rsf_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.9 * (double)fr);
    // a blocking stream: ordered after work the caller queued on the legacy default stream
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    c->prof.stream = c->stream;
    // the kernels' bounded waits report expiry here: mapped pinned host memory, read by the
    // host after the synchronisation that ends each call, with no copy
    e = cudaHostAlloc((void **)&c->h_err, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&c->d_err, c->h_err, 0);
    if (e != cudaSuccess) {
        if (c->h_err) cudaFreeHost(c->h_err);
        cudaStreamDestroy(c->stream);
        delete c;
        return cuda_fail(e, "error word");
    }
    *c->h_err = 0;
    *out = c;
    return RSF_OK;
}

extern "C" void rsf_destroy(rsf_ctx *c) {
    if (!c) return;
    rsf_serve_shutdown(c);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        free_fields(c);
        dev_free(c, c->f.cs, sizeof(float) * 4);
        dev_free(c, c->f.partials, sizeof(float) * 3 * rsf::kStatBlocks);
        dev_free(c, c->staging, c->staging_cap);
        dev_free(c, c->dump, c->dump_cap);
        free_desc(c, c->desc);
        dev_free(c, c->pool, c->pool_cap);
        c->prof.release();
        cudaStreamDestroy(c->stream);
        cudaFreeHost(c->h_err);
    }
    delete c;
}

extern "C" void *rsf_stream(rsf_ctx *c) { return c ? (void *)c->stream : nullptr; }

// Shared body of rsf_evolve and rsf_step_stages.
static rsf_status run(rsf_ctx *c, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                      const float *phi0, float *phi_out, float *stages, float sigma, float eps, float lambda1,
                      float lambda2, float nu, float mu, float dt, int32_t iters) {
    RSF_CUDA(cudaSetDevice(c->device));
    rsf_status st = ensure_fields(c, (int)nx, (int)ny, (int)nz);
    if (st) return st;
    rsf::Fields &f = c->f;
    const long long n = f.d.n;
    bool ready = f.I && f.prof && f.cs && f.partials && f.phi[0] && f.phi[1] && f.q[0] && f.q[1];
    for (float *p : f.t) ready = ready && p;
    if (!ready) return fail(RSF_E_CUDA, "internal error: working fields are not allocated");
    float *dump = nullptr;
    if (stages) {
        if (on_device(stages)) {
            dump = stages;
        } else {
            size_t bytes = sizeof(float) * (size_t)n * RSF_NSTAGES;
            if (bytes > c->dump_cap) {
                dev_free(c, c->dump, c->dump_cap);
                c->dump = nullptr;
                c->dump_cap = 0;
                if ((st = dev_alloc(c, (void **)&c->dump, bytes))) return st;
                c->dump_cap = bytes;
            }
            dump = c->dump;
        }
    }
    const void *vol = nullptr;
    if ((st = device_volume(c, volume, vt, n, &vol))) return st;
    const rsf::Taps taps = make_taps(sigma);
    const rsf::Coeffs co{eps, lambda1, lambda2, nu, mu, dt};
    const int storage = c->opt_storage;
    const bool tiled = c->opt_path != RSF_PATH_PASSES && rsf::tiled_supports(taps.R) && rsf::tiled_fits(nx, ny, nz);
    if (c->opt_path == RSF_PATH_TILED && !tiled)
        return fail(RSF_E_INVAL, "the tiled path has no kernels for radius %d or for %lld voxels (pitched, 2^32 at most)",
                    taps.R, (long long)rsf::tiled_pitch((int)nx) * ny * nz);
    if (storage != RSF_STORE_F32 && !tiled)
        return fail(RSF_E_INVAL, "16-bit storage needs the tiled path (radius %d, path option %d)", taps.R, c->opt_path);
    const int force = c->opt_force;
    if (force != RSF_FORCE_LI && !tiled)
        return fail(RSF_E_INVAL, "the Eq. (15) force form needs the tiled path (radius %d, path option %d)", taps.R,
                    c->opt_path);
    // the tiled path reads the image in its own type and centres it on load
    RSF_CUDA(rsf::setup_image(vol, (int)vt, taps, f, c->stream, !tiled));
    if (c->opt_poison) {  // NaN bytes in everything the iteration must write before it reads
        RSF_CUDA(cudaMemsetAsync(f.t[0], 0xFF, sizeof(float) * 8 * (size_t)c->cap_np, c->stream));
        for (float *p : {f.phi[1], f.q[0], f.q[1]}) RSF_CUDA(cudaMemsetAsync(p, 0xFF, sizeof(float) * n, c->stream));
    }
    RSF_CUDA(xfer(f.phi[0], phi0, sizeof(float) * n, c->stream));
    int cur = 0;
    if (tiled) {
        RSF_CUDA(rsf::tiled_prepare(storage, taps.R, force));
        rsf::BrickDev b{};
        b.nx = (int)nx;
        b.ny = (int)ny;
        b.nz = (int)nz;
        b.px = f.px;
        b.img = vol;
        b.cs = f.cs;
        b.prof = f.prof;
        b.phi[0] = f.phi[0];
        b.phi[1] = f.phi[1];
        b.q[0] = f.q[0];
        b.q[1] = f.q[1];
        rsf::tiled_stage_views(storage, force, f.t[0], (long long)f.px * ny * nz, &b.u2, &b.ab, &b.abxy, &b.ki);
        b.eps = eps;
        b.lambda1 = lambda1;
        b.lambda2 = lambda2;
        b.nu = nu;
        b.mu = mu;
        b.dt = dt;
        b.zc = c->opt_zchunk;
        b.xyp = rsf::kDefaultXYPlanes;
        if (b.zc <= 0) {  // enough z chunks for about 16 CTAs per SM
            int sms = 0;
            RSF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
            const long long nxy = (long long)((nx + 31) / 32) * ((ny + 7) / 8);
            const long long chunks = std::max<long long>(1, (16LL * sms + nxy - 1) / nxy);
            b.zc = (int)std::max<long long>(16, (nz + chunks - 1) / chunks);
        }
        b.dump = dump;  // only rsf_step_stages asks for stages, and it runs one iteration
        std::vector<GroupSpec> specs(1);
        specs[0].storage = storage;
        specs[0].force = force;
        specs[0].imgtype = (int)vt;
        specs[0].taps = taps;
        specs[0].bricks.push_back(b);
        std::vector<rsf::TiledGroup> groups;
        if ((st = upload_groups(c, c->desc, c->stream, specs, &groups))) return st;
        const rsf::TiledGroup &g = groups[0];
        if (iters > 0) {
            RSF_CUDA(rsf::tiled_q_init(f.phi[0], f.q[0], n, eps, c->stream));
            RSF_CUDA(rsf::tiled_ki_init(b, (int)vt, taps, c->stream));
        }
        for (int it = 0; it < iters; ++it) {
            cudaError_t e = rsf::tiled_iterate(g, it & 1, &c->prof, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "iteration launch");
        }
        cur = iters & 1;
    } else {
        for (int it = 0; it < iters; ++it) {
            float *d_it = it == iters - 1 ? dump : nullptr;
            cudaError_t e = rsf::iterate_passes(taps, co, f, f.phi[cur], f.phi[cur ^ 1], d_it, &c->prof, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "iteration launch");
            cur ^= 1;
        }
    }
    RSF_CUDA(xfer(phi_out, f.phi[cur], sizeof(float) * n, c->stream));
    if (stages && dump != stages)
        RSF_CUDA(xfer(stages, dump, sizeof(float) * n * RSF_NSTAGES, c->stream));
    RSF_CUDA(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

extern "C" rsf_status rsf_evolve(rsf_ctx *c, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                                 const float *phi0, float *phi_out, float sigma, float eps, float lambda1,
                                 float lambda2, float nu, float mu, float dt, int32_t iters) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    rsf_status st = check_args(volume, vt, nx, ny, nz, phi0, phi_out, sigma, eps, dt, iters);
    if (st) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return run(c, volume, vt, nx, ny, nz, phi0, phi_out, nullptr, sigma, eps, lambda1, lambda2, nu, mu, dt, iters);
}

extern "C" rsf_status rsf_step_stages(rsf_ctx *c, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny,
                                      int64_t nz, const float *phi, float *phi_next, float *stages, float sigma,
                                      float eps, float lambda1, float lambda2, float nu, float mu, float dt) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!stages) return fail(RSF_E_INVAL, "null stages pointer");
    rsf_status st = check_args(volume, vt, nx, ny, nz, phi, phi_next, sigma, eps, dt, 1);
    if (st) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    return run(c, volume, vt, nx, ny, nz, phi, phi_next, stages, sigma, eps, lambda1, lambda2, nu, mu, dt, 1);
}

// ----------------------------------------------------------------- options

extern "C" rsf_status rsf_set_option(rsf_ctx *c, int32_t key, int64_t value) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    std::lock_guard<std::mutex> lk(c->mu);
    switch (key) {
        case RSF_OPT_PATH:
            if (value < RSF_PATH_AUTO || value > RSF_PATH_TILED) return fail(RSF_E_INVAL, "unknown path %lld", (long long)value);
            c->opt_path = (int)value;
            return RSF_OK;
        case RSF_OPT_STORAGE:
            if (value != RSF_STORE_F32 && value != RSF_STORE_BF16 && value != RSF_STORE_F16)
                return fail(RSF_E_INVAL, "unknown storage %lld", (long long)value);
            c->opt_storage = (int)value;
            return RSF_OK;
        case RSF_OPT_FORCE:
            if (value != RSF_FORCE_LI && value != RSF_FORCE_EQ15)
                return fail(RSF_E_INVAL, "unknown force form %lld", (long long)value);
            c->opt_force = (int)value;
            return RSF_OK;
        case RSF_OPT_SERVE_SLOTS:
            if (value < 1 || value > (1 << 20)) return fail(RSF_E_INVAL, "slots must lie in [1, 2^20]");
            c->opt_serve_slots = value;
            return RSF_OK;
        case RSF_OPT_FAULT_ADMISSION:
            if (value < 0) return fail(RSF_E_INVAL, "fault admission index must be >= 0");
            c->opt_inject_admission = value;
            return RSF_OK;
        case RSF_OPT_FAULT_UPLOAD:
            if (value < 0) return fail(RSF_E_INVAL, "fault upload index must be >= 0");
            c->opt_inject_upload = value;
            return RSF_OK;
        case RSF_OPT_AUTOTUNE:
            c->opt_autotune = value != 0;
            return RSF_OK;
        case RSF_OPT_POISON:
            c->opt_poison = value != 0;
            return RSF_OK;
        case RSF_OPT_FAULT_WAIT:
            c->opt_fault_wait = value != 0;
            return RSF_OK;
        case RSF_OPT_GRAPH:
            c->opt_graph = value != 0;
            return RSF_OK;
        case RSF_OPT_ZCHUNK:
            if (value < 0 || value > (1 << 20)) return fail(RSF_E_INVAL, "z chunk must lie in [0, 2^20]");
            if (value != 0 && value < 8) return fail(RSF_E_INVAL, "z chunk must be 0 (automatic) or >= 8");
            c->opt_zchunk = (int)value;
            return RSF_OK;
        default:
            return fail(RSF_E_INVAL, "unknown option key %d", (int)key);
    }
}

// ----------------------------------------------------------- kernel timing

extern "C" rsf_status rsf_prof_enable(rsf_ctx *c, int32_t on) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    RSF_CUDA(cudaStreamSynchronize(c->stream));
    c->prof.on = on != 0;
    if (on) c->prof.reset();
    return RSF_OK;
}

extern "C" int32_t rsf_prof_count(void) { return rsf::KID_COUNT; }

extern "C" const char *rsf_prof_name(int32_t k) { return rsf::kernel_name(k); }

extern "C" rsf_status rsf_prof_get(rsf_ctx *c, int32_t k, int64_t *launches, double *total_ms) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (k < 0 || k >= rsf::KID_COUNT) return fail(RSF_E_INVAL, "unknown kernel index %d", (int)k);
    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    RSF_CUDA(cudaStreamSynchronize(c->stream));
    int64_t cnt = 0;
    double ms = 0.0;
    for (const auto &r : c->prof.recs) {
        if (r.id != k) continue;
        float t = 0.f;
        RSF_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return RSF_OK;
}
