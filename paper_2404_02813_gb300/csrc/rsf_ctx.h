// rsf_ctx.h -- the context behind the C ABI's opaque rsf_ctx and the host
// helpers shared by the translation units of the C ABI (rsf_api.cu,
// rsf_batch.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rsf.h"
#include "rsf_internal.h"

// Device copies of launch-group descriptors, owned by one user of the tiled kernels.
struct DescBuffers {
    rsf::BrickDev *d_bricks = nullptr;  // descriptors of every group of the last upload
    int *d_starts = nullptr;            // per group: 4 x (nb + 1) CTA offsets
    int cap_bricks = 0, cap_starts = 0;
};

// Launch choices the batch autotuner picked for one group key, with the measured
// iteration times (ms: the choice, ms_default: the default choice).
struct TunedGroup {
    int zc = 0;     // update kernel z chunk
    int xyp = 0;    // z planes per CTA of the x/y kernels
    int order = 0;  // 0: largest bricks first in the CTA order, 1: smallest first
    float ms = 0.f, ms_default = 0.f;
};

struct rsf_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;

    rsf::Fields f;
    long long cap_n = 0;     // elements per big field currently allocated
    long long cap_np = 0;    // elements per stage field (pitched) currently allocated
    long long cap_prof = 0;  // profile floats allocated
    void *staging = nullptr; // device copy of a host volume
    size_t staging_cap = 0;
    float *dump = nullptr;   // device stage dump for host destinations
    size_t dump_cap = 0;
    rsf::Profiler prof;
    int opt_path = RSF_PATH_AUTO;
    int opt_zchunk = 0;
    int opt_storage = RSF_STORE_F32;
    int opt_force = RSF_FORCE_LI;
    DescBuffers desc;                   // brick descriptors of rsf_evolve / rsf_evolve_batch launches
    int opt_autotune = 0;
    int opt_graph = 1;
    void *pool = nullptr;               // per-brick fields of rsf_evolve_batch
    size_t pool_cap = 0;
    std::map<std::string, TunedGroup> tuned;  // autotuned launch choices per group key
    std::mutex alloc_mu;                // guards `used` (the serving thread allocates too)
    std::mutex serve_mu;                // guards creation of the serving loop
    void *server = nullptr;             // the serving loop (rsf_serve.cu), created by rsf_submit
    int64_t opt_inject_admission = 0;   // host-side fault injection for the serving loop: an admission
    int64_t opt_inject_upload = 0;      // and a descriptor upload of the active set
    int64_t opt_serve_slots = 64;       // bricks the serving loop advances together at most
    int opt_poison = 0;                 // fill working fields with NaN bytes before each solve (tests)
    int opt_fault_wait = 0;             // z pass of group A expects bytes no copy delivers (tests)
    int *h_err = nullptr;               // error word of the kernels' bounded waits: mapped pinned host
    int *d_err = nullptr;               // memory and its device address; nonzero stays (the context is spent)
};

// One launch group before upload: bricks sharing radius, image type, storage.
struct GroupSpec {
    int storage = 0, imgtype = 0, force = 0;
    rsf::Taps taps{};
    std::vector<rsf::BrickDev> bricks;
};

rsf_status fail(rsf_status st, const char *fmt, ...);
rsf_status cuda_fail(cudaError_t e, const char *what);
// The kernels' error word (rsf_ctx::h_err; read after a synchronisation): its
// value, and RSF_OK or RSF_E_CUDA with a message.
int device_error_code(const rsf_ctx *c);
rsf_status device_error(const rsf_ctx *c);
#define RSF_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)
rsf_status dev_alloc(rsf_ctx *c, void **p, size_t bytes);
void dev_free(rsf_ctx *c, void *p, size_t bytes);
bool on_device(const void *p);
// Copy `bytes` on stream s between any two of device, pinned host and pageable
// host memory; pinned host memory is read or written by a copy kernel.
cudaError_t xfer(void *dst, const void *src, size_t bytes, cudaStream_t s);
size_t dtype_size(rsf_dtype vt);
rsf_status check_args(const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz, const void *phi0,
                      const void *phi_out, float sigma, float eps, float dt, int32_t iters);
rsf::Taps make_taps(float sigma);
rsf_status upload_groups(rsf_ctx *c, DescBuffers &buf, cudaStream_t s, const std::vector<GroupSpec> &specs,
                         std::vector<rsf::TiledGroup> *out);
void free_desc(rsf_ctx *c, DescBuffers &buf);
void rsf_serve_shutdown(rsf_ctx *c);
