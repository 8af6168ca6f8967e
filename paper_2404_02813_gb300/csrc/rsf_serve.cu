// rsf_serve.cu -- the request loop behind rsf_submit / rsf_poll / rsf_wait /
// rsf_cancel: continuous batching of brick segmentation requests at iteration
// granularity.
//
// A scheduler thread per context runs "ticks".  Before each round it admits
// queued requests in arrival order while their device footprint fits the
// context's HBM budget and a slot is free: the brick's fields are allocated
// from the stream-ordered pool, its image statistics, K*1 profiles, phi0 and q
// are prepared on a set-up stream, and the compute stream of its lane waits on
// that work.  Active bricks are split into four lanes by voxel count, each with
// its own stream: a tick of a lane is one iteration of every brick in it -- one
// launch per kernel for each group of bricks sharing a kernel radius, image
// type, storage and force form (the batched kernels of rsf_evolve_batch); a
// brick admitted at its lane's tick T0 runs its iteration k at tick T0 + k (its
// buffer parity is flipped accordingly).  Lanes advance independently, so a
// small brick is not paced by the iterations of large ones, and their kernels
// overlap on the GPU.  A brick that has done its iterations (or was cancelled,
// or suspended after its current iteration) retires at once: its phi is copied
// to the caller's phi_out, a host callback stamps its completion time, and its
// memory returns to the pool in stream order, so the next admission can use
// it.  While a lane's active set cannot change (no brick due to finish,
// nothing waiting in the queue, nothing to cancel or suspend), one dispatch
// enqueues up to kMaxTicks of its ticks without a host round trip; each lane
// runs at most kMaxAhead dispatches ahead of the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rsf.h"
#include "rsf_ctx.h"
#include "rsf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr size_t kMaxQueue = 1 << 20;
constexpr int kMaxAhead = 3;          // dispatches the loop may run ahead of the GPU
constexpr int kMaxTicks = 8;          // ticks one dispatch may enqueue while the active set stays fixed
constexpr int kLanes = 4;             // per-iteration cost classes, each advanced on its own stream
constexpr int kParamChunk = 6144;      // floats per parameter upload launch

struct ParamChunk {
    int offset, count;
    float v[kParamChunk];
};

__global__ void k_put(ParamChunk c, float *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.count; i += gridDim.x * blockDim.x)
        dst[c.offset + i] = c.v[i];
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Request {
    uint64_t ticket = 0;
    rsf_request req{};
    double t_submit = 0.0;
    std::atomic<int> status{RSF_PENDING};
    std::atomic<bool> cancel{false};
    std::atomic<bool> suspend{false};
    int32_t *iters_out = nullptr;  // where a suspension reports its completed iterations (under mu)
    double t_done = 0.0;
    // set at admission
    rsf::BrickDev d{};
    rsf::Taps taps{};
    int imgtype = 0, storage = 0, force = 0;
    long long n = 0;
    size_t bytes = 0;
    void *mem = nullptr;
    int done_iters = 0;
    int lane = 0;
    cudaEvent_t ready = nullptr;
};

// Active bricks of one cost class: advanced together, one tick (iteration) at a
// time, on the lane's stream; lanes progress independently of each other, so a
// small brick is not paced by the iterations of large ones.
struct Lane {
    cudaStream_t stream = nullptr;
    std::vector<std::shared_ptr<Request>> active;
    uint64_t tick = 0;
    bool groups_dirty = true;
    std::vector<rsf::TiledGroup> groups;
    DescBuffers desc;
    std::deque<cudaEvent_t> inflight;  // one event per dispatch not yet known complete
};

// The lane of a brick by its voxel count: below 2^19, 2^21, 2^23, and larger.
int lane_of(long long n) { return n < (1LL << 19) ? 0 : (n < (1LL << 21) ? 1 : (n < (1LL << 23) ? 2 : 3)); }

struct Server;

struct DoneArg {
    Server *srv;
    std::shared_ptr<Request> r;
    int status;
};

struct Server {
    rsf_ctx *ctx = nullptr;
    std::thread th;
    std::mutex mu;                   // queue, tickets, stop, stats
    std::condition_variable cv;      // work for the scheduler
    std::condition_variable done_cv; // completions for rsf_wait
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    // scheduler-thread state
    Lane lanes[kLanes];
    cudaStream_t s_setup = nullptr;
    float *partials = nullptr;
    int sms = 0;
    // statistics (mu)
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, suspended = 0, admitted = 0;
    double vox_iters = 0.0, t_first = 0.0, t_last = 0.0;
    std::vector<double> latencies;
    // host-side fault injection: the k-th admission (1-based) fails its set-up;
    // the k-th descriptor upload of the active set fails
    int64_t inject_admission = 0;
    int64_t inject_upload = 0;
    uint64_t uploads = 0;
    int64_t slots = 64;  // bricks advanced together at most
    bool poison = false; // NaN bytes in each brick's working fields at admission (tests)
};

void CUDART_CB done_cb(void *p) {
    DoneArg *a = static_cast<DoneArg *>(p);
    Server *s = a->srv;
    // a kernel's bounded wait expired on this context (the error word stays set): the
    // request's result is unreliable
    if ((a->status == RSF_OK || a->status == RSF_SUSPENDED) && device_error_code(s->ctx) != 0)
        a->status = RSF_E_CUDA;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        a->r->t_done = now_s();
        if (a->status == RSF_SUSPENDED && a->r->iters_out) *a->r->iters_out = a->r->done_iters;
        a->r->status.store(a->status);
        if (a->status == RSF_SUSPENDED) {
            ++s->suspended;
            s->vox_iters += (double)a->r->n * a->r->done_iters;
            s->t_last = a->r->t_done;
        } else if (a->status == RSF_OK) {
            ++s->completed;
            s->latencies.push_back(a->r->t_done - a->r->t_submit);
            s->vox_iters += (double)a->r->n * a->r->req.iters;
            s->t_last = a->r->t_done;
        } else if (a->status == RSF_E_CANCELLED) {
            ++s->cancelled;
        } else {
            ++s->failed;
        }
    }
    s->done_cv.notify_all();
    delete a;
}

// Device bytes of one served brick: phi and q pairs, profiles, centring
// constants, the pitched intermediate fields and (host images) a device copy.
size_t footprint(const rsf_request &r, bool stage_image) {
    const long long n = (long long)r.nx * r.ny * r.nz;
    const long long np = (long long)rsf::tiled_pitch((int)r.nx) * r.ny * r.nz;
    size_t b = 4 * align256(sizeof(float) * n) + align256(sizeof(float) * (r.nx + r.ny + r.nz)) + align256(64);
    b += align256(rsf::tiled_stage_bytes((int)r.storage, np));
    if (stage_image) b += align256(dtype_size(r.vt) * n);
    return b;
}

// Finish a request that never became active (or failed in set-up).
void finish_now(Server *s, const std::shared_ptr<Request> &r, int status) {
    DoneArg *a = new DoneArg{s, r, status};
    done_cb(a);
}

// Admission of one request on the set-up stream; returns false (and finishes
// the request) on failure.
bool admit(Server *s, const std::shared_ptr<Request> &r) {
    rsf_ctx *c = s->ctx;
    const rsf_request &q = r->req;
    ++s->admitted;
    if (s->inject_admission > 0 && (int64_t)s->admitted == s->inject_admission) {
        rsf::set_last_error("injected set-up failure");
        finish_now(s, r, RSF_E_CUDA);
        return false;
    }
    const bool stage_img = !on_device(q.volume);
    r->bytes = footprint(q, stage_img);
    {
        std::lock_guard<std::mutex> lk(c->alloc_mu);
        c->used += r->bytes;
    }
    auto fail_admit = [&](int st) {
        if (r->mem) cudaFreeAsync(r->mem, s->s_setup);
        r->mem = nullptr;
        std::lock_guard<std::mutex> lk(c->alloc_mu);
        c->used -= std::min<uint64_t>(c->used, r->bytes);
        finish_now(s, r, st);
        return false;
    };
    if (q.stream) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail_admit(RSF_E_CUDA);
        cudaEventRecord(ev, (cudaStream_t)q.stream);
        cudaStreamWaitEvent(s->s_setup, ev, 0);
        cudaEventDestroy(ev);
    }
    if (cudaMallocAsync(&r->mem, r->bytes, s->s_setup) != cudaSuccess) {
        cudaGetLastError();
        return fail_admit(RSF_E_NOMEM);
    }
    const long long n = (long long)q.nx * q.ny * q.nz;
    const int px = rsf::tiled_pitch((int)q.nx);
    r->n = n;
    r->lane = lane_of(n);
    r->taps = make_taps(q.sigma);
    r->imgtype = (int)q.vt;
    r->storage = (int)q.storage;
    char *p = static_cast<char *>(r->mem);
    auto take = [&](size_t b) {
        char *x = p;
        p += align256(b);
        return x;
    };
    rsf::BrickDev &d = r->d;
    d = rsf::BrickDev{};
    d.nx = (int)q.nx;
    d.ny = (int)q.ny;
    d.nz = (int)q.nz;
    d.px = px;
    for (int k = 0; k < 2; ++k) d.phi[k] = reinterpret_cast<float *>(take(sizeof(float) * n));
    for (int k = 0; k < 2; ++k) d.q[k] = reinterpret_cast<float *>(take(sizeof(float) * n));
    float *prof = reinterpret_cast<float *>(take(sizeof(float) * (q.nx + q.ny + q.nz)));
    float *cs = reinterpret_cast<float *>(take(64));
    d.prof = prof;
    d.cs = cs;
    const long long np = (long long)px * q.ny * q.nz;
    rsf::tiled_stage_views(r->storage, r->force, take(rsf::tiled_stage_bytes(r->storage, np)), np, &d.u2, &d.ab, &d.abxy, &d.ki);
    if (stage_img) {
        void *img = take(dtype_size(q.vt) * n);
        if (xfer(img, q.volume, dtype_size(q.vt) * n, s->s_setup) != cudaSuccess)
            return fail_admit(RSF_E_CUDA);
        d.img = img;
    } else {
        d.img = q.volume;
    }
    d.eps = q.eps;
    d.lambda1 = q.lambda1;
    d.lambda2 = q.lambda2;
    d.nu = q.nu;
    d.mu = q.mu;
    d.dt = q.dt;
    d.zc = 16;
    d.xyp = rsf::kDefaultXYPlanes;
    d.flip = (int)(s->lanes[r->lane].tick & 1);  // its iteration k runs at its lane's tick (admission + k)
    // centring constants (the profiles are set below, exactly as rsf_evolve computes them)
    rsf::Fields f;
    f.d = rsf::Dims{d.nx, d.ny, d.nz, (long long)q.nx * q.ny, n};
    f.partials = s->partials;
    f.cs = cs;
    if (rsf::image_stats(d.img, (int)q.vt, f, s->s_setup) != cudaSuccess) return fail_admit(RSF_E_CUDA);
    std::vector<float> pr((size_t)(q.nx + q.ny + q.nz));
    rsf::zero_padding_profiles(r->taps, d.nx, d.ny, d.nz, pr.data());
    for (size_t o = 0; o < pr.size(); o += kParamChunk) {
        ParamChunk ch;
        ch.offset = (int)o;
        ch.count = (int)std::min<size_t>(kParamChunk, pr.size() - o);
        memcpy(ch.v, pr.data() + o, sizeof(float) * ch.count);
        k_put<<<(ch.count + 255) / 256, 256, 0, s->s_setup>>>(ch, prof);
    }
    if (s->poison) {  // NaN bytes in everything the iteration must write before it reads
        if (cudaMemsetAsync(d.u2, 0xFF, rsf::tiled_stage_bytes(r->storage, np), s->s_setup) != cudaSuccess)
            return fail_admit(RSF_E_CUDA);
        for (float *p : {d.phi[1], d.q[0], d.q[1]})
            if (cudaMemsetAsync(p, 0xFF, sizeof(float) * n, s->s_setup) != cudaSuccess) return fail_admit(RSF_E_CUDA);
    }
    if (xfer(d.phi[0], q.phi0, sizeof(float) * n, s->s_setup) != cudaSuccess)
        return fail_admit(RSF_E_CUDA);
    if (q.iters > 0 && rsf::tiled_q_init(d.phi[0], d.q[0], n, q.eps, s->s_setup) != cudaSuccess)
        return fail_admit(RSF_E_CUDA);
    if (q.iters > 0 && rsf::tiled_ki_init(d, (int)q.vt, r->taps, s->s_setup) != cudaSuccess)
        return fail_admit(RSF_E_CUDA);
    if (rsf::tiled_prepare(r->storage, r->taps.R, r->force) != cudaSuccess) return fail_admit(RSF_E_CUDA);
    if (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess) return fail_admit(RSF_E_CUDA);
    cudaEventRecord(r->ready, s->s_setup);
    if (cudaGetLastError() != cudaSuccess) return fail_admit(RSF_E_CUDA);
    return true;
}

// Retire an active request after its last launch with `outcome`: RSF_OK and
// RSF_SUSPENDED copy phi after its done_iters iterations (the buffer of that
// parity) to the caller; RSF_E_CANCELLED and RSF_E_CUDA (a launch or upload of
// its tick failed) copy nothing.  Stamps completion, returns its memory in
// stream order.
void retire(Server *s, const std::shared_ptr<Request> &r, int outcome) {
    rsf_ctx *c = s->ctx;
    const cudaStream_t st_lane = s->lanes[r->lane].stream;
    int st = outcome;
    if ((st == RSF_OK || st == RSF_SUSPENDED) &&
        xfer(r->req.phi_out, r->d.phi[r->done_iters & 1], sizeof(float) * r->n, st_lane) != cudaSuccess)
        st = RSF_E_CUDA;
    cudaLaunchHostFunc(st_lane, done_cb, new DoneArg{s, r, st});
    cudaFreeAsync(r->mem, st_lane);
    if (r->ready) cudaEventDestroy(r->ready);
    r->mem = nullptr;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    c->used -= std::min<uint64_t>(c->used, r->bytes);
}

// Launch groups of the active set; false (and the groups left empty) when the
// descriptor upload failed.
bool rebuild_groups(Server *s, Lane &L) {
    std::vector<std::shared_ptr<Request>> order = L.active;
    std::stable_sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a->n > b->n; });
    std::vector<GroupSpec> specs;
    std::vector<std::tuple<int, int, int, int>> keys;
    for (const auto &r : order) {
        std::tuple<int, int, int, int> k{r->taps.R, r->imgtype, r->storage, r->force};
        size_t gi = std::find(keys.begin(), keys.end(), k) - keys.begin();
        if (gi == keys.size()) {
            keys.push_back(k);
            specs.emplace_back();
            specs.back().storage = r->storage;
            specs.back().force = r->force;
            specs.back().imgtype = r->imgtype;
            specs.back().taps = r->taps;
        }
        specs[gi].bricks.push_back(r->d);
    }
    for (GroupSpec &g : specs) {
        long long work = 0;
        int maxnz = 16;
        for (const rsf::BrickDev &b : g.bricks) {
            work += (long long)((b.nx + 31) / 32) * ((b.ny + 7) / 8) * b.nz;
            maxnz = std::max(maxnz, b.nz);
        }
        const int zc = (int)std::min<long long>(maxnz, std::max<long long>(16, work / std::max(1LL, 16LL * s->sms)));
        for (rsf::BrickDev &b : g.bricks) b.zc = zc;
    }
    // the copy comes from pageable memory and waits for the compute stream; the
    // loop already bounds how far it runs ahead, so this costs one short sync
    L.groups.clear();
    rsf_status st;
    if (s->inject_upload > 0 && (int64_t)++s->uploads == s->inject_upload) {
        rsf::set_last_error("injected descriptor upload failure");
        st = RSF_E_CUDA;
    } else {
        st = upload_groups(s->ctx, L.desc, L.stream, specs, &L.groups);
    }
    if (st != RSF_OK) {
        L.groups.clear();
        return false;
    }
    L.groups_dirty = false;
    return true;
}

// One dispatch of a lane: up to kMaxTicks ticks, then the retirements they cause.
void dispatch(Server *s, Lane &L, bool queued) {
    // Ticks to enqueue in this dispatch: the lane's active set stays fixed until its first
    // brick finishes, so up to that many ticks (at most kMaxTicks) go out without a host
    // round trip -- unless a request waits in the queue (it may become admissible when a
    // brick retires, and requests arriving meanwhile join after the dispatch) or a brick is
    // to be cancelled or suspended (they leave after their current iteration).
    int nticks = queued ? 1 : kMaxTicks;
    for (auto &r : L.active) {
        nticks = std::min(nticks, r->req.iters - r->done_iters);
        if (r->cancel.load() || r->suspend.load()) nticks = 1;
    }
    nticks = std::max(nticks, 1);
    // a tick counts only if the upload and every launch of it succeeded; otherwise the
    // lane's requests fail with RSF_E_CUDA (queued ones are admitted later)
    bool ok = !L.groups_dirty || rebuild_groups(s, L);
    for (int k = 0; k < nticks && ok; ++k) {
        for (const rsf::TiledGroup &g : L.groups)
            if (ok && rsf::tiled_iterate(g, (int)(L.tick & 1), nullptr, L.stream) != cudaSuccess) ok = false;
        if (ok) ++L.tick;
    }
    if (!ok) {
        cudaGetLastError();  // not sticky: later launches are not blamed for it
        for (auto &r : L.active) retire(s, r, RSF_E_CUDA);
        L.active.clear();
        L.groups.clear();
        L.groups_dirty = true;
        return;
    }
    // retire finished or cancelled bricks
    std::vector<std::shared_ptr<Request>> keep;
    keep.reserve(L.active.size());
    for (auto &r : L.active) {
        r->done_iters += nticks;
        const bool cancelled = r->cancel.load();
        const bool finished = r->done_iters >= r->req.iters;
        const bool suspended = !cancelled && !finished && r->suspend.load();
        if (cancelled || finished || suspended) {
            retire(s, r, cancelled ? RSF_E_CANCELLED : (suspended ? RSF_SUSPENDED : RSF_OK));
            L.groups_dirty = true;
        } else {
            keep.push_back(r);
        }
    }
    L.active.swap(keep);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, L.stream);
        L.inflight.push_back(ev);
    }
}

size_t n_active(const Server *s) {
    size_t k = 0;
    for (const Lane &L : s->lanes) k += L.active.size();
    return k;
}

void loop(Server *s) {
    rsf_ctx *c = s->ctx;
    cudaSetDevice(c->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> admit_now;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || n_active(s) > 0; });
            if (s->stop) break;
            // FIFO admission by footprint
            while (!s->queue.empty()) {
                std::shared_ptr<Request> r = s->queue.front();
                if (r->cancel.load()) {
                    s->queue.pop_front();
                    lk.unlock();
                    finish_now(s, r, RSF_E_CANCELLED);
                    lk.lock();
                    continue;
                }
                if (r->suspend.load()) {  // suspended before admission: its state is phi0, 0 iterations
                    s->queue.pop_front();
                    lk.unlock();
                    r->done_iters = 0;
                    cudaError_t e = xfer(r->req.phi_out, r->req.phi0, sizeof(float) * r->req.nx * r->req.ny * r->req.nz,
                                         s->s_setup);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_setup);
                    finish_now(s, r, e == cudaSuccess ? RSF_SUSPENDED : RSF_E_CUDA);
                    lk.lock();
                    continue;
                }
                const size_t need = footprint(r->req, !on_device(r->req.volume));
                uint64_t used, budget;
                {
                    std::lock_guard<std::mutex> al(c->alloc_mu);
                    used = c->used;
                    budget = c->budget;
                }
                if (used + need > budget && n_active(s) > 0) break;  // wait for retirements
                if ((int64_t)(n_active(s) + admit_now.size()) >= s->slots) break;  // wait for a free slot
                s->queue.pop_front();
                admit_now.push_back(r);
                if (used + need > budget) break;  // nothing active: admit it alone and try
            }
        }
        for (auto &r : admit_now) {
            if (admit(s, r)) {
                Lane &L = s->lanes[r->lane];
                cudaStreamWaitEvent(L.stream, r->ready, 0);
                r->done_iters = 0;
                if (r->req.iters == 0) {
                    retire(s, r, RSF_OK);
                } else {
                    L.active.push_back(r);
                    L.groups_dirty = true;
                }
            }
        }
        bool queued;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            queued = !s->queue.empty();
        }
        // each lane with work and fewer than kMaxAhead dispatches in flight gets one dispatch
        bool dispatched = false;
        for (Lane &L : s->lanes) {
            if (L.active.empty()) continue;
            while (!L.inflight.empty()) {
                const cudaError_t q = cudaEventQuery(L.inflight.front());
                if (q == cudaErrorNotReady) {
                    if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
                    break;
                }
                cudaEventDestroy(L.inflight.front());
                L.inflight.pop_front();
            }
            if ((int)L.inflight.size() >= kMaxAhead) continue;
            dispatch(s, L, queued);
            dispatched = true;
        }
        if (!dispatched) {  // every lane with work is kMaxAhead dispatches ahead of the GPU
            for (Lane &L : s->lanes)
                if (!L.inflight.empty()) {
                    cudaEventSynchronize(L.inflight.front());
                    break;
                }
        }
    }
    // shutdown: cancel what is queued or active, let the GPU finish
    std::vector<std::shared_ptr<Request>> rest;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        rest.assign(s->queue.begin(), s->queue.end());
        s->queue.clear();
    }
    for (auto &r : rest) finish_now(s, r, RSF_E_CANCELLED);
    for (Lane &L : s->lanes) {
        for (auto &r : L.active) retire(s, r, RSF_E_CANCELLED);
        L.active.clear();
    }
    for (Lane &L : s->lanes) cudaStreamSynchronize(L.stream);
    cudaStreamSynchronize(s->s_setup);
    for (Lane &L : s->lanes) {
        for (cudaEvent_t e : L.inflight) cudaEventDestroy(e);
        L.inflight.clear();
    }
}

Server *server(rsf_ctx *c, rsf_status *st) {
    std::lock_guard<std::mutex> lk(c->serve_mu);
    if (c->server) return static_cast<Server *>(c->server);
    Server *s = new Server();
    s->ctx = c;
    cudaSetDevice(c->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, c->device);
    bool streams_ok = cudaStreamCreateWithFlags(&s->s_setup, cudaStreamNonBlocking) == cudaSuccess;
    for (Lane &L : s->lanes) streams_ok = streams_ok && cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!streams_ok) {
        *st = cuda_fail(cudaGetLastError(), "serving streams");
        delete s;
        return nullptr;
    }
    if ((*st = dev_alloc(c, (void **)&s->partials, sizeof(float) * 3 * rsf::kStatBlocks))) {
        delete s;
        return nullptr;
    }
    s->inject_admission = c->opt_inject_admission;
    s->inject_upload = c->opt_inject_upload;
    s->slots = c->opt_serve_slots;
    s->poison = c->opt_poison != 0;
    s->th = std::thread(loop, s);
    c->server = s;
    return s;
}

}  // namespace

void rsf_serve_shutdown(rsf_ctx *c) {
    Server *s = static_cast<Server *>(c->server);
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    dev_free(c, s->partials, sizeof(float) * 3 * rsf::kStatBlocks);
    for (Lane &L : s->lanes) {
        free_desc(c, L.desc);
        cudaStreamDestroy(L.stream);
    }
    cudaStreamDestroy(s->s_setup);
    delete s;
    c->server = nullptr;
}

extern "C" rsf_status rsf_submit(rsf_ctx *c, const rsf_request *req, uint64_t *ticket) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!req || !ticket) return fail(RSF_E_INVAL, "null request or ticket pointer");
    rsf_status st = check_args(req->volume, req->vt, req->nx, req->ny, req->nz, req->phi0, req->phi_out, req->sigma,
                               req->eps, req->dt, req->iters);
    if (st) return st;
    if (req->storage != RSF_STORE_F32 && req->storage != RSF_STORE_BF16 && req->storage != RSF_STORE_F16)
        return fail(RSF_E_INVAL, "unknown storage %d", (int)req->storage);
    const int R = make_taps(req->sigma).R;
    if (!rsf::tiled_supports(R)) return fail(RSF_E_INVAL, "no served kernels for radius %d", R);
    if (!rsf::tiled_fits(req->nx, req->ny, req->nz)) return fail(RSF_E_INVAL, "a brick of 2^32 pitched voxels or more");
    if (req->halo >= 0 && (2 * (int64_t)req->halo >= req->nx || 2 * (int64_t)req->halo >= req->ny ||
                           2 * (int64_t)req->halo >= req->nz))
        return fail(RSF_E_INVAL, "halo %d leaves no core in a %lld x %lld x %lld brick", (int)req->halo,
                    (long long)req->nx, (long long)req->ny, (long long)req->nz);
    const size_t need = footprint(*req, !on_device(req->volume));
    if (need > c->budget)
        return fail(RSF_E_NOMEM, "request needs %zu bytes of device memory; the budget is %llu", need,
                    (unsigned long long)c->budget);
    Server *s = server(c, &st);
    if (!s) return st;
    auto r = std::make_shared<Request>();
    r->req = *req;
    r->force = c->opt_force;  // the context's data-term form at submission
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.size() >= kMaxQueue) return fail(RSF_E_BUSY, "request queue full");
        r->ticket = s->next_ticket++;
        s->tickets[r->ticket] = r;
        s->queue.push_back(r);
        ++s->submitted;
        if (s->t_first == 0.0) s->t_first = r->t_submit;
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return RSF_OK;
}

extern "C" rsf_status rsf_poll(rsf_ctx *c, uint64_t ticket, double *latency_s) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    Server *s = static_cast<Server *>(c->server);
    if (!s) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const int st = it->second->status.load();
    if (st == RSF_PENDING) return RSF_PENDING;
    if (latency_s) *latency_s = it->second->t_done - it->second->t_submit;
    s->tickets.erase(it);
    if (st < 0) return fail(st, "request %llu ended with status %d", (unsigned long long)ticket, st);
    return st;
}

extern "C" rsf_status rsf_wait(rsf_ctx *c, uint64_t ticket, int32_t timeout_ms) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    Server *s = static_cast<Server *>(c->server);
    if (!s) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        std::shared_ptr<Request> r = it->second;
        auto done = [&] { return r->status.load() != RSF_PENDING; };
        if (timeout_ms < 0) {
            s->done_cv.wait(lk, done);
        } else if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
            return fail(RSF_E_TIMEOUT, "request %llu still pending after %d ms", (unsigned long long)ticket,
                        (int)timeout_ms);
        }
    }
    return rsf_poll(c, ticket, nullptr);
}

extern "C" rsf_status rsf_cancel(rsf_ctx *c, uint64_t ticket) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    Server *s = static_cast<Server *>(c->server);
    if (!s) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    it->second->cancel.store(true);
    s->cv.notify_all();
    return RSF_OK;
}

extern "C" rsf_status rsf_suspend(rsf_ctx *c, uint64_t ticket, int32_t *iters_done) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    Server *s = static_cast<Server *>(c->server);
    if (!s) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RSF_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    it->second->iters_out = iters_done;
    it->second->suspend.store(true);
    s->cv.notify_all();
    return RSF_OK;
}

extern "C" rsf_status rsf_serve_stats(rsf_ctx *c, rsf_serve_stat *out) {
    if (!c || !out) return fail(RSF_E_INVAL, "null context or output");
    memset(out, 0, sizeof *out);
    Server *s = static_cast<Server *>(c->server);
    if (!s) return RSF_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->cancelled = s->cancelled;
    out->suspended = s->suspended;
    out->queued = s->queue.size();
    out->voxel_iterations = s->vox_iters;
    out->busy_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>((double)l.size() - 1, std::ceil(q * l.size()) - 1);
            return l[i];
        };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        out->latency_max_s = l.back();
    }
    return RSF_OK;
}
