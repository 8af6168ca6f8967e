// rsf_batch.cu -- rsf_evolve_batch: many independent bricks (halo-padded
// sub-volumes, each with its own image, level set, parameters and iteration
// count) advanced together, one launch per kernel and brick group per
// iteration (the volume-level parallelism of arXiv 2404.02813, Sec. 4.1, on
// one GPU).
//
// Schedule.  Bricks are grouped by (kernel radius, image type); within a group
// the largest bricks come first in the launch so that their CTAs start first
// and the small bricks fill the tail.  All bricks start together; between two
// retirements the active set is fixed and the iteration is a fixed sequence of
// launches, captured once as a CUDA graph of two iterations (both buffer
// parities) and replayed.  A brick that has done its iterations retires (its
// phi is copied out) and the groups are rebuilt.  With autotuning on, the z
// chunk of the update kernel is chosen per group by timing candidates on a
// first iteration that is then discarded (it only writes the second buffer).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "rsf.h"
#include "rsf_ctx.h"
#include "rsf_internal.h"

namespace {

struct BrickState {
    int index;                 // position in the caller's array
    rsf::BrickDev d;           // device view
    int iters;
    rsf_dtype vt;
    float *phi_out;
    long long n;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device bytes one brick needs in the pool.
size_t brick_bytes(const rsf_brick &b, int storage, bool stage_image) {
    const long long n = (long long)b.nx * b.ny * b.nz;
    const long long np = (long long)rsf::tiled_pitch((int)b.nx) * b.ny * b.nz;
    size_t s = 4 * align256(sizeof(float) * n);                          // phi[2], q[2]
    s += align256(sizeof(float) * (b.nx + b.ny + b.nz)) + align256(64);  // profiles, centring constants
    s += align256(rsf::tiled_stage_bytes(storage, np));
    if (stage_image) s += align256(dtype_size(b.vt) * n);
    return s;
}

int default_zc(const std::vector<rsf::BrickDev> &g, int sms) {
    long long work = 0;
    int maxnz = 16;
    for (const rsf::BrickDev &b : g) {
        work += (long long)((b.nx + 31) / 32) * ((b.ny + 7) / 8) * b.nz;
        maxnz = std::max(maxnz, b.nz);
    }
    const long long zc = work / std::max(1LL, 16LL * sms);
    return (int)std::min<long long>(maxnz, std::max<long long>(16, zc));
}

std::string group_key(const GroupSpec &g) {
    long long vox = 0;
    for (const rsf::BrickDev &b : g.bricks) vox += (long long)b.nx * b.ny * b.nz;
    char buf[128];
    snprintf(buf, sizeof buf, "R%d/i%d/s%d/f%d/nb%zu/v%lld", g.taps.R, g.imgtype, g.storage, g.force, g.bricks.size(),
             (long long)std::llround(std::log2((double)std::max(vox, 1LL))));
    return buf;
}

void set_zc(GroupSpec &g, int zc) {
    for (rsf::BrickDev &b : g.bricks) b.zc = zc;
}

// One iteration of every group at `parity`.
rsf_status launch_all(rsf_ctx *c, const std::vector<rsf::TiledGroup> &groups, int parity, rsf::Profiler *prof) {
    for (const rsf::TiledGroup &g : groups) {
        cudaError_t e = rsf::tiled_iterate(g, parity, prof, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batched iteration launch");
    }
    return RSF_OK;
}

void set_xyp(GroupSpec &g, int xyp) {
    for (rsf::BrickDev &b : g.bricks) b.xyp = xyp;
}

// The tuned choices on a group whose bricks are in largest-first order.
void apply_tuned(GroupSpec &g, const TunedGroup &t) {
    set_zc(g, t.zc);
    set_xyp(g, t.xyp);
    if (t.order) std::reverse(g.bricks.begin(), g.bricks.end());
}

// Device time of one iteration (parity 0: reads phi[0], writes phi[1]) of `g`, the
// second of two back-to-back launches (the first warms caches and attributes).
rsf_status time_iteration(rsf_ctx *c, const GroupSpec &g, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    std::vector<GroupSpec> one{g};
    std::vector<rsf::TiledGroup> up;
    rsf_status st = upload_groups(c, c->desc, c->stream, one, &up);
    if (st) return st;
    for (int rep = 0; rep < 2; ++rep) {
        RSF_CUDA(cudaEventRecord(e0, c->stream));
        if ((st = launch_all(c, up, 0, nullptr))) return st;
        RSF_CUDA(cudaEventRecord(e1, c->stream));
    }
    RSF_CUDA(cudaEventSynchronize(e1));
    RSF_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return device_error(c);
}

// Pick the group's launch choices by timing iterations, one knob after the other from
// the defaults: z planes per x/y CTA {16, 8, 32}, then the update kernel's z chunk
// {size heuristic, 32, 64, 128, 256}, then the brick order (largest or smallest
// first).  The iterations are discarded (the real first iteration rewrites their
// outputs); the choice is cached in the context per group key.
rsf_status autotune(rsf_ctx *c, GroupSpec &g, int sms) {
    const std::string key = group_key(g);
    auto hit = c->tuned.find(key);
    if (hit != c->tuned.end()) {
        apply_tuned(g, hit->second);
        return RSF_OK;
    }
    int maxnz = 16;
    for (const rsf::BrickDev &b : g.bricks) maxnz = std::max(maxnz, b.nz);
    cudaEvent_t e0, e1;
    RSF_CUDA(cudaEventCreate(&e0));
    RSF_CUDA(cudaEventCreate(&e1));
    const GroupSpec base = g;
    rsf_status st = RSF_OK;
    auto trial = [&](const TunedGroup &t, float *ms) {
        GroupSpec h = base;
        apply_tuned(h, t);
        return time_iteration(c, h, e0, e1, ms);
    };
    TunedGroup best;
    best.zc = default_zc(g.bricks, sms);
    best.xyp = rsf::kDefaultXYPlanes;
    float ms = 0.f;
    if (!(st = trial(best, &ms))) {
        best.ms = best.ms_default = ms;
        auto consider = [&](TunedGroup cand) {
            if (st) return;
            if ((st = trial(cand, &ms))) return;
            if (ms < best.ms) {
                cand.ms = ms;
                cand.ms_default = best.ms_default;
                best = cand;
            }
        };
        for (int xyp : {8, 32}) {
            TunedGroup cand = best;
            cand.xyp = xyp;
            consider(cand);
        }
        for (int zc : {32, 64, 128, 256}) {
            if (zc == best.zc || zc > maxnz) continue;
            TunedGroup cand = best;
            cand.zc = zc;
            consider(cand);
        }
        if (g.bricks.size() > 1) {
            TunedGroup cand = best;
            cand.order = 1;
            consider(cand);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    c->tuned[key] = best;
    apply_tuned(g, best);
    return RSF_OK;
}

}  // namespace

extern "C" rsf_status rsf_evolve_batch(rsf_ctx *c, const rsf_brick *bricks, int32_t nb) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (nb < 0 || (nb > 0 && !bricks)) return fail(RSF_E_INVAL, "bad brick array");
    if (nb == 0) return RSF_OK;
    for (int i = 0; i < nb; ++i) {
        const rsf_brick &b = bricks[i];
        rsf_status st = check_args(b.volume, b.vt, b.nx, b.ny, b.nz, b.phi0, b.phi_out, b.sigma, b.eps, b.dt, b.iters);
        if (st) return fail(st, "brick %d: %s", i, rsf_last_error());
        if (!rsf::tiled_supports(make_taps(b.sigma).R))
            return fail(RSF_E_INVAL, "brick %d: no batched kernels for radius %d", i, make_taps(b.sigma).R);
        if (!rsf::tiled_fits(b.nx, b.ny, b.nz))
            return fail(RSF_E_INVAL, "brick %d: 2^32 pitched voxels or more", i);
    }
    std::lock_guard<std::mutex> lk(c->mu);
    RSF_CUDA(cudaSetDevice(c->device));
    const int storage = c->opt_storage;
    const int force = c->opt_force;
    int sms = 0;
    RSF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));

    // ---- memory: one pool for every brick's fields
    std::vector<bool> stage_img(nb);
    size_t total = 0;
    for (int i = 0; i < nb; ++i) {
        stage_img[i] = !on_device(bricks[i].volume);
        total += brick_bytes(bricks[i], storage, stage_img[i]);
    }
    if (total > c->pool_cap) {
        dev_free(c, c->pool, c->pool_cap);
        c->pool = nullptr;
        c->pool_cap = 0;
        rsf_status st = dev_alloc(c, &c->pool, total);
        if (st) return st;
        c->pool_cap = total;
    }
    if (!c->f.partials) {
        rsf_status st = dev_alloc(c, (void **)&c->f.partials, sizeof(float) * 3 * rsf::kStatBlocks);
        if (st) return st;
    }

    // ---- per brick: placement, centring constants, profiles, phi0, q
    std::vector<BrickState> bs(nb);
    char *p = static_cast<char *>(c->pool);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += align256(bytes);
        return r;
    };
    for (int i = 0; i < nb; ++i) {
        const rsf_brick &b = bricks[i];
        BrickState &s = bs[i];
        const long long n = (long long)b.nx * b.ny * b.nz;
        const int px = rsf::tiled_pitch((int)b.nx);
        s.index = i;
        s.iters = b.iters;
        s.vt = b.vt;
        s.phi_out = b.phi_out;
        s.n = n;
        rsf::BrickDev &d = s.d;
        d = rsf::BrickDev{};
        d.nx = (int)b.nx;
        d.ny = (int)b.ny;
        d.nz = (int)b.nz;
        d.px = px;
        for (int k = 0; k < 2; ++k) d.phi[k] = reinterpret_cast<float *>(take(sizeof(float) * n));
        for (int k = 0; k < 2; ++k) d.q[k] = reinterpret_cast<float *>(take(sizeof(float) * n));
        float *prof = reinterpret_cast<float *>(take(sizeof(float) * (b.nx + b.ny + b.nz)));
        float *cs = reinterpret_cast<float *>(take(64));
        d.prof = prof;
        d.cs = cs;
        const long long np = (long long)px * b.ny * b.nz;
        rsf::tiled_stage_views(storage, force, take(rsf::tiled_stage_bytes(storage, np)), np, &d.u2, &d.ab, &d.abxy, &d.ki);
        if (stage_img[i]) {
            void *img = take(dtype_size(b.vt) * n);
            RSF_CUDA(xfer(img, b.volume, dtype_size(b.vt) * n, c->stream));
            d.img = img;
        } else {
            d.img = b.volume;
        }
        d.eps = b.eps;
        d.lambda1 = b.lambda1;
        d.lambda2 = b.lambda2;
        d.nu = b.nu;
        d.mu = b.mu;
        d.dt = b.dt;
        d.zc = 16;
        d.xyp = rsf::kDefaultXYPlanes;
        rsf::Fields f;
        f.d = rsf::Dims{d.nx, d.ny, d.nz, (long long)b.nx * b.ny, n};
        f.partials = c->f.partials;
        f.cs = cs;
        f.prof = prof;
        RSF_CUDA(rsf::setup_image(d.img, (int)b.vt, make_taps(b.sigma), f, c->stream, false));
        if (c->opt_poison) {  // NaN bytes in everything the iteration must write before it reads
            RSF_CUDA(cudaMemsetAsync(d.u2, 0xFF, rsf::tiled_stage_bytes(storage, np), c->stream));
            for (float *q : {d.phi[1], d.q[0], d.q[1]}) RSF_CUDA(cudaMemsetAsync(q, 0xFF, sizeof(float) * n, c->stream));
        }
        RSF_CUDA(xfer(d.phi[0], b.phi0, sizeof(float) * n, c->stream));
        if (b.iters > 0) {
            RSF_CUDA(rsf::tiled_q_init(d.phi[0], d.q[0], n, b.eps, c->stream));
            RSF_CUDA(rsf::tiled_ki_init(d, (int)b.vt, make_taps(b.sigma), c->stream));
        }
    }

    // ---- iterate: fixed active sets between retirements
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return bs[a].n > bs[b].n; });  // largest first
    auto retire = [&](int t) -> rsf_status {
        for (int i = 0; i < nb; ++i)
            if (bs[i].iters == t)
                RSF_CUDA(xfer(bs[i].phi_out, bs[i].d.phi[t & 1], sizeof(float) * bs[i].n, c->stream));
        return RSF_OK;
    };
    rsf_status st = retire(0);
    if (st) return st;
    int t = 0;
    bool tuned_once = false;
    for (;;) {
        int t_next = -1;
        for (int i = 0; i < nb; ++i)
            if (bs[i].iters > t && (t_next < 0 || bs[i].iters < t_next)) t_next = bs[i].iters;
        if (t_next < 0) break;
        // groups of the active bricks, keyed by (R, image type), largest bricks first
        std::vector<GroupSpec> specs;
        std::vector<std::pair<int, int>> keys;
        for (int i : order) {
            if (bs[i].iters <= t) continue;
            const rsf::Taps tp = make_taps(bricks[i].sigma);
            std::pair<int, int> k{tp.R, (int)bs[i].vt};
            size_t gi = std::find(keys.begin(), keys.end(), k) - keys.begin();
            if (gi == keys.size()) {
                keys.push_back(k);
                specs.emplace_back();
                specs.back().storage = storage;
                specs.back().force = force;
                specs.back().imgtype = (int)bs[i].vt;
                specs.back().taps = tp;
            }
            specs[gi].bricks.push_back(bs[i].d);
        }
        for (GroupSpec &g : specs) {
            RSF_CUDA(rsf::tiled_prepare(storage, g.taps.R, force));
            if (c->opt_zchunk > 0) {
                set_zc(g, c->opt_zchunk);
            } else if (c->opt_autotune && t == 0 && !tuned_once) {
                if ((st = autotune(c, g, sms))) return st;
            } else {
                set_zc(g, default_zc(g.bricks, sms));
            }
        }
        tuned_once = true;
        std::vector<rsf::TiledGroup> groups;
        if ((st = upload_groups(c, c->desc, c->stream, specs, &groups))) return st;
        int steps = t_next - t;
        rsf::Profiler *prof = c->prof.on ? &c->prof : nullptr;
        if (c->opt_graph && !prof && steps >= 4) {
            // capture the two parities once, replay
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            RSF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            rsf_status cst = launch_all(c, groups, t & 1, nullptr);
            if (!cst) cst = launch_all(c, groups, (t + 1) & 1, nullptr);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
            if (cst) {
                if (graph) cudaGraphDestroy(graph);
                return cst;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
            for (int k = 0; k + 1 < steps; k += 2) {
                ce = cudaGraphLaunch(exec, c->stream);
                if (ce != cudaSuccess) {
                    cudaGraphExecDestroy(exec);
                    return cuda_fail(ce, "cudaGraphLaunch");
                }
            }
            cudaGraphExecDestroy(exec);
            if (steps & 1)
                if ((st = launch_all(c, groups, (t_next - 1) & 1, nullptr))) return st;
        } else {
            for (int k = t; k < t_next; ++k)
                if ((st = launch_all(c, groups, k & 1, prof))) return st;
        }
        t = t_next;
        if ((st = retire(t))) return st;
    }
    RSF_CUDA(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

extern "C" rsf_status rsf_autotune_report(rsf_ctx *c, char *buf, int32_t cap) {
    if (!c) return fail(RSF_E_INVAL, "null context");
    if (!buf || cap <= 0) return fail(RSF_E_INVAL, "null or empty buffer");
    std::lock_guard<std::mutex> lk(c->mu);
    std::string out;
    for (const auto &kv : c->tuned) {
        char line[256];
        snprintf(line, sizeof line, "%s zc=%d xyp=%d order=%s ms=%.4f default_ms=%.4f\n", kv.first.c_str(),
                 kv.second.zc, kv.second.xyp, kv.second.order ? "smallest" : "largest", kv.second.ms,
                 kv.second.ms_default);
        out += line;
    }
    const size_t n = std::min(out.size(), (size_t)cap - 1);
    memcpy(buf, out.data(), n);
    buf[n] = 0;
    return RSF_OK;
}
