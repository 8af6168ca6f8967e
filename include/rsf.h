/*
 * rsf.h -- C ABI of the GB300 (sm_103a) 3D region-scalable-fitting (RSF)
 * level-set library `librsf.so`.
 *
 * The library evolves a level-set function phi over a voxel volume I with the
 * explicit update of arXiv 2404.02813, Eq. (1):
 *
 *     phi_{n+1} = phi_n + dt * ( mu * (L phi - kappa) + delta_eps(phi) * (nu * kappa - g) )
 *
 * with (Sec. 3) the Heaviside H_eps of Eq. (10) and its derivative delta_eps of
 * Eq. (14); the local fits f_1 = K*(H I) / K*H and f_2 = K*((1-H) I) / K*(1-H)
 * of Eq. (6), K the normalised discrete Gaussian of Eq. (7) with radius
 * R = round(2 sigma) and zero padding outside the volume; the data terms
 * e_i = (K*1) I^2 - 2 I (K*f_i) + K*(f_i^2) and g = lambda1 e_1 - lambda2 e_2
 * (the directional forces of Eqs. (11)-(12)); kappa = div(grad phi / (|grad phi| + 1e-10))
 * and the 7-point Laplacian L (Eqs. (3)-(4), (13)) with central differences and
 * reflect-101 boundaries (-1 -> 1, n -> n-2).  Every term is evaluated at phi_n.
 *
 * Conventions shared by every entry point
 *  - Volumes are dense, x fastest: element (x, y, z) is at (z*ny + y)*nx + x.
 *  - Each dimension must be >= 4; nx*ny*nz must be <= 2^34.
 *  - Pointers may be host or device memory of the context's device; the
 *    library tells them apart with the CUDA runtime.  Host pointers are
 *    staged through device buffers the library owns.
 *  - The caller owns every pointer it passes.  The library owns every device
 *    buffer it allocates (working fields, staging copies); they are charged
 *    against the context's HBM budget and freed by rsf_destroy.
 *  - No entry point throws, aborts or exits.  Errors are returned as a
 *    negative rsf_status; rsf_last_error() then describes the last one on the
 *    calling thread.
 *  - Arithmetic is FP32 on the GPU with FP32 accumulation in every
 *    convolution; no step runs in FP64 on the GPU.
 */
#ifndef RSF_H
#define RSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsf_ctx rsf_ctx; /* opaque; one per device */

typedef int32_t rsf_status;
#define RSF_OK 0
#define RSF_PENDING 1
#define RSF_SUSPENDED 2      /* final status of a suspended serving request (rsf_suspend) */
#define RSF_E_INVAL (-1)     /* bad argument: null pointer, dim < 4, NaN or non-positive sigma/eps/dt, iters < 0 */
#define RSF_E_NOMEM (-2)     /* the HBM budget or a device allocation was exceeded */
#define RSF_E_CUDA (-3)      /* a CUDA runtime call failed, or a kernel's bounded wait for its
                                TMA copies expired (the context then stays in error: destroy
                                it); see rsf_last_error() */
#define RSF_E_TIMEOUT (-4)   /* rsf_wait: its time limit expired before a final status */
#define RSF_E_NOTFOUND (-5)  /* unknown ticket */
#define RSF_E_BUSY (-6)      /* queue full */
#define RSF_E_CANCELLED (-7) /* request cancelled */

typedef enum { RSF_U8 = 0, RSF_U16 = 1, RSF_F32 = 2 } rsf_dtype;

/* Storage precision of I and the convolved fields (phi is always FP32). */
typedef enum { RSF_STORE_F32 = 0, RSF_STORE_BF16 = 1, RSF_STORE_F16 = 2 } rsf_storage;

/*
 * rsf_create -- open a context on CUDA device `device`.
 *   out               receives the context (set to NULL on failure).
 *   hbm_budget_bytes  upper bound on the device memory the context may hold
 *                     at once; 0 means 90% of the device's free memory.
 *   flags             reserved, must be 0.
 * The context owns one CUDA stream (see rsf_stream) on which all its work runs.
 * Errors: RSF_E_INVAL (out NULL, flags != 0), RSF_E_CUDA (no such device).
 */
rsf_status rsf_create(rsf_ctx **out, int device, uint64_t hbm_budget_bytes, uint32_t flags);

/* rsf_destroy -- wait for the context's work, free every buffer it owns, and
 * release it.  NULL is ignored. */
void rsf_destroy(rsf_ctx *ctx);

/* rsf_stream -- the context's cudaStream_t (as void*), for callers that time
 * or order work around the library's launches. */
void *rsf_stream(rsf_ctx *ctx);

/*
 * rsf_evolve -- run `iters` iterations of Eq. (1) from phi0 and write the
 * result to phi_out.  Blocking: returns once phi_out holds the result.
 *   volume   nx*ny*nz image values of type vt (RSF_U8, RSF_U16 or RSF_F32).
 *   phi0     nx*ny*nz FP32 initial level set (phi > 0 is the H side, fit f_1).
 *   phi_out  nx*ny*nz FP32 result; may alias phi0.
 *   sigma    Gaussian width (> 0); R = round(2 sigma) must be <= 16.
 *   eps      Heaviside width (> 0).
 *   lambda1, lambda2  weights of e_1 and e_2.
 *   nu       weight of the curvature term delta * kappa.
 *   mu       weight of the regulariser L phi - kappa.
 *   dt       time step (> 0).
 *   iters    number of iterations (>= 0; 0 copies phi0 to phi_out).
 * Set-up work (centring of I, the K*1 profiles) runs once per call.
 * Errors: RSF_E_INVAL, RSF_E_NOMEM, RSF_E_CUDA.
 */
rsf_status rsf_evolve(rsf_ctx *ctx, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                      const float *phi0, float *phi_out, float sigma, float eps, float lambda1, float lambda2,
                      float nu, float mu, float dt, int32_t iters);

/*
 * rsf_evolve_batch -- evolve `nbricks` independent bricks together.
 *
 * Each brick is a volume of its own (for example a halo-padded sub-volume of
 * a larger image, the volume-level parallelism of Sec. 4.1) with its own
 * parameters and iteration count; its result is the same as rsf_evolve on the
 * same brick with the same context options (every voxel is computed by the
 * same arithmetic in the same order).  All bricks start together and advance
 * one iteration per step, one launch per kernel for each group of bricks that
 * share a kernel radius and image type; a brick that has done its iterations
 * retires and its phi is copied to its phi_out.  Between retirements the
 * iteration is replayed from a captured CUDA graph (RSF_OPT_GRAPH).
 *   bricks    array of nbricks descriptors (fields as in rsf_evolve); host or
 *             device pointers; phi_out may alias phi0.
 * Only the tiled kernels run batched: every brick's radius round(2 sigma) must
 * be one of 2-6, 8, 10, 12.  Blocking.  Device memory for all bricks is taken
 * at once from the context's HBM budget.
 * Errors: RSF_E_INVAL (a brick's arguments, with its index in the message),
 * RSF_E_NOMEM, RSF_E_CUDA.
 */
typedef struct {
    const void *volume;
    rsf_dtype vt;
    int64_t nx, ny, nz;
    const float *phi0;
    float *phi_out;
    float sigma, eps, lambda1, lambda2, nu, mu, dt;
    int32_t iters;
} rsf_brick;

rsf_status rsf_evolve_batch(rsf_ctx *ctx, const rsf_brick *bricks, int32_t nbricks);

/*
 * rsf_evolve_curtain -- the volume-level parallelism of Sec. 4.1: the volume
 * is divided into overlapping sub-volumes, each is evolved as a volume of its
 * own (all together, as by rsf_evolve_batch), and neighbouring results are
 * merged by linear interpolation across the overlap (the curtain).
 *   Along each axis of length n, sub-volumes of `edge` voxels start at
 *   multiples of edge - curtain and the last one is moved to end at n (one
 *   sub-volume when edge >= n); neighbours overlap by at least `curtain`.
 *   Sub-volume b has the weight w_b(x) = product over the axes of h, with
 *   h = 1 inside, min(1, (x - s + 1/2)/curtain) after a start face s > 0 and
 *   min(1, (e - x - 1/2)/curtain) before an end face e < n; the result is
 *   sum_b w_b phi_b / sum_b w_b (FP32).
 *   edge      sub-volume edge in voxels, >= 4.
 *   curtain   overlap in voxels, 1 <= curtain <= edge / 2.
 * The other arguments are those of rsf_evolve (host or device pointers;
 * phi_out may alias phi0).  The context's storage and force options apply;
 * round(2 sigma) must be a radius with tiled kernels.  Blocking.  Device
 * memory: every sub-volume's image and phi, staging of host inputs, plus
 * what rsf_evolve_batch takes.
 * Errors: RSF_E_INVAL (arguments), RSF_E_NOMEM, RSF_E_CUDA.
 */
rsf_status rsf_evolve_curtain(rsf_ctx *ctx, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                              const float *phi0, float *phi_out, float sigma, float eps, float lambda1,
                              float lambda2, float nu, float mu, float dt, int32_t iters, int32_t edge,
                              int32_t curtain);

/*
 * rsf_init_phi0 -- the seed initialisation of Sec. 4.3: blob seeds from the
 * determinant of the Hessian in every z slice, then phi0 = r0 - the Euclidean
 * distance to the nearest seed (the distance the paper's fast sweeping
 * approximates, here exact).
 *   Taps of the sampled Gaussian and its first and second derivatives,
 *   k = -R..R, R = round(3 s): g_k = exp(-k^2/2s^2)/sum, g'_k = -(k/s^2) g_k,
 *   g''_k = (k^2/s^4 - 1/s^2) g_k; in-slice correlation with zero padding:
 *   I_xx = (g'' in x, g in y), I_yy = (g in x, g'' in y), I_xy = (g' in x,
 *   g' in y); response D = s^4 (I_xx I_yy - I_xy^2) where I_xx + I_yy < 0,
 *   else -inf.  A voxel is a seed when D > t * (maximum of D over its slice),
 *   that maximum > 0, and D exceeds D at each existing in-slice neighbour.
 *   blob_sigma     s > 0 with round(3 s) <= 16
 *   rel_threshold  t in [0, 1)
 *   r0             > 0, the radius of the initial regions around the seeds
 *   phi0_out       nx*ny*nz floats, host or device
 *   nseeds         receives the number of seeds
 *   seeds_out      optional nx*ny*nz bytes, 1 at seeds (host or device, or NULL)
 *   response_out   optional nx*ny*nz floats, D (host or device, or NULL)
 * Dimensions: nx, ny in [4, 2^20], nz in [1, 2^20], with the largest squared
 * distance below 2^24 (it is then exact in FP32).  Blocking.
 * Errors: RSF_E_INVAL (arguments; no seed found: phi0_out is left untouched,
 * seeds_out and response_out are written), RSF_E_NOMEM, RSF_E_CUDA.
 */
rsf_status rsf_init_phi0(rsf_ctx *ctx, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                         float blob_sigma, float rel_threshold, float r0, float *phi0_out, int64_t *nseeds,
                         uint8_t *seeds_out, float *response_out);

/*
 * rsf_overlap -- segmentation scores (the paper's Dice coefficient and Jaccard
 * index, Sec. 5.3): counts[0] = |phi > 0|, counts[1] = |truth != 0|,
 * counts[2] = |phi > 0 and truth != 0| over n voxels.  Dice = 2 c2/(c0 + c1),
 * Jaccard = c2/(c0 + c1 - c2).
 *   phi, truth   n floats and n bytes, host or device.
 * Blocking.  Errors: RSF_E_INVAL, RSF_E_NOMEM, RSF_E_CUDA.
 */
rsf_status rsf_overlap(rsf_ctx *ctx, const float *phi, const uint8_t *truth, int64_t n, int64_t counts[3]);

/*
 * rsf_isosurface -- the phi = iso surface as triangles (the surfaces the paper
 * renders, Figs. 8-9), by marching tetrahedra: every voxel cube is split into
 * six tetrahedra along its main diagonal (corners 0, e_a, e_a + e_b, (1,1,1)
 * for each order of the axes); a tetrahedron with 1 or 3 corners where
 * phi > iso gives one triangle, with 2 such corners two; edges are cut by
 * linear interpolation from their corner of smaller grid index; the normal
 * (v1 - v0) x (v2 - v0) points from phi > iso towards phi < iso.
 *   phi          nx*ny*nz floats, host or device; dimensions >= 2.
 *   triangles    capacity * 9 floats (x, y, z of three vertices, voxel units),
 *                host or device, or NULL with capacity 0 to count only.
 *   keys         optional capacity int64: (cube index) * 12 + (tetrahedron) * 2
 *                + (triangle), cube index (z*(ny-1) + y)*(nx-1) + x.
 *   ntriangles   receives the number of triangles of the surface; when it
 *                exceeds capacity only `capacity` of them are written.
 * The set of triangles is deterministic; their order in the output is not.
 * Blocking.  Errors: RSF_E_INVAL, RSF_E_NOMEM, RSF_E_CUDA.
 */
rsf_status rsf_isosurface(rsf_ctx *ctx, const float *phi, int64_t nx, int64_t ny, int64_t nz, float iso,
                          float *triangles, int64_t *keys, int64_t capacity, int64_t *ntriangles);

/*
 * rsf_step_stages -- one iteration from phi with the intermediate fields
 * written out, for checking each stage against a reference.
 *   stages   host or device buffer of RSF_NSTAGES * nx*ny*nz floats,
 *            slot s at offset s*nx*ny*nz, in the order of rsf_stage_id.
 *   phi_next nx*ny*nz FP32 result of the iteration.
 * Other arguments as rsf_evolve.  Errors as rsf_evolve.
 */
typedef enum {
    RSF_STAGE_F1 = 0,   /* local fit f_1 (Eq. 6, H side) */
    RSF_STAGE_F2 = 1,   /* local fit f_2 (Eq. 6, 1-H side) */
    RSF_STAGE_G = 2,    /* g = lambda1 e_1 - lambda2 e_2 */
    RSF_STAGE_KAPPA = 3,/* curvature div(grad phi / |grad phi|) */
    RSF_STAGE_LAP = 4,  /* 7-point Laplacian of phi */
    RSF_NSTAGES = 5
} rsf_stage_id;

rsf_status rsf_step_stages(rsf_ctx *ctx, const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                           const float *phi, float *phi_next, float *stages, float sigma, float eps,
                           float lambda1, float lambda2, float nu, float mu, float dt);

/*
 * rsf_set_option -- per-context settings of the iteration schedule.
 *   RSF_OPT_PATH    RSF_PATH_AUTO (default): the tiled four-kernel iteration
 *                   where it has kernels for the radius R (2-6, 8, 10, 12),
 *                   else the six-pass iteration; RSF_PATH_PASSES: always the
 *                   six-pass iteration; RSF_PATH_TILED: the tiled iteration
 *                   (other radii then fail with RSF_E_INVAL).
 *   RSF_OPT_ZCHUNK  z planes per CTA of the z-marching kernel; 0 (default)
 *                   picks enough chunks for about 16 CTAs per SM; else >= 8.
 *                   Results do not depend on it.
 *   RSF_OPT_STORAGE rsf_storage of the tiled path's stored fits'
 *                   combinations a, b; RSF_STORE_F32 (default), RSF_STORE_BF16
 *                   or RSF_STORE_F16.  Accumulation is FP32 throughout; phi,
 *                   the image (read in its own type), the x/y-convolved pair
 *                   (H I, H), K*I and the x/y-convolved a, b stay exact /
 *                   FP32 (group A forms K*((1-H) I) and K*(1-H) as
 *                   differences, which 16-bit storage would not survive).
 *                   16-bit storage needs the tiled path.
 *   RSF_OPT_AUTOTUNE 1: rsf_evolve_batch picks each brick group's launch
 *                   shape by timing discarded first iterations, one knob after
 *                   the other: z planes per CTA of the x/y kernels (16, 8, 32),
 *                   the update kernel's z chunk (a size heuristic, 32, 64, 128,
 *                   256) and the brick-to-CTA order (largest or smallest bricks
 *                   first); the choice is remembered in the context per group
 *                   (radius, image type, storage, form, brick count, size
 *                   class) and listed by rsf_autotune_report.  0 (default):
 *                   16 planes, the size heuristic, largest first.
 *   RSF_OPT_GRAPH   1 (default): rsf_evolve_batch replays its iterations from
 *                   a captured CUDA graph; 0: direct launches.
 *   RSF_OPT_SERVE_SLOTS  the most bricks the serving loop advances together
 *                   (default 64); further requests wait in the queue.  Read
 *                   when the serving loop starts (the first rsf_submit).
 *   RSF_OPT_FAULT_ADMISSION  k > 0: the serving loop fails the set-up of its
 *                   k-th admission with RSF_E_CUDA, on the host, without any
 *                   device work (for testing failure handling); 0: off.  Read
 *                   when the serving loop starts (the first rsf_submit).
 *   RSF_OPT_FAULT_UPLOAD  k > 0: the serving loop's k-th upload of the active
 *                   bricks' launch descriptors fails on the host, without any
 *                   device work (for testing failure handling); the requests
 *                   active at that tick resolve RSF_E_CUDA with phi_out
 *                   unwritten, queued ones are served afterwards; 0: off.
 *                   (A failed launch of a tick is handled the same way.)  Read
 *                   when the serving loop starts (the first rsf_submit).
 *   RSF_OPT_FAULT_WAIT  1: the z pass of group A arms each of its copy barriers
 *                   for 16 bytes more than its TMA copies deliver, so that its
 *                   bounded waits run out (1 s, then 1 s more for the copies in
 *                   flight) and the kernel records the expiry in the context's
 *                   error word: the call returns RSF_E_CUDA, and so does every
 *                   later call on the context (for testing the device-side
 *                   failure path; no fault is raised); 0 (default): off.  Read
 *                   per call (per descriptor upload in the serving loop).
 *   RSF_OPT_FORCE   the data terms e_1, e_2 of the force: RSF_FORCE_LI
 *                   (default), Li et al.'s e_i = (K*1) I^2 - 2 I K*f_i +
 *                   K*(f_i^2), read into Eqs. (11)-(12), which convolve the
 *                   fits again (six convolved fields per iteration);
 *                   RSF_FORCE_EQ15, the paper's own Eq. (15) with sigma_2 = 0,
 *                   its setting for the 3-D runs (Sec. 5.3): e_i = (I - f_i)^2
 *                   (four convolved fields).  RSF_FORCE_EQ15 needs the tiled
 *                   path (RSF_E_INVAL otherwise).  rsf_evolve, rsf_step_stages
 *                   and rsf_evolve_batch read it per call; rsf_submit per
 *                   request.
 *   RSF_OPT_POISON  1: before each solve (rsf_evolve, rsf_step_stages, each
 *                   brick of rsf_evolve_batch, each served request at
 *                   admission) fill the working fields the iteration writes
 *                   before it reads them -- the intermediate fields, the
 *                   second phi buffer and both Heaviside-argument buffers --
 *                   with all-ones bytes, a NaN in FP32, FP16 and BF16: a
 *                   result that depends on memory the iteration did not write
 *                   then carries NaN or differs from the unpoisoned one (a
 *                   check for tests, in place of a memory sanitizer); 0
 *                   (default): off.  Read per call; the serving loop reads it
 *                   when it starts.
 * The paths give the same result per voxel up to the order of FP32 rounding.
 * Errors: RSF_E_INVAL (unknown key or value).
 */
#define RSF_OPT_PATH 1
#define RSF_OPT_ZCHUNK 2
#define RSF_OPT_STORAGE 3
#define RSF_OPT_AUTOTUNE 4
#define RSF_OPT_GRAPH 5
#define RSF_OPT_FAULT_ADMISSION 6
#define RSF_OPT_SERVE_SLOTS 7
#define RSF_OPT_FORCE 8
#define RSF_OPT_POISON 9
#define RSF_OPT_FAULT_UPLOAD 10
#define RSF_OPT_FAULT_WAIT 11
#define RSF_FORCE_LI 0
#define RSF_FORCE_EQ15 1
#define RSF_PATH_AUTO 0
#define RSF_PATH_PASSES 1
#define RSF_PATH_TILED 2
rsf_status rsf_set_option(rsf_ctx *ctx, int32_t key, int64_t value);

/*
 * rsf_autotune_report -- the launch shapes the batch autotuner chose in this
 * context (RSF_OPT_AUTOTUNE), one text line per brick group:
 *   "<group key> zc=<z chunk> xyp=<x/y planes per CTA> order=<largest|smallest>
 *    ms=<iteration time of the choice> default_ms=<iteration time with the
 *    defaults>"
 * written NUL-terminated into buf (cap bytes, truncated to fit); "" when
 * nothing was tuned.  A tuning aid with no counterpart in the paper.
 * Errors: RSF_E_INVAL (null context, null buffer or cap <= 0).
 */
rsf_status rsf_autotune_report(rsf_ctx *ctx, char *buf, int32_t cap);

/*
 * Serving: continuous batching of brick requests (no counterpart in the
 * paper's method beyond its independent sub-volumes, Sec. 4.1).
 *
 * rsf_submit queues a request and returns at once with a ticket.  A
 * scheduler thread of the context admits queued requests in arrival order
 * while their device footprint fits the context's HBM budget, keeps every
 * admitted brick's phi and working fields resident on the device, and
 * advances all admitted bricks together one iteration per step (continuous
 * batching: a request admitted while others run joins at the next step; a
 * brick that has done its iterations leaves at once and frees its memory for
 * the next admission).  Each brick's result is the same as rsf_evolve on that
 * brick with the same storage.
 *   volume, phi0, phi_out  host or device pointers; the caller keeps them
 *            valid and unchanged until the ticket is no longer pending.
 *            Host images are copied at admission; pinned host memory keeps
 *            that copy asynchronous.
 *   storage  RSF_STORE_F32 / BF16 / F16 for this brick's intermediate fields.
 *   halo     the padding already included in nx, ny, nz on each side (for the
 *            caller's bookkeeping; -1 = 3 sigma); it must leave a core.
 *   stream   NULL, or a cudaStream_t whose work queued before admission must
 *            finish before the brick's inputs are read.
 * Errors of rsf_submit: RSF_E_INVAL (arguments), RSF_E_NOMEM (the request
 * alone exceeds the HBM budget), RSF_E_BUSY (queue full).
 *
 * rsf_poll returns RSF_PENDING, or the request's final status (RSF_OK,
 * RSF_SUSPENDED, RSF_E_CANCELLED, RSF_E_NOMEM, RSF_E_CUDA) together with its latency from
 * submission to completion in seconds (nullable); a ticket is released by the
 * first poll that returns a final status (later polls: RSF_E_NOTFOUND).
 * rsf_wait blocks up to timeout_ms (< 0: no limit) for a final status, then
 * behaves as rsf_poll; on expiry it returns RSF_E_TIMEOUT and keeps the ticket.
 * Active requests are advanced in four lanes by voxel count (below 2^19, 2^21,
 * 2^23 voxels, and larger), each on its own stream; within a lane every brick
 * advances one iteration per tick, in dispatches of one to eight ticks: while
 * no brick of the lane is due to finish and nothing waits in the queue, a
 * dispatch enqueues several ticks without a host round trip.
 * rsf_cancel marks a request cancelled: it leaves the queue, or the batch at
 * the end of the current dispatch, and its phi_out is not written.
 * rsf_suspend marks a request for suspension (checkpointing): it leaves the
 * queue, or the batch at the end of the current dispatch; phi_out receives phi after the
 * iterations it completed (phi0 itself if none), their count is written to
 * *iters_done (host memory, nullable, valid until the ticket resolves), and
 * the final status is RSF_SUSPENDED.  phi and the iteration count are the
 * whole state of the method: submitting phi_out with the remaining
 * iterations (same volume, parameters, storage and form) resumes it, and the
 * result equals the uninterrupted one bit for bit.  A request that finishes
 * its iterations in the same step ends with RSF_OK instead.  Errors:
 * RSF_E_NOTFOUND (unknown or already resolved ticket).
 * rsf_serve_stats reports counts, completed voxel-iterations, the busy time
 * from the first submission to the last completion, and latency percentiles
 * of the completed requests.
 */
typedef struct {
    const void *volume;
    rsf_dtype vt;
    int64_t nx, ny, nz;
    const float *phi0;
    float *phi_out;
    float sigma, eps, lambda1, lambda2, nu, mu, dt;
    int32_t iters;
    rsf_storage storage;
    int32_t halo;
    void *stream;
} rsf_request;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, queued;
    double voxel_iterations;
    double busy_s;
    double latency_p50_s, latency_p99_s, latency_max_s;
    uint64_t suspended;
} rsf_serve_stat;

rsf_status rsf_submit(rsf_ctx *ctx, const rsf_request *req, uint64_t *ticket);
rsf_status rsf_poll(rsf_ctx *ctx, uint64_t ticket, double *latency_s);
rsf_status rsf_wait(rsf_ctx *ctx, uint64_t ticket, int32_t timeout_ms);
rsf_status rsf_cancel(rsf_ctx *ctx, uint64_t ticket);
rsf_status rsf_suspend(rsf_ctx *ctx, uint64_t ticket, int32_t *iters_done);
rsf_status rsf_serve_stats(rsf_ctx *ctx, rsf_serve_stat *out);

/*
 * Kernel timing.  While enabled, the context records a CUDA event pair on its
 * stream around every launch of its per-iteration kernels; rsf_prof_get
 * returns, for the kernel named `kernel` (see rsf_prof_name), the number of
 * launches and their summed device time in milliseconds since the last
 * rsf_prof_enable(ctx, 1).  Errors: RSF_E_INVAL (unknown kernel index).
 */
rsf_status rsf_prof_enable(rsf_ctx *ctx, int32_t on);
int32_t rsf_prof_count(void);
const char *rsf_prof_name(int32_t kernel);
rsf_status rsf_prof_get(rsf_ctx *ctx, int32_t kernel, int64_t *launches, double *total_ms);

/*
 * rsf_evolve_noalloc -- rsf_evolve for small volumes without any device
 * allocation.  The paper has no counterpart; this entry exists for callers
 * that may not allocate GPU memory while they run: a plug-in whose host
 * application owns all device memory through its own pool, a streaming or
 * real-time thread that cannot afford the device-wide synchronisation a
 * cudaMalloc / cudaFree may cause, or a service whose memory was sized once
 * at start-up.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   volume, phi0, phi_out  DEVICE pointers of the current device (host
 *            pointers are rejected with RSF_E_INVAL); phi_out may alias phi0.
 *   stream   the cudaStream_t (as void*) the work is queued on; NULL is the
 *            legacy default stream.
 *   other arguments as rsf_evolve.
 * Working fields live in one static device array built into the library
 * (about 10.5 MB, held by every GPU that loads librsf.so until the process
 * exits), which limits the volume to nx*ny*nz <= 262144 voxels (e.g. 64^3);
 * larger volumes are rejected with RSF_E_INVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Asynchronous:
 * returns once the work is queued; phi_out is ready when `stream` reaches it.
 * All calls on a device share the array and it keeps the last call's
 * contents (nothing in it needs to start at zero); calls whose work overlaps
 * on the GPU race on it and must be serialised by the caller.
 * Errors: RSF_E_INVAL (arguments, size limit), RSF_E_CUDA (launch failures).
 */
rsf_status rsf_evolve_noalloc(const void *volume, rsf_dtype vt, int64_t nx, int64_t ny, int64_t nz,
                              const float *phi0, float *phi_out, float sigma, float eps, float lambda1,
                              float lambda2, float nu, float mu, float dt, int32_t iters, void *stream);

/* Thread-local description of the last error returned on this thread. */
const char *rsf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RSF_H */
