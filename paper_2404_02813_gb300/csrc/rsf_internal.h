// rsf_internal.h -- host-side interfaces between the C ABI layer and the
// kernel translation units of librsf.so.  Not installed; not part of the ABI.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "rsf_device.cuh"

namespace rsf {

// Kernel identifiers for the per-launch timing of rsf_prof_*.
enum KernelId {
    KID_AX = 0,    // group A, x pass: H products + x convolution
    KID_AY,        // group A, y pass
    KID_AZ,        // group A, z pass + local fits epilogue
    KID_BX,        // group B, x pass
    KID_BY,        // group B, y pass
    KID_BZ,        // group B, z pass + data term, curvature and update epilogue
    KID_TA_XY,     // tiled: group A, H products + x and y convolution
    KID_TA_Z,      // tiled: group A, z convolution + local fits
    KID_TB_XY,     // tiled: group B, x and y convolution
    KID_TB_Z,      // tiled: group B, z convolution + data term, curvature, update
    KID_COUNT
};
const char *kernel_name(int id);

// Records CUDA event pairs around launches while enabled.
struct Profiler {
    bool on = false;
    cudaStream_t stream = nullptr;
    struct Rec { int id; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    int open_id = -1;
    cudaEvent_t open_a = nullptr;

    cudaEvent_t take();
    void begin(int id);
    void end();
    void reset();
    void release();
};

// RAII bracket around one launch.
struct ProfScope {
    Profiler *p;
    ProfScope(Profiler *prof, int id) : p(prof && prof->on ? prof : nullptr) { if (p) p->begin(id); }
    ~ProfScope() { if (p) p->end(); }
};

// Device fields of one volume (all FP32, n elements unless noted).
struct Fields {
    Dims d{};
    float *I = nullptr;       // centred, scaled image  (I - m) / s
    float *prof = nullptr;    // zero-padding profiles p_x[nx], p_y[ny], p_z[nz]; K*1 = p_x p_y p_z
    float *cs = nullptr;      // [0] m, [1] 1/s, [2] s^2, [3] s   (centring constants)
    float *partials = nullptr;// reduction scratch, 3 * kStatBlocks floats
    float *phi[2] = {nullptr, nullptr};
    float *q[2] = {nullptr, nullptr};   // tiled path: +-atan(eps/|phi|)/pi of phi[i]
    float *t[8] = {};         // stage buffers: one block of 8 * capacity floats, t[i] = t[0] + i * capacity,
                              // capacity >= px * ny * nz (the tiled path's pitched fields use the block
                              // as u (float4), ab and abxy (float2) at offsets 0, 4 np, 6 np)
    int px = 0;               // x pitch of the tiled path's intermediate fields (multiple of 32)
};

constexpr int kStatBlocks = 1024;

// Set-up: centring constants, the K*1 profiles and (when `centre`) the
// centred image f.I.  `vol` is a device pointer of dtype vt (0 u8, 1 u16, 2 f32).
cudaError_t setup_image(const void *vol, int vt, const Taps &taps, Fields &f, cudaStream_t s, bool centre = true);

// Centring constants only (f.cs from the image statistics), no other field.
cudaError_t image_stats(const void *vol, int vt, Fields &f, cudaStream_t s);
// Zero-padding profiles p_a(i) = sum of the in-volume taps (double sums rounded
// once), nx + ny + nz floats: K*1 = p_x p_y p_z.
void zero_padding_profiles(const Taps &taps, int nx, int ny, int nz, float *out);

// The centring half of setup_image alone (statistics and centred image, no
// profiles); enqueues on `s` and never synchronises.
cudaError_t centre_image(const void *vol, int vt, Fields &f, cudaStream_t s);

// Sets the calling thread's rsf_last_error() text.
void set_last_error(const char *msg);

// One brick of the tiled path: an independent volume with its own fields and
// scalars.  Device copies of these descriptors drive the batched launches.
struct BrickDev {
    int nx, ny, nz, px;     // dimensions; x pitch of the intermediate fields
    const void *img;        // image, nx*ny*nz values of the group's image type
    const float *cs;        // centring constants [m, 1/s, s^2, s]
    const float *prof;      // K*1 profiles p_x[nx], p_y[ny], p_z[nz]
    float *phi[2], *q[2];   // ping-pong level set and its q = +-atan(eps/|phi|)/pi
    float2 *u2;             // pitched x/y-convolved (H I~, H), FP32 (Eq. (15) form: one float4 per voxel,
                            // ((H I~, H), ((1-H) I~, 1-H)))
    void *ab;               // pitched (a, b), storage type
    float2 *abxy;           // pitched x/y-convolved (a, b), FP32 (also the set-up's scratch for ki;
                            // Eq. (15) form: the fits (f1, f2))
    float *ki;              // pitched K*I~ (the centred image convolved), FP32, set once per solve
    float eps, lambda1, lambda2, nu, mu, dt;
    int zc;                 // z chunk of the update kernel
    int xyp;                // z planes per CTA of the x/y kernels (<= 0: kDefaultXYPlanes)
    int flip;               // this brick's buffer parity is the launch parity xor flip
    float *dump;            // optional 5 * n stage fields (f1, f2, g, kappa, L)
    // TMA descriptors (tiled_encode_maps).  Group A's z pass: u2 as FP32 [nz][ny][c nx]
    // (row pitch c px; c = 2, or 4 in the Eq. (15) form) in boxes of 32 c floats x 1 row x
    // (64 + 2R) planes, and ki as FP32 [nz][ny][nx] in boxes of 32 x 1 x 64.  Group B's x/y
    // kernel (Li's form, FP32 storage, even R): ab as FP32 [nz][ny][2 nx] in boxes of one
    // input tile, 2 tiled_xy_in_pitch(R) floats x (32 + 2R) rows x 1 plane.  Group A's x/y
    // kernel (Li's form, even R, xy_tma): q[0], q[1] as FP32 [nz][ny][nx] and the image in
    // its type, in boxes of one staged plane (16-byte aligned column origin, 32 + 2R rows)
    CUtensorMap tm_u, tm_k, tm_ab, tm_q[2], tm_img;
    int xy_tma;             // 1: tm_q and tm_img are encoded (rows a multiple of 16 bytes, aligned bases)
};

// A set of bricks launched together: same radius, image type and storage.
struct TiledGroup {
    int storage;            // 0 FP32, 1 BF16, 2 FP16 (rsf_storage)
    int force;              // 0 Li's data terms (group B convolutions), 1 Eq. (15) with sigma_2 = 0
    int imgtype;            // 0 uint8, 1 uint16, 2 float
    Taps taps;
    const BrickDev *bricks; // device array of nb descriptors
    int nb;
    const int *starts[4];   // device: per kernel, nb + 1 CTA offsets
    unsigned ncta[4];       // CTAs per kernel launch
    int dump;               // 1: some brick has a stage dump (its update kernel writes g, kappa, L)
    int *err;               // device-visible error word of the kernels' bounded waits (nonzero: expired)
    unsigned fault_tx;      // bytes the TMA barriers expect beyond their copies (0; > 0 in a fault test)
    int xy_tma;             // 1: every brick has xy_tma set; group A's x/y kernel takes its inputs by TMA
};

// Device error word values (TiledGroup::err).
constexpr int kErrWaitExpired = 1;  // a bounded wait for a TMA copy ran out (1 s)
constexpr int kErrSmemAlign = 2;    // a TMA destination in shared memory was not 128-byte aligned

constexpr int kDefaultXYPlanes = 16;

// Tiled four-kernel path (rsf_tiled*.cu) for the radii it is instantiated for.
bool tiled_supports(int R);
// The tiled kernels address a brick's pitched fields with 32-bit offsets: they take
// bricks of fewer than 2^32 pitched voxels.
bool tiled_fits(long long nx, long long ny, long long nz);
int tiled_pitch(int nx);
// Encodes b's tensor maps from its dimensions, pitch and field views for its
// group's form (force), storage and radius R: b.tm_u, b.tm_k (Li's form) and
// b.tm_ab (Li's form, FP32 storage, even R); the others zeroed.
cudaError_t tiled_encode_maps(BrickDev &b, int force, int storage, int imgtype, int R);
// Row pitch (float2) of the x/y kernels' input tile for radius R: 32 + 2R
// rounded up to a multiple of 16, plus 2.
constexpr int tiled_xy_in_pitch(int R) { return ((32 + 2 * R + 15) / 16) * 16 + 2; }
cudaError_t tiled_prepare(int storage, int R, int force);
cudaError_t tiled_iterate(const TiledGroup &g, int parity, Profiler *prof, cudaStream_t s);
void tiled_cta_counts(const BrickDev &b, unsigned counts[4]);
size_t tiled_stage_bytes(int storage, long long np);
// Views of one brick's intermediate fields in a block of tiled_stage_bytes(storage, np)
// bytes, for Li's form (force 0) or the Eq. (15) form (u2 then holds two pairs per
// voxel, abxy the fits (f1, f2); ab and ki are null).
void tiled_stage_views(int storage, int force, void *base, long long np, float2 **u2, void **ab, float2 **abxy,
                       float **ki);
// q = +-atan(eps/|phi|)/pi (sign of phi) before the first tiled iteration.
cudaError_t tiled_q_init(const float *phi, float *q, long long n, float eps, cudaStream_t s);
// b.ki = K*I~ before the first tiled iteration (b.img, b.cs set; uses b.abxy as scratch);
// nothing when b.ki is null (the Eq. (15) form).
cudaError_t tiled_ki_init(const BrickDev &b, int imgtype, const Taps &taps, cudaStream_t s);

// One iteration of the separable pass path: phi_in -> phi_out.
// `stages`, when not null, receives RSF_NSTAGES fields (f1, f2, g, kappa, L).
cudaError_t iterate_passes(const Taps &taps, const Coeffs &c, Fields &f, const float *phi_in, float *phi_out,
                           float *stages, Profiler *prof, cudaStream_t s);

}  // namespace rsf
