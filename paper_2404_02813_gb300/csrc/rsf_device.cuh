// rsf_device.cuh -- device-side building blocks of the RSF level-set update
// (arXiv 2404.02813, Sec. 3): the Heaviside and Dirac functions, the
// reflect-101 boundary map of the finite differences, and the parameter
// blocks every kernel receives by value.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsf {

constexpr int RMAX = 16;                 // largest supported kernel radius (sigma <= 8)
constexpr float INV_PI = 0.318309886183790671538f;

// Normalised discrete Gaussian taps of Eq. (7), g[k + R] for k = -R..R.
struct Taps {
    int R;
    float g[2 * RMAX + 1];
};

// Volume shape, x fastest.
struct Dims {
    int nx, ny, nz;
    long long plane;  // nx * ny
    long long n;      // nx * ny * nz
};

// Scalars of the update, Eqs. (1), (13), (14).
struct Coeffs {
    float eps, lambda1, lambda2, nu, mu, dt;
};

// Eq. (10), H = 1/2 + atan(u/eps)/pi, evaluated without cancellation on the
// small side: for u < 0, H = atan(eps/|u|)/pi; for u >= 0, H = 1 - atan(eps/u)/pi.
// (u = 0 gives eps/0 = inf, atan(inf) = pi/2, H = 1/2.)
__device__ __forceinline__ float heaviside(float u, float eps) {
    float r = atanf(eps / fabsf(u)) * INV_PI;
    return u < 0.f ? r : 1.f - r;
}

// 1 - H for the same u, also without cancellation on its small side.
__device__ __forceinline__ float heaviside_c(float u, float eps) {
    float r = atanf(eps / fabsf(u)) * INV_PI;
    return u < 0.f ? 1.f - r : r;
}

// The tiled path stores the small side of Eq. (10), q = atan(eps/|u|)/pi in
// (0, 1/2], carrying the sign of u (heaviside_q_fast in rsf_tiled.cuh); H is
// -q for q < 0, else 1 - q.
__device__ __forceinline__ float h_of_q(float q) { return q < 0.f ? -q : 1.f - q; }
// 1 - H for the same q: 1 + q for q < 0, else q (its small side is q itself).
__device__ __forceinline__ float hc_of_q(float q) { return q < 0.f ? 1.f + q : q; }

// sqrt and reciprocal by the hardware approximations (PTX sqrt.approx.f32,
// rcp.approx.ftz.f32, relative error of a few ulp); used for the unit normal only.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Eq. (14), delta = (eps/pi) / (eps^2 + u^2).
__device__ __forceinline__ float dirac(float u, float eps) {
    return (eps * INV_PI) / (eps * eps + u * u);
}

// Reflect-101 index map onto [0, n): -1 -> 1, n -> n-2 (needs n >= 2 and |overshoot| < n).
__device__ __forceinline__ int refl101(int i, int n) {
    i = i < 0 ? -i : i;
    return i >= n ? 2 * (n - 1) - i : i;
}

}  // namespace rsf
