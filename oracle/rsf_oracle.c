/*
 * rsf_oracle.c -- plain, slow FP64 CPU oracle of one 3D RSF level-set
 * iteration and of the iterated evolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library: the Gaussian taps, the Heaviside / Dirac functions, the
 * convolutions and the stencils are all written out again here.
 *
 * What is computed (3D region-scalable fitting, arXiv 2404.02813):
 *   Eq. (1)     phi_{n+1} = phi_n + dt * E
 *   Eq. (13)    E = mu*(L phi - kappa) + delta(phi) * (nu*kappa + F)
 *   Eq. (6)     f_1 = K*(H I) / K*H,  f_2 = K*((1-H) I) / K*(1-H)
 *   Eq. (7)     K: Gaussian of width sigma, here the discrete taps
 *               exp(-k^2 / 2 sigma^2), k = -R..R, R = round(2 sigma),
 *               normalised to sum 1 (the printed normalisation is garbled)
 *   Eq. (8)-(10) H = H_eps(phi) = 1/2 (1 + 2/pi atan(phi/eps)), H_- = 1 - H
 *   Eq. (11)-(12) with Li et al.'s data terms (force mode 0):
 *               e_i = (K*1) I^2 - 2 I (K*f_i) + K*(f_i^2),
 *               F = -(lambda1 e_1 - lambda2 e_2)
 *   Eq. (15)    the paper's own force with sigma_2 = 0, its setting for the
 *               3-D runs (Sec. 5.3), force mode 1: K(sigma_2) is the
 *               identity, so F_+- = I^2 - 2 r_+- I + r_+-^2 = (I - r_+-)^2
 *               with r_+ = f_1, r_- = f_2; e_i = (I - f_i)^2 in the same F
 *   Eq. (3)-(4) kappa = div(grad phi / |grad phi|) (the printed operator is
 *               garbled; the curvature reading), L = 7-point Laplacian
 *   Eq. (14)    delta_eps(u) = (eps/pi) / (eps^2 + u^2)
 *
 * Readings where the paper is silent: zero padding outside the volume for
 * every convolution; reflect-101 index mapping (-1 -> 1, n -> n-2) for every
 * finite difference, including the difference of the unit normal; central
 * differences D_a F = (F(i+e_a) - F(i-e_a)) / 2; unit normal
 * grad phi / (|grad phi| + 1e-10); isotropic unit voxel spacing; explicit
 * Euler with every term taken at phi_n.
 *
 * Layout: every field is a dense [nz][ny][nx] array of double, x fastest,
 * index (z*ny + y)*nx + x.
 *
 * Compiled twice by the build: once plain (-O2, single thread) and once with
 * -fopenmp.  The OpenMP build only splits loops over independent output
 * voxels, so both give bit-identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

typedef int64_t i64;

static i64 idx3(i64 x, i64 y, i64 z, i64 nx, i64 ny) { return (z * ny + y) * nx + x; }

/* ---------------------------------------------------------------- kernel */

/* Kernel radius R = round(2 sigma), halves rounded away from zero. */
int rsf_oracle_radius(double sigma) { return (int)floor(2.0 * sigma + 0.5); }

/* Normalised discrete Gaussian taps g[0..2R], g[k+R] ~ exp(-k^2/(2 sigma^2)).
 * Eq. (7), with the normalising constant replaced by the discrete sum. */
int rsf_oracle_taps(double sigma, double *g)
{
    int R = rsf_oracle_radius(sigma);
    double s = 0.0;
    for (int k = -R; k <= R; ++k) {
        g[k + R] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        s += g[k + R];
    }
    for (int k = 0; k < 2 * R + 1; ++k) g[k] /= s;
    return R;
}

/* One 1-D pass along axis `axis` (0 = x, 1 = y, 2 = z) with zero padding:
 * out(i) = sum_{k=-R..R} g[k+R] * in(i + k e_axis), in = 0 outside. */
static void conv_axis(const double *in, double *out, i64 nx, i64 ny, i64 nz,
                      const double *g, int R, int axis)
{
    i64 n_a = axis == 0 ? nx : (axis == 1 ? ny : nz);
    i64 stride = axis == 0 ? 1 : (axis == 1 ? nx : nx * ny);
#pragma omp parallel for schedule(static)
    for (i64 z = 0; z < nz; ++z)
        for (i64 y = 0; y < ny; ++y)
            for (i64 x = 0; x < nx; ++x) {
                i64 i = axis == 0 ? x : (axis == 1 ? y : z);
                i64 p = idx3(x, y, z, nx, ny);
                double acc = 0.0;
                for (int k = -R; k <= R; ++k) {
                    i64 j = i + k;
                    if (j < 0 || j >= n_a) continue;
                    acc += g[k + R] * in[p + k * stride];
                }
                out[p] = acc;
            }
}

/* Separable 3-D Gaussian convolution K*F: x pass, then y, then z. */
void rsf_oracle_conv3(const double *in, double *out, i64 nx, i64 ny, i64 nz, double sigma)
{
    double g[256];
    int R = rsf_oracle_taps(sigma, g);
    i64 N = nx * ny * nz;
    double *t1 = (double *)malloc(sizeof(double) * N);
    double *t2 = (double *)malloc(sizeof(double) * N);
    conv_axis(in, t1, nx, ny, nz, g, R, 0);
    conv_axis(t1, t2, nx, ny, nz, g, R, 1);
    conv_axis(t2, out, nx, ny, nz, g, R, 2);
    free(t1);
    free(t2);
}

/* ------------------------------------------------------ pointwise terms */

/* Eq. (10). */
double rsf_oracle_heaviside(double u, double eps)
{
    return 0.5 * (1.0 + (2.0 / ORACLE_PI) * atan(u / eps));
}

/* Eq. (14). */
double rsf_oracle_dirac(double u, double eps)
{
    return (eps / ORACLE_PI) / (eps * eps + u * u);
}

/* -------------------------------------------------------------- stencils */

/* Reflect-101 index map onto [0, n): -1 -> 1, n -> n-2. Needs n >= 2. */
static i64 refl(i64 i, i64 n)
{
    if (i < 0) return -i;
    if (i >= n) return 2 * (n - 1) - i;
    return i;
}

static double at_refl(const double *F, i64 x, i64 y, i64 z, i64 nx, i64 ny, i64 nz)
{
    return F[idx3(refl(x, nx), refl(y, ny), refl(z, nz), nx, ny)];
}

/* Curvature kappa = D_x n_x + D_y n_y + D_z n_z with n = grad phi/(|grad phi|+1e-10),
 * and the 7-point Laplacian, both with reflect-101 boundaries (Eqs. (3)-(4)). */
void rsf_oracle_stencils(const double *phi, i64 nx, i64 ny, i64 nz,
                         double *kappa, double *lap)
{
    i64 N = nx * ny * nz;
    double *n0 = (double *)malloc(sizeof(double) * N);
    double *n1 = (double *)malloc(sizeof(double) * N);
    double *n2 = (double *)malloc(sizeof(double) * N);
#pragma omp parallel for schedule(static)
    for (i64 z = 0; z < nz; ++z)
        for (i64 y = 0; y < ny; ++y)
            for (i64 x = 0; x < nx; ++x) {
                double gx = (at_refl(phi, x + 1, y, z, nx, ny, nz) - at_refl(phi, x - 1, y, z, nx, ny, nz)) / 2.0;
                double gy = (at_refl(phi, x, y + 1, z, nx, ny, nz) - at_refl(phi, x, y - 1, z, nx, ny, nz)) / 2.0;
                double gz = (at_refl(phi, x, y, z + 1, nx, ny, nz) - at_refl(phi, x, y, z - 1, nx, ny, nz)) / 2.0;
                double m = sqrt(gx * gx + gy * gy + gz * gz) + 1e-10;
                i64 p = idx3(x, y, z, nx, ny);
                n0[p] = gx / m;
                n1[p] = gy / m;
                n2[p] = gz / m;
            }
#pragma omp parallel for schedule(static)
    for (i64 z = 0; z < nz; ++z)
        for (i64 y = 0; y < ny; ++y)
            for (i64 x = 0; x < nx; ++x) {
                i64 p = idx3(x, y, z, nx, ny);
                double k = (at_refl(n0, x + 1, y, z, nx, ny, nz) - at_refl(n0, x - 1, y, z, nx, ny, nz)) / 2.0
                         + (at_refl(n1, x, y + 1, z, nx, ny, nz) - at_refl(n1, x, y - 1, z, nx, ny, nz)) / 2.0
                         + (at_refl(n2, x, y, z + 1, nx, ny, nz) - at_refl(n2, x, y, z - 1, nx, ny, nz)) / 2.0;
                double c = phi[p];
                double l = (at_refl(phi, x + 1, y, z, nx, ny, nz) + at_refl(phi, x - 1, y, z, nx, ny, nz) - 2.0 * c)
                         + (at_refl(phi, x, y + 1, z, nx, ny, nz) + at_refl(phi, x, y - 1, z, nx, ny, nz) - 2.0 * c)
                         + (at_refl(phi, x, y, z + 1, nx, ny, nz) + at_refl(phi, x, y, z - 1, nx, ny, nz) - 2.0 * c);
                kappa[p] = k;
                lap[p] = l;
            }
    free(n0);
    free(n1);
    free(n2);
}

/* ------------------------------------------------------------- one step */

/* Stage dump slots (each an N-element block of `dump`, when dump != NULL). */
enum {
    DUMP_H = 0,   /* H_eps(phi)                         */
    DUMP_F1,      /* f_1 = K*(H I) / K*H               */
    DUMP_F2,      /* f_2 = K*((1-H) I) / K*(1-H)       */
    DUMP_E1,      /* e_1                                 */
    DUMP_E2,      /* e_2                                 */
    DUMP_G,       /* lambda1 e_1 - lambda2 e_2           */
    DUMP_KAPPA,   /* div(grad phi / |grad phi|)          */
    DUMP_LAP,     /* 7-point Laplacian                   */
    DUMP_NSLOTS
};

int rsf_oracle_dump_slots(void) { return DUMP_NSLOTS; }

/* One iteration given the precomputed K*1 (K1) and K*I (unused here: the
 * complement fit convolves (1-H) I directly) fields.  Writes phi_next. */
enum { FORCE_LI = 0, FORCE_EQ15 = 1 };

static void step_with(const double *I, const double *K1, const double *phi, double *phi_next,
                      i64 nx, i64 ny, i64 nz, double sigma, double eps,
                      double lambda1, double lambda2, double nu, double mu, double dt,
                      double *dump, int force)
{
    i64 N = nx * ny * nz;
    double *H = (double *)malloc(sizeof(double) * N);
    double *a = (double *)malloc(sizeof(double) * N);
    double *b = (double *)malloc(sizeof(double) * N);
    double *c = (double *)malloc(sizeof(double) * N);
    double *d = (double *)malloc(sizeof(double) * N);
    double *f1 = (double *)malloc(sizeof(double) * N);
    double *f2 = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    double *kap = (double *)malloc(sizeof(double) * N);
    double *lap = (double *)malloc(sizeof(double) * N);

    /* Eqs. (8)-(10) */
    for (i64 p = 0; p < N; ++p) H[p] = rsf_oracle_heaviside(phi[p], eps);

    /* Eq. (6), H_+ side: f_1 = K*(H I) / K*H */
    for (i64 p = 0; p < N; ++p) a[p] = H[p] * I[p];
    rsf_oracle_conv3(a, b, nx, ny, nz, sigma);
    rsf_oracle_conv3(H, c, nx, ny, nz, sigma);
    for (i64 p = 0; p < N; ++p) f1[p] = b[p] / c[p];

    /* Eq. (6), H_- side, convolving the complement directly */
    for (i64 p = 0; p < N; ++p) { a[p] = (1.0 - H[p]) * I[p]; d[p] = 1.0 - H[p]; }
    rsf_oracle_conv3(a, b, nx, ny, nz, sigma);
    rsf_oracle_conv3(d, c, nx, ny, nz, sigma);
    for (i64 p = 0; p < N; ++p) f2[p] = b[p] / c[p];

    if (force == FORCE_EQ15) {
        /* Eq. (15), sigma_2 = 0: e_i = (I - f_i)^2, g = l1 e1 - l2 e2 */
        for (i64 p = 0; p < N; ++p) {
            double e1 = (I[p] - f1[p]) * (I[p] - f1[p]);
            double e2 = (I[p] - f2[p]) * (I[p] - f2[p]);
            g[p] = lambda1 * e1 - lambda2 * e2;
            if (dump) { dump[DUMP_E1 * N + p] = e1; dump[DUMP_E2 * N + p] = e2; }
        }
    } else {
    /* Eqs. (11)-(12): e_i = K1 I^2 - 2 I K*f_i + K*f_i^2, g = l1 e1 - l2 e2 */
    rsf_oracle_conv3(f1, a, nx, ny, nz, sigma);                  /* K*f1   */
    for (i64 p = 0; p < N; ++p) d[p] = f1[p] * f1[p];
    rsf_oracle_conv3(d, b, nx, ny, nz, sigma);                   /* K*f1^2 */
    for (i64 p = 0; p < N; ++p) {
        double e1 = K1[p] * I[p] * I[p] - 2.0 * I[p] * a[p] + b[p];
        g[p] = lambda1 * e1;
        if (dump) dump[DUMP_E1 * N + p] = e1;
    }
    rsf_oracle_conv3(f2, a, nx, ny, nz, sigma);                  /* K*f2   */
    for (i64 p = 0; p < N; ++p) d[p] = f2[p] * f2[p];
    rsf_oracle_conv3(d, b, nx, ny, nz, sigma);                   /* K*f2^2 */
    for (i64 p = 0; p < N; ++p) {
        double e2 = K1[p] * I[p] * I[p] - 2.0 * I[p] * a[p] + b[p];
        g[p] -= lambda2 * e2;
        if (dump) dump[DUMP_E2 * N + p] = e2;
    }
    }

    /* Eqs. (3)-(4) */
    rsf_oracle_stencils(phi, nx, ny, nz, kap, lap);

    /* Eqs. (1), (13), (14) */
    for (i64 p = 0; p < N; ++p) {
        double del = rsf_oracle_dirac(phi[p], eps);
        double E = mu * (lap[p] - kap[p]) + del * (nu * kap[p] - g[p]);
        phi_next[p] = phi[p] + dt * E;
    }

    if (dump) {
        memcpy(dump + DUMP_H * N, H, sizeof(double) * N);
        memcpy(dump + DUMP_F1 * N, f1, sizeof(double) * N);
        memcpy(dump + DUMP_F2 * N, f2, sizeof(double) * N);
        memcpy(dump + DUMP_G * N, g, sizeof(double) * N);
        memcpy(dump + DUMP_KAPPA * N, kap, sizeof(double) * N);
        memcpy(dump + DUMP_LAP * N, lap, sizeof(double) * N);
    }
    free(H); free(a); free(b); free(c); free(d);
    free(f1); free(f2); free(g); free(kap); free(lap);
}

/* One iteration phi -> phi_next (phi_next must not alias phi).  `dump`, when
 * not NULL, receives DUMP_NSLOTS blocks of N doubles (see the enum above). */
void rsf_oracle_step(const double *I, const double *phi, double *phi_next,
                     i64 nx, i64 ny, i64 nz, double sigma, double eps,
                     double lambda1, double lambda2, double nu, double mu, double dt,
                     double *dump, int force)
{
    i64 N = nx * ny * nz;
    double *one = (double *)malloc(sizeof(double) * N);
    double *K1 = (double *)malloc(sizeof(double) * N);
    for (i64 p = 0; p < N; ++p) one[p] = 1.0;
    rsf_oracle_conv3(one, K1, nx, ny, nz, sigma);
    step_with(I, K1, phi, phi_next, nx, ny, nz, sigma, eps, lambda1, lambda2, nu, mu, dt, dump, force);
    free(one);
    free(K1);
}

/* `iters` iterations from phi0 (Eq. (1) repeated, Jacobi double buffering).
 * phi_out may alias phi0.  K*1 is computed once. */
void rsf_oracle_evolve(const double *I, const double *phi0, double *phi_out,
                       i64 nx, i64 ny, i64 nz, double sigma, double eps,
                       double lambda1, double lambda2, double nu, double mu, double dt,
                       int iters, int force)
{
    i64 N = nx * ny * nz;
    double *one = (double *)malloc(sizeof(double) * N);
    double *K1 = (double *)malloc(sizeof(double) * N);
    double *pa = (double *)malloc(sizeof(double) * N);
    double *pb = (double *)malloc(sizeof(double) * N);
    for (i64 p = 0; p < N; ++p) one[p] = 1.0;
    rsf_oracle_conv3(one, K1, nx, ny, nz, sigma);
    memcpy(pa, phi0, sizeof(double) * N);
    for (int it = 0; it < iters; ++it) {
        step_with(I, K1, pa, pb, nx, ny, nz, sigma, eps, lambda1, lambda2, nu, mu, dt, NULL, force);
        double *t = pa; pa = pb; pb = t;
    }
    memcpy(phi_out, pa, sizeof(double) * N);
    free(one); free(K1); free(pa); free(pb);
}

/* ------------------------------------------- one voxel, by brute force */

/* phi_{n+1} at the single voxel (px,py,pz), written straight from the
 * definitions with direct triple sums over the 3-D kernel
 * K(a,b,c) = g[a] g[b] g[c] and global-volume bounds checks, without the
 * separable passes.  Used to check sampled voxels of volumes too large for
 * the full oracle, and as an independent check of rsf_oracle_step. */
double rsf_oracle_point_next(const double *I, const double *phi, i64 nx, i64 ny, i64 nz,
                             i64 px, i64 py, i64 pz, double sigma, double eps,
                             double lambda1, double lambda2, double nu, double mu, double dt,
                             double *terms, int force)
{
    double g[256];
    int R = rsf_oracle_taps(sigma, g);
    int W = 4 * R + 1;                      /* box of H values around p, radius 2R */
    double *Hb = (double *)malloc(sizeof(double) * (size_t)W * W * W);
    for (int c = -2 * R; c <= 2 * R; ++c)
        for (int b = -2 * R; b <= 2 * R; ++b)
            for (int a = -2 * R; a <= 2 * R; ++a) {
                i64 x = px + a, y = py + b, z = pz + c;
                double h = 0.0;
                if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)
                    h = rsf_oracle_heaviside(phi[idx3(x, y, z, nx, ny)], eps);
                Hb[((c + 2 * R) * W + (b + 2 * R)) * W + (a + 2 * R)] = h;
            }

    double K1 = 0.0, Kf1 = 0.0, Kf1s = 0.0, Kf2 = 0.0, Kf2s = 0.0, f1p = 0.0, f2p = 0.0;
    for (int c = -R; c <= R; ++c)
        for (int b = -R; b <= R; ++b)
            for (int a = -R; a <= R; ++a) {
                i64 qx = px + a, qy = py + b, qz = pz + c;
                if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
                double w = g[a + R] * g[b + R] * g[c + R];
                /* f_1(q), f_2(q) by direct sums around q */
                double n1 = 0.0, d1 = 0.0, n2 = 0.0, d2 = 0.0;
                for (int cc = -R; cc <= R; ++cc)
                    for (int bb = -R; bb <= R; ++bb)
                        for (int aa = -R; aa <= R; ++aa) {
                            i64 sx = qx + aa, sy = qy + bb, sz = qz + cc;
                            if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz) continue;
                            double ww = g[aa + R] * g[bb + R] * g[cc + R];
                            double h = Hb[((c + cc + 2 * R) * W + (b + bb + 2 * R)) * W + (a + aa + 2 * R)];
                            double iv = I[idx3(sx, sy, sz, nx, ny)];
                            n1 += ww * h * iv;
                            d1 += ww * h;
                            n2 += ww * (1.0 - h) * iv;
                            d2 += ww * (1.0 - h);
                        }
                double f1 = n1 / d1, f2 = n2 / d2;
                if (a == 0 && b == 0 && c == 0) { f1p = f1; f2p = f2; }
                K1 += w;
                Kf1 += w * f1;
                Kf1s += w * f1 * f1;
                Kf2 += w * f2;
                Kf2s += w * f2 * f2;
            }
    free(Hb);

    double Ip = I[idx3(px, py, pz, nx, ny)];
    double e1 = K1 * Ip * Ip - 2.0 * Ip * Kf1 + Kf1s;
    double e2 = K1 * Ip * Ip - 2.0 * Ip * Kf2 + Kf2s;
    if (force == FORCE_EQ15) {          /* Eq. (15), sigma_2 = 0 */
        e1 = (Ip - f1p) * (Ip - f1p);
        e2 = (Ip - f2p) * (Ip - f2p);
    }
    double gg = lambda1 * e1 - lambda2 * e2;

    /* unit normal at a (reflected) voxel, then its central-difference divergence */
    double kap = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        for (int s = -1; s <= 1; s += 2) {
            i64 q[3] = {px, py, pz};
            i64 nn[3] = {nx, ny, nz};
            q[ax] += s;
            q[ax] = refl(q[ax], nn[ax]);
            double gr[3];
            for (int bx = 0; bx < 3; ++bx) {
                i64 u[3] = {q[0], q[1], q[2]}, v[3] = {q[0], q[1], q[2]};
                u[bx] += 1;
                v[bx] -= 1;
                gr[bx] = (at_refl(phi, u[0], u[1], u[2], nx, ny, nz) - at_refl(phi, v[0], v[1], v[2], nx, ny, nz)) / 2.0;
            }
            double m = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]) + 1e-10;
            kap += s * (gr[ax] / m) / 2.0;
        }
    double c0 = phi[idx3(px, py, pz, nx, ny)];
    double lap = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        i64 u[3] = {px, py, pz}, v[3] = {px, py, pz};
        u[ax] += 1;
        v[ax] -= 1;
        lap += at_refl(phi, u[0], u[1], u[2], nx, ny, nz) + at_refl(phi, v[0], v[1], v[2], nx, ny, nz) - 2.0 * c0;
    }
    double del = rsf_oracle_dirac(c0, eps);
    if (terms) {  /* e1, e2, g, kappa, L at the voxel */
        terms[0] = e1;
        terms[1] = e2;
        terms[2] = gg;
        terms[3] = kap;
        terms[4] = lap;
    }
    return c0 + dt * (mu * (lap - kap) + del * (nu * kap - gg));
}
