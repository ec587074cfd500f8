// Far cells in groups (OBEM_STEP_CELL_GROUPS) for the cell field of
// Eq. (BEM3).  The paper sums every cell for every charge; the cell kernels
// already replace a far cell by a few quadrature points.  Here, in addition,
// cells are grouped (OBEM_GRP_K consecutive in the Morton order of their
// centroids) and a group far from a block of targets is replaced by
// OBEM_GRP_M equivalent point charges on the sphere of the group's radius R
// around its centre.  The charges are the least-squares fit of the group's
// potential at OBEM_GRP_CHECK points on the sphere of OBEM_GRP_RC R (the
// potential outside a sphere holding all sources is fixed by its values on a
// surrounding sphere, so matching it there matches the field beyond).
//
//   obem_cell_groups_build  host, at mesh load: group order, centres, radii,
//                           directions, and the fit matrix for a unit radius
//                           (normal equations, Cholesky, FP64)
//   grp_fit_kernel          one block per group: the group's 7-point rule
//                           sources (FP64 vertices, current sigma), their
//                           potential at the check points, the fitted charges
//                           (FP64, stored as binary32)
//
// The fit depends on sigma only; it is redone when sigma changes.  Measured on
// the CPU with these host arrays for 250 groups of 32 cells of the 60k-cell
// GEM mesh, random-sign densities, against the closed-form field: the 49
// charges give the group's field to 2.8e-6 of sum |q| / d^2 at 8 radii and
// 1.4e-6 at 9 (the separation used; the per-cell tiers are held to 3.6e-6).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "obem_internal.cuh"

// 7-point degree-5 rule on a triangle: the centroid and (a, b, b)
// permutations, written as c + t (v_k - c)
#define G7_W0 0.225
#define G7_W1 0.132394152788506
#define G7_W2 0.125939180544827
#define G7_T1 (-0.410426192315345)
#define G7_T2 0.696140478029631

static uint32_t spread10(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// n points spread over the unit sphere (golden-angle spiral)
static void sphere_points(int n, std::vector<double> &p)
{
    const double pi = 3.14159265358979323846;
    p.resize(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double z = 1.0 - 2.0 * (i + 0.5) / n;
        const double r = sqrt(fmax(0.0, 1.0 - z * z));
        const double th = pi * (1.0 + sqrt(5.0)) * (i + 0.5);
        p[3 * i] = r * cos(th);
        p[3 * i + 1] = r * sin(th);
        p[3 * i + 2] = z;
    }
}

void obem_cell_groups_free(obem_ctx *c)
{
    void *p[] = {c->d_grp_perm, c->d_grp_cr, c->d_grp_h2min, c->d_grp_u, c->d_grp_q, c->d_grp_c64, c->d_grp_v,
                 c->d_grp_pinv};
    for (void *q : p)
        if (q) cudaFree(q);
    c->d_grp_perm = NULL;
    c->d_grp_cr = NULL;
    c->d_grp_h2min = NULL;
    c->d_grp_u = NULL;
    c->d_grp_q = NULL;
    c->d_grp_c64 = NULL;
    c->d_grp_v = NULL;
    c->d_grp_pinv = NULL;
    c->ngrp = 0;
    c->grp_fit_sigma = NULL;
}

// Host side of the groups: order, centres and radii, smallest h^2,
// directions, and the fit matrix (all that the device arrays hold).
struct GroupHost {
    int ng;
    std::vector<int32_t> perm;
    std::vector<float4> cr, u;
    std::vector<float> h2min;
    std::vector<double> c64, vd, P;
};

static int grp_host_build(const double *tri, const float4 *g0_h, int np, GroupHost &H)
{
    const int K = OBEM_GRP_K, M = OBEM_GRP_M, NC = OBEM_GRP_CHECK;
    // group order: Morton code (10 bits per axis) of the centroids, stable
    std::vector<double> cen(3 * (size_t)np), area(np);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < np; ++i) {
        const double *v = tri + 9 * (size_t)i;
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            cen[3 * i + k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
            lo[k] = fmin(lo[k], cen[3 * i + k]);
            hi[k] = fmax(hi[k], cen[3 * i + k]);
            e1[k] = v[3 + k] - v[k];
            e2[k] = v[6 + k] - v[k];
        }
        const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                     nz = e1[0] * e2[1] - e1[1] * e2[0];
        area[i] = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
    }
    std::vector<uint32_t> code(np);
    for (int i = 0; i < np; ++i) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            const double ext = hi[k] - lo[k];
            double t = ext > 0.0 ? (cen[3 * i + k] - lo[k]) * (1024.0 / ext) : 0.0;
            int qi = (int)t;
            q[k] = (uint32_t)(qi < 0 ? 0 : (qi > 1023 ? 1023 : qi));
        }
        code[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    }
    std::vector<int32_t> perm(np);
    for (int i = 0; i < np; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
    // per group: area-weighted centre (rounded to binary32), radius over the
    // vertices (rounded up), smallest h^2
    const int ng = (np + K - 1) / K;
    std::vector<float4> cr(ng);
    std::vector<float> h2min(ng);
    std::vector<double> c64(4 * (size_t)ng);
    for (int g = 0; g < ng; ++g) {
        double s[3] = {0.0, 0.0, 0.0}, a = 0.0;
        float hm = 3e38f;
        const int e = std::min(np, (g + 1) * K);
        for (int t = g * K; t < e; ++t) {
            const int j = perm[t];
            for (int k = 0; k < 3; ++k) s[k] += area[j] * cen[3 * (size_t)j + k];
            a += area[j];
            hm = fminf(hm, g0_h[j].w);
        }
        const float cx = (float)(s[0] / a), cy = (float)(s[1] / a), cz = (float)(s[2] / a);
        double R = 0.0;
        for (int t = g * K; t < e; ++t) {
            const double *v = tri + 9 * (size_t)perm[t];
            for (int q = 0; q < 3; ++q) {
                const double dx = v[3 * q] - cx, dy = v[3 * q + 1] - cy, dz = v[3 * q + 2] - cz;
                R = fmax(R, sqrt(dx * dx + dy * dy + dz * dz));
            }
        }
        float Rf = (float)(R * (1.0 + 1e-6));
        if ((double)Rf < R) Rf = nextafterf(Rf, 3e38f);
        cr[g] = make_float4(cx, cy, cz, Rf);
        h2min[g] = hm;
        c64[4 * (size_t)g] = cx;
        c64[4 * (size_t)g + 1] = cy;
        c64[4 * (size_t)g + 2] = cz;
        c64[4 * (size_t)g + 3] = Rf;
    }
    // directions (the equivalent charges' as binary32, used as such by the fit)
    std::vector<double> ud, vd;
    sphere_points(M, ud);
    sphere_points(NC, vd);
    std::vector<float4> u(M);
    for (int k = 0; k < M; ++k) {
        u[k] = make_float4((float)ud[3 * k], (float)ud[3 * k + 1], (float)ud[3 * k + 2], 0.f);
        ud[3 * k] = u[k].x; ud[3 * k + 1] = u[k].y; ud[3 * k + 2] = u[k].z;
    }
    // fit for a unit radius: A[l][k] = 1 / |RC v_l - u_k|, pinv = (A^T A)^-1 A^T
    std::vector<double> A((size_t)NC * M), N((size_t)M * M, 0.0), P((size_t)M * NC);
    for (int l = 0; l < NC; ++l)
        for (int k = 0; k < M; ++k) {
            const double dx = OBEM_GRP_RC * vd[3 * l] - ud[3 * k], dy = OBEM_GRP_RC * vd[3 * l + 1] - ud[3 * k + 1],
                         dz = OBEM_GRP_RC * vd[3 * l + 2] - ud[3 * k + 2];
            A[(size_t)l * M + k] = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
        }
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            double s = 0.0;
            for (int l = 0; l < NC; ++l) s += A[(size_t)l * M + a] * A[(size_t)l * M + b];
            N[(size_t)a * M + b] = s;
        }
    // Cholesky N = L L^T (in place, lower triangle)
    for (int j = 0; j < M; ++j) {
        double d = N[(size_t)j * M + j];
        for (int k = 0; k < j; ++k) d -= N[(size_t)j * M + k] * N[(size_t)j * M + k];
        if (!(d > 0.0)) return OBEM_ERR_SINGULAR;
        d = sqrt(d);
        N[(size_t)j * M + j] = d;
        for (int i = j + 1; i < M; ++i) {
            double s = N[(size_t)i * M + j];
            for (int k = 0; k < j; ++k) s -= N[(size_t)i * M + k] * N[(size_t)j * M + k];
            N[(size_t)i * M + j] = s / d;
        }
    }
    // column l of pinv: solve L L^T x = A[l][:]
    std::vector<double> x(M);
    for (int l = 0; l < NC; ++l) {
        for (int i = 0; i < M; ++i) {
            double s = A[(size_t)l * M + i];
            for (int k = 0; k < i; ++k) s -= N[(size_t)i * M + k] * x[k];
            x[i] = s / N[(size_t)i * M + i];
        }
        for (int i = M - 1; i >= 0; --i) {
            double s = x[i];
            for (int k = i + 1; k < M; ++k) s -= N[(size_t)k * M + i] * x[k];
            x[i] = s / N[(size_t)i * M + i];
        }
        for (int k = 0; k < M; ++k) P[(size_t)k * NC + l] = x[k];
    }
    H.ng = ng;
    H.perm.swap(perm);
    H.cr.swap(cr);
    H.h2min.swap(h2min);
    H.c64.swap(c64);
    H.u.swap(u);
    H.vd.swap(vd);
    H.P.swap(P);
    return OBEM_OK;
}

int obem_cell_groups_build(obem_ctx *c, const double *tri, const float4 *g0_h, int np)
{
    obem_cell_groups_free(c);
    if (np <= 0) return OBEM_OK;
    GroupHost H;
    if (grp_host_build(tri, g0_h, np, H) != OBEM_OK)
        return obem_fail(c, OBEM_ERR_SINGULAR, "cell groups: fit matrix not positive definite");
    const int ng = H.ng, M = OBEM_GRP_M, NC = OBEM_GRP_CHECK;
    int rc = OBEM_OK;
#define GUP(dst, src, bytes)                                                                  \
    do {                                                                                      \
        if (rc == OBEM_OK && (cudaMalloc((void **)&(dst), (bytes)) != cudaSuccess ||          \
                              cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice) != cudaSuccess)) \
            rc = obem_fail(c, OBEM_ERR_CUDA, "cell groups: upload failed");                  \
    } while (0)
    GUP(c->d_grp_perm, H.perm.data(), sizeof(int32_t) * np);
    GUP(c->d_grp_cr, H.cr.data(), sizeof(float4) * ng);
    GUP(c->d_grp_h2min, H.h2min.data(), sizeof(float) * ng);
    GUP(c->d_grp_u, H.u.data(), sizeof(float4) * M);
    GUP(c->d_grp_c64, H.c64.data(), sizeof(double) * 4 * ng);
    GUP(c->d_grp_v, H.vd.data(), sizeof(double) * 3 * NC);
    GUP(c->d_grp_pinv, H.P.data(), sizeof(double) * M * NC);
#undef GUP
    if (rc == OBEM_OK && cudaMalloc((void **)&c->d_grp_q, sizeof(float) * (size_t)ng * M) != cudaSuccess)
        rc = obem_fail(c, OBEM_ERR_CUDA, "cell groups: allocation failed");
    if (rc != OBEM_OK) {
        obem_cell_groups_free(c);
        return rc;
    }
    c->ngrp = ng;
    return OBEM_OK;
}

// One block per group: the group's cells as 7-point sources (FP64 vertices,
// k_C A sigma w), their potential at the check points, the fitted charges.
#define GF_THREADS 128
__global__ void __launch_bounds__(GF_THREADS)
grp_fit_kernel(const double *__restrict__ v64, const float *__restrict__ sigma, const int32_t *__restrict__ perm,
               int np, const double *__restrict__ c64, const double *__restrict__ vdir,
               const double *__restrict__ pinv, float *__restrict__ q)
{
    __shared__ double sp[OBEM_GRP_K * 7][4];
    __shared__ double sb[OBEM_GRP_CHECK];
    const int g = blockIdx.x, tid = threadIdx.x;
    const double cx = c64[4 * (size_t)g], cy = c64[4 * (size_t)g + 1], cz = c64[4 * (size_t)g + 2],
                 R = c64[4 * (size_t)g + 3];
    for (int p = tid; p < OBEM_GRP_K * 7; p += GF_THREADS) {
        const int slot = g * OBEM_GRP_K + p / 7, r = p % 7;
        double x = 0.0, y = 0.0, z = 0.0, w = 0.0;
        if (slot < np) {
            const int j = perm[slot];
            const double *v = v64 + 9 * (size_t)j;
            const double mx = (v[0] + v[3] + v[6]) / 3.0, my = (v[1] + v[4] + v[7]) / 3.0,
                         mz = (v[2] + v[5] + v[8]) / 3.0;
            const double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
            const double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
            const double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
            const double A = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
            double t = 0.0, wr = G7_W0;
            int k = 0;
            if (r >= 1 && r <= 3) { t = G7_T1; wr = G7_W1; k = r - 1; }
            else if (r >= 4) { t = G7_T2; wr = G7_W2; k = r - 4; }
            x = mx + t * (v[3 * k] - mx) - cx;
            y = my + t * (v[3 * k + 1] - my) - cy;
            z = mz + t * (v[3 * k + 2] - mz) - cz;
            w = OBEM_KC * A * (double)sigma[j] * wr;
        }
        sp[p][0] = x; sp[p][1] = y; sp[p][2] = z; sp[p][3] = w;
    }
    __syncthreads();
    for (int l = tid; l < OBEM_GRP_CHECK; l += GF_THREADS) {
        const double px = OBEM_GRP_RC * R * vdir[3 * l], py = OBEM_GRP_RC * R * vdir[3 * l + 1],
                     pz = OBEM_GRP_RC * R * vdir[3 * l + 2];
        double b = 0.0;
        for (int p = 0; p < OBEM_GRP_K * 7; ++p) {
            const double dx = px - sp[p][0], dy = py - sp[p][1], dz = pz - sp[p][2];
            b += sp[p][3] * rsqrt(dx * dx + dy * dy + dz * dz);
        }
        sb[l] = b;
    }
    __syncthreads();
    for (int k = tid; k < OBEM_GRP_M; k += GF_THREADS) {
        double s = 0.0;
        for (int l = 0; l < OBEM_GRP_CHECK; ++l) s += pinv[(size_t)k * OBEM_GRP_CHECK + l] * sb[l];
        q[(size_t)g * OBEM_GRP_M + k] = (float)(R * s);
    }
}

// The groups for a launch with this sigma: refits unless the charges already
// belong to the context's own sigma at its current version.
int obem_cell_groups_fit(obem_ctx *c, const float *sigma, cudaStream_t s, CellGroups *G, int *launched)
{
    *launched = 0;
    if (c->ngrp <= 0 || !sigma) return obem_fail(c, OBEM_ERR_STATE, "cell groups: not built");
    const bool cached = sigma == c->d_sigma && c->grp_fit_sigma == sigma && c->grp_fit_ver == c->sigma_ver;
    if (!cached) {
        grp_fit_kernel<<<c->ngrp, GF_THREADS, 0, s>>>(c->d_v64, sigma, c->d_grp_perm, c->np, c->d_grp_c64,
                                                      c->d_grp_v, c->d_grp_pinv, c->d_grp_q);
        OBEM_LAUNCH(c);
        c->grp_fit_sigma = sigma == c->d_sigma ? sigma : NULL;
        c->grp_fit_ver = c->sigma_ver;
        *launched = 1;
    }
    G->ng = c->ngrp;
    G->perm = c->d_grp_perm;
    G->cr = c->d_grp_cr;
    G->h2min = c->d_grp_h2min;
    G->u = c->d_grp_u;
    G->q = c->d_grp_q;
    return OBEM_OK;
}
