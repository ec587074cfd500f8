// Backward (vector-Jacobian product) of the field evaluation of Eqs. (BEM2),
// (BEM3) and (nbody): for an upstream gradient g_t = (gE_t, gV_t) on the field
// and potential at every target,
//   dL/dsigma_j = k_C sum_t gE_t . F_j(x_t) + gV_t phi_j(x_t)
//   dL/dx_t     = (dE_t/dx_t)^T gE_t - gV_t E_t            (grad V = -E)
//   dL/dy_p     = k_C q_p sum_t -T(d)^T gE_t + gV_t d / |d|^3
//   dL/dq_p     = k_C sum_t gE_t . d / |d|^3 + gV_t / |d|
// with d = x_t - y_p and T(d) = I/|d|^3 - 3 d d^T / |d|^5 (symmetric).  For a
// point of weight w at y, the target-side term is
//   w |d|^-3 gE - w |d|^-3 (3 (d.gE) |d|^-2 + gV) d
// and the source-side term is its negative; the charge / density term is
//   w ((d.gE) |d|^-3 + gV |d|^-1).
// Cells enter through the same point formulas at their quadrature points
// (tiers by centroid distance in units of the longest edge h) and through the
// FP64 closed form of F and of its Jacobian near the cell.
//
// Pair arithmetic is FP32 (rsqrt.approx); partial sums of at most BW_CHUNK
// pair terms (or of one target's quadrature points) are added into FP64
// accumulators, so cancelling terms of both signs lose no more than ~16 ulps
// of the largest term.  Pairs at zero distance, and the pair t == p when
// self_exclude is set, are skipped.
#include "obem_internal.cuh"
#include "field_common.cuh"

#define BW_THREADS 128
#define BW_TILE 128            // points staged per shared-memory tile
#define BW_CHUNK 16            // pair terms summed in FP32 before each FP64 add
#define BS_WARPS 8
#define BS_PANELS 32           // cells per block of the dL/dsigma kernel
#define BS_TILE 256            // targets staged per tile of the dL/dsigma kernel

// Jacobian tiers (squared centroid distance in units of h^2); each keeps the
// per-cell relative error of dF/dr below ~2e-6
#define BJ_1PT 160000.0f       // d >= 400 h
#define BJ_3PT 1024.0f         // d >= 32 h
#define BJ_7PT 16.0f           // d >= 4 h
#define BJ_28PT 4.0f           // d >= 2 h
#define BJ_112PT 2.25f         // d >= 1.5 h, closed form below
// field / potential tiers of the forward evaluation (for dL/dsigma)
#define BF_1PT 40000.0f        // d >= 200 h
#define BF_3PT 256.0f          // d >= 16 h
#define BF_7PT 9.0f            // d >= 3 h
#define BF_28PT 2.25f          // d >= 1.5 h
#define BF_112PT 1.0f          // d >= h, closed form below

struct BwLaunch {
    const float4 *targets;
    int nt;
    const float4 *sources;     // (x, y, z, q) or NULL
    int ns;
    int self_exclude;
    const float *sigma;        // NULL: no cell part in dL/dx
    PanelsDev panels;
    const float4 *g;           // (gEx, gEy, gEz, gV) per target
    float *dsigma;
    float4 *dtargets;
    float4 *dsources;
};

// target-side term of one point of weight w at offset d = x - y
__device__ __forceinline__ void tgt_term(float dx, float dy, float dz, float w, float4 g, float &ax, float &ay,
                                         float &az)
{
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (!(r2 > 0.f)) return;
    const float inv = rsq(r2);
    const float inv2 = inv * inv;
    const float c1 = w * inv * inv2;
    const float dg = fmaf(dz, g.z, fmaf(dy, g.y, dx * g.x));
    const float c2 = c1 * fmaf(3.0f * dg, inv2, g.w);
    ax = fmaf(c1, g.x, fmaf(-c2, dx, ax));
    ay = fmaf(c1, g.y, fmaf(-c2, dy, ay));
    az = fmaf(c1, g.z, fmaf(-c2, dz, az));
}

// density-side term (w = k_C A w_k for a unit density): w (d.gE / |d|^3 + gV / |d|)
__device__ __forceinline__ float dens_term(float dx, float dy, float dz, float w, float4 g)
{
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (!(r2 > 0.f)) return 0.f;
    const float inv = rsq(r2);
    const float dg = fmaf(dz, g.z, fmaf(dy, g.y, dx * g.x));
    return w * inv * fmaf(dg, inv * inv, g.w);
}

// dF/dr (row-major) and F of a unit uniform density on a flat triangle, FP64.
// F = Omega n + sum_i u_i L_i (edge decomposition); the edge terms'
// gradients are written without cancellation in the three cases of the
// foot of r relative to the edge, and the solid angle's gradient is the
// Biot-Savart integral of a unit current around the triangle,
// (lhat x w) (l+/R+ - l-/R-) / R0^2 per edge (w = the perpendicular from r's
// line foot to the edge's line, R0 = |w|), rewritten without R0^2 when l-
// and l+ have the same sign.
__device__ __noinline__ void tri_closed_jac(const double *v, double rx, double ry, double rz, double *J,
                                            double *F)
{
    const double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    const double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const double a2 = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= a2; ny /= a2; nz /= a2;
    double ax[3], ay[3], az[3], R[3];
    for (int i = 0; i < 3; ++i) {
        ax[i] = v[3 * i] - rx;
        ay[i] = v[3 * i + 1] - ry;
        az[i] = v[3 * i + 2] - rz;
        R[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
    const double h = -(ax[0] * nx + ay[0] * ny + az[0] * nz);
    double go[3] = {0.0, 0.0, 0.0}, fin[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 9; ++k) J[k] = 0.0;
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        double tx = v[3 * j] - v[3 * i], ty = v[3 * j + 1] - v[3 * i + 1], tz = v[3 * j + 2] - v[3 * i + 2];
        const double len = sqrt(tx * tx + ty * ty + tz * tz);
        tx /= len; ty /= len; tz /= len;
        const double ux = ty * nz - tz * ny, uy = tz * nx - tx * nz, uz = tx * ny - ty * nx;
        const double lm = ax[i] * tx + ay[i] * ty + az[i] * tz;
        const double lp = ax[j] * tx + ay[j] * ty + az[j] * tz;
        const double wx = ax[i] - lm * tx, wy = ay[i] - lm * ty, wz = az[i] - lm * tz;
        const double p0 = ax[i] * ux + ay[i] * uy + az[i] * uz;
        const double r0sq = p0 * p0 + h * h;
        double L, cw;
        if (lm >= 0.0) {
            L = log((R[j] + lp) / (R[i] + lm));
            cw = 1.0 / (R[i] * (R[i] + lm)) - 1.0 / (R[j] * (R[j] + lp));
        } else if (lp <= 0.0) {
            L = log((R[i] - lm) / (R[j] - lp));
            cw = 1.0 / (R[j] * (R[j] - lp)) - 1.0 / (R[i] * (R[i] - lm));
        } else {
            L = log((R[j] + lp) * (R[i] - lm) / r0sq);
            cw = (R[i] - lm) / (R[i] * r0sq) - 1.0 / (R[j] * (R[j] + lp));
        }
        const double cl = 1.0 / R[i] - 1.0 / R[j];
        const double gx = cl * tx + cw * wx, gy = cl * ty + cw * wy, gz = cl * tz + cw * wz;
        J[0] += ux * gx; J[1] += ux * gy; J[2] += ux * gz;
        J[3] += uy * gx; J[4] += uy * gy; J[5] += uy * gz;
        J[6] += uz * gx; J[7] += uz * gy; J[8] += uz * gz;
        fin[0] += ux * L; fin[1] += uy * L; fin[2] += uz * L;
        const double c = lm * lp > 0.0 ? (lp * lp - lm * lm) / ((lp * R[i] + lm * R[j]) * R[i] * R[j])
                                       : (lp / R[j] - lm / R[i]) / r0sq;
        go[0] += c * (ty * wz - tz * wy);
        go[1] += c * (tz * wx - tx * wz);
        go[2] += c * (tx * wy - ty * wx);
    }
    const double D = R[0] * R[1] * R[2] + (ax[0] * ax[1] + ay[0] * ay[1] + az[0] * az[1]) * R[2] +
                     (ax[0] * ax[2] + ay[0] * ay[2] + az[0] * az[2]) * R[1] +
                     (ax[1] * ax[2] + ay[1] * ay[2] + az[1] * az[2]) * R[0];
    const double om = (h == 0.0) ? 0.0 : 2.0 * atan2(a2 * h, D);
    const double n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) J[3 * a + b] += n[a] * go[b];
    F[0] = fin[0] + om * nx;
    F[1] = fin[1] + om * ny;
    F[2] = fin[2] + om * nz;
}

// number of quadrature points of a tier (0: closed form) for squared
// centroid distance d2 and squared longest edge h2
__device__ __forceinline__ int jac_tier(float d2, float h2)
{
    return d2 >= BJ_1PT * h2 ? 1 : d2 >= BJ_3PT * h2 ? 3 : d2 >= BJ_7PT * h2 ? 7 : d2 >= BJ_28PT * h2 ? 28
         : d2 >= BJ_112PT * h2 ? 112 : 0;
}
__device__ __forceinline__ int fld_tier(float d2, float h2)
{
    return d2 >= BF_1PT * h2 ? 1 : d2 >= BF_3PT * h2 ? 3 : d2 >= BF_7PT * h2 ? 7 : d2 >= BF_28PT * h2 ? 28
         : d2 >= BF_112PT * h2 ? 112 : 0;
}

// point k of an n-point tier: offset from the centroid and weight fraction
__device__ __forceinline__ void tier_point(int n, int k, float3 g0, float3 g1, float3 g2, float3 &off, float &wf)
{
    if (n == 1) { off = make_float3(0.f, 0.f, 0.f); wf = 1.0f; return; }
    if (n == 3) {
        const float3 g = k == 0 ? g0 : (k == 1 ? g1 : g2);
        off = make_float3(0.5f * g.x, 0.5f * g.y, 0.5f * g.z);
        wf = 1.0f / 3.0f;
        return;
    }
    rule_point(n == 7 ? 0 : (n == 28 ? 1 : 2), k, g0, g1, g2, off, wf);
}

// ---------------------------------------------------------------- dL/dx
// One warp per target: the lanes take every 32nd charge and every 32nd cell
// (a target's sums are split across 32 lanes, so a few thousand probe points
// fill the GPU), each lane summing in FP64 partial sums of at most BW_CHUNK
// FP32 charge terms or one cell's quadrature points; the lanes' sums are
// added by a fixed butterfly of shuffles (deterministic).
__global__ void __launch_bounds__(BW_THREADS) bw_targets_kernel(BwLaunch B)
{
    const int t = (blockIdx.x * BW_THREADS + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= B.nt) return;                              // warp-uniform
    const float4 x = B.targets[t];
    const float4 g = B.g[t];
    double acc[3] = {0.0, 0.0, 0.0};
    const float kC = (float)OBEM_KC;
    // point charges
    for (int p0 = 0; p0 < B.ns; p0 += 32 * BW_CHUNK) {
        float ax = 0.f, ay = 0.f, az = 0.f;
        const int p1 = min(B.ns, p0 + 32 * BW_CHUNK);
        for (int p = p0 + lane; p < p1; p += 32) {
            if (B.self_exclude && p == t) continue;
            const float4 s = B.sources[p];
            tgt_term(x.x - s.x, x.y - s.y, x.z - s.z, kC * s.w, g, ax, ay, az);
        }
        acc[0] += ax; acc[1] += ay; acc[2] += az;
    }
    // cells
    if (B.sigma) {
        const PanelsDev &P = B.panels;
        for (int j = lane; j < P.np; j += 32) {
            const float4 ca = P.c_a[j], cl = P.c_lo[j], g0 = P.g0_h[j];
            // exact target - centroid: x - c_hi is exact for nearby targets
            const float ex = (x.x - ca.x) - cl.x, ey = (x.y - ca.y) - cl.y, ez = (x.z - ca.z) - cl.z;
            const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
            const int n = jac_tier(d2, g0.w);
            const float sg = B.sigma[j];
            if (n > 0) {
                const float4 g1 = P.g1[j], g2 = P.g2[j];
                const float3 G0 = make_float3(g0.x, g0.y, g0.z), G1 = make_float3(g1.x, g1.y, g1.z),
                             G2 = make_float3(g2.x, g2.y, g2.z);
                const float wq = ca.w * sg;
                float ax = 0.f, ay = 0.f, az = 0.f;
                for (int k = 0; k < n; ++k) {
                    float3 off;
                    float wf;
                    tier_point(n, k, G0, G1, G2, off, wf);
                    tgt_term(ex - off.x, ey - off.y, ez - off.z, wq * wf, g, ax, ay, az);
                }
                acc[0] += ax; acc[1] += ay; acc[2] += az;
            } else {
                double J[9], F[3];
                tri_closed_jac(P.v64 + 9 * (size_t)j, (double)x.x, (double)x.y, (double)x.z, J, F);
                const double s = OBEM_KC * (double)sg;
                for (int b = 0; b < 3; ++b)
                    acc[b] += s * (J[b] * g.x + J[3 + b] * g.y + J[6 + b] * g.z - (double)g.w * F[b]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0) B.dtargets[t] = make_float4((float)acc[0], (float)acc[1], (float)acc[2], 0.f);
}

// ---------------------------------------------------------------- dL/dy, dL/dq
__global__ void __launch_bounds__(BW_THREADS) bw_sources_kernel(BwLaunch B)
{
    __shared__ float4 s_x[BW_TILE], s_g[BW_TILE];
    const int p = blockIdx.x * BW_THREADS + threadIdx.x;
    const bool live = p < B.ns;
    const float4 y = live ? B.sources[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int tb = 0; tb < B.nt; tb += BW_TILE) {
        __syncthreads();
        for (int l = threadIdx.x; l < BW_TILE; l += BW_THREADS) {
            const int t = tb + l;
            s_x[l] = t < B.nt ? B.targets[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            s_g[l] = t < B.nt ? B.g[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int n = min(BW_TILE, B.nt - tb);
        for (int l0 = 0; l0 < n; l0 += BW_CHUNK) {
            float ax = 0.f, ay = 0.f, az = 0.f, aq = 0.f;
            for (int l = l0; l < min(n, l0 + BW_CHUNK); ++l) {
                if (B.self_exclude && tb + l == p) continue;
                const float4 x = s_x[l], g = s_g[l];
                const float dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
                tgt_term(dx, dy, dz, 1.0f, g, ax, ay, az);
                aq += dens_term(dx, dy, dz, 1.0f, g);
            }
            acc[0] += ax; acc[1] += ay; acc[2] += az; acc[3] += aq;
        }
    }
    if (live) {
        const double kq = OBEM_KC * (double)y.w;
        B.dsources[p] = make_float4((float)(-kq * acc[0]), (float)(-kq * acc[1]), (float)(-kq * acc[2]),
                                    (float)(OBEM_KC * acc[3]));
    }
}

// ---------------------------------------------------------------- dL/dsigma
// Block: BS_PANELS cells, warp w takes cells w, w + 8, ...; lanes stride over
// a tile of BS_TILE targets staged in shared memory.
__global__ void __launch_bounds__(BS_WARPS * 32) bw_sigma_kernel(BwLaunch B)
{
    __shared__ float4 s_x[BS_TILE], s_g[BS_TILE];
    constexpr int PER_WARP = BS_PANELS / BS_WARPS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const PanelsDev &P = B.panels;
    double acc[PER_WARP];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) acc[i] = 0.0;
    for (int tb = 0; tb < B.nt; tb += BS_TILE) {
        __syncthreads();
        for (int l = threadIdx.x; l < BS_TILE; l += BS_WARPS * 32) {
            const int t = tb + l;
            s_x[l] = t < B.nt ? B.targets[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            s_g[l] = t < B.nt ? B.g[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int n = min(BS_TILE, B.nt - tb);
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            const int j = blockIdx.x * BS_PANELS + warp + BS_WARPS * i;
            if (j >= P.np) continue;
            const float4 ca = P.c_a[j], cl = P.c_lo[j], g0 = P.g0_h[j], g1 = P.g1[j], g2 = P.g2[j];
            const float3 G0 = make_float3(g0.x, g0.y, g0.z), G1 = make_float3(g1.x, g1.y, g1.z),
                         G2 = make_float3(g2.x, g2.y, g2.z);
            double ad = 0.0;
            for (int l = lane; l < n; l += 32) {
                float a = 0.f;
                const float4 x = s_x[l], g = s_g[l];
                const float ex = (x.x - ca.x) - cl.x, ey = (x.y - ca.y) - cl.y, ez = (x.z - ca.z) - cl.z;
                const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                const int nq = fld_tier(d2, g0.w);
                if (nq > 0) {
                    for (int k = 0; k < nq; ++k) {
                        float3 off;
                        float wf;
                        tier_point(nq, k, G0, G1, G2, off, wf);
                        a += dens_term(ex - off.x, ey - off.y, ez - off.z, ca.w * wf, g);
                    }
                } else {
                    double phi, fx, fy, fz;
                    tri_closed_form(P.v64 + 9 * (size_t)j, (double)x.x, (double)x.y, (double)x.z, phi, fx, fy, fz);
                    ad += OBEM_KC * ((double)g.x * fx + (double)g.y * fy + (double)g.z * fz + (double)g.w * phi);
                }
                ad += (double)a;   // one target's quadrature points in FP32, targets summed in FP64
            }
            acc[i] += ad;
        }
    }
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int j = blockIdx.x * BS_PANELS + warp + BS_WARPS * i;
        if (lane == 0 && j < P.np) B.dsigma[j] = (float)v;
    }
}

// ---------------------------------------------------------------- influence of the charges on the cells
// S_j = k_C sum_p q_p (phi_j(y_p), F_j(y_p)) for every cell j (Eqs. (potpart),
// (fldpart) before the division by the cell area): the transpose cell
// operator of dL/dsigma with the forward's tiers, four sums per cell.  Block:
// BS_PANELS cells, warp w takes cells w, w + 8, ...; lanes stride over a tile
// of BS_TILE charges in shared memory; one charge's quadrature points are
// summed in FP32, charges in FP64; the FP64 closed form below one cell size.
__global__ void __launch_bounds__(BS_WARPS * 32) infl_kernel(const float4 *src, int ns, PanelsDev P, double *S)
{
    __shared__ float4 s_x[BS_TILE];
    constexpr int PER_WARP = BS_PANELS / BS_WARPS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[PER_WARP][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;
    for (int tb = 0; tb < ns; tb += BS_TILE) {
        __syncthreads();
        for (int l = threadIdx.x; l < BS_TILE; l += BS_WARPS * 32) {
            const int t = tb + l;
            s_x[l] = t < ns ? src[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int n = min(BS_TILE, ns - tb);
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            const int j = blockIdx.x * BS_PANELS + warp + BS_WARPS * i;
            if (j >= P.np) continue;
            const float4 ca = P.c_a[j], cl = P.c_lo[j], g0 = P.g0_h[j], g1 = P.g1[j], g2 = P.g2[j];
            const float3 G0 = make_float3(g0.x, g0.y, g0.z), G1 = make_float3(g1.x, g1.y, g1.z),
                         G2 = make_float3(g2.x, g2.y, g2.z);
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            for (int l = lane; l < n; l += 32) {
                const float4 x = s_x[l];
                const float ex = (x.x - ca.x) - cl.x, ey = (x.y - ca.y) - cl.y, ez = (x.z - ca.z) - cl.z;
                const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                const int nq = fld_tier(d2, g0.w);
                if (nq > 0) {
                    float vp = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
                    for (int k = 0; k < nq; ++k) {
                        float3 off;
                        float wf;
                        tier_point(nq, k, G0, G1, G2, off, wf);
                        const float dx = ex - off.x, dy = ey - off.y, dz = ez - off.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        if (!(r2 > 0.f)) continue;
                        const float inv = rsq(r2);
                        const float w = ca.w * wf * inv;
                        const float w3 = w * inv * inv;
                        vp += w;
                        vx = fmaf(w3, dx, vx); vy = fmaf(w3, dy, vy); vz = fmaf(w3, dz, vz);
                    }
                    a0 += (double)x.w * vp; a1 += (double)x.w * vx; a2 += (double)x.w * vy; a3 += (double)x.w * vz;
                } else {
                    double phi, fx, fy, fz;
                    tri_closed_form(P.v64 + 9 * (size_t)j, (double)x.x, (double)x.y, (double)x.z, phi, fx, fy, fz);
                    const double qk = (double)x.w * OBEM_KC;
                    a0 += qk * phi; a1 += qk * fx; a2 += qk * fy; a3 += qk * fz;
                }
            }
            acc[i][0] += a0; acc[i][1] += a1; acc[i][2] += a2; acc[i][3] += a3;
        }
    }
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        const int j = blockIdx.x * BS_PANELS + warp + BS_WARPS * i;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = acc[i][c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && j < P.np) S[4 * (size_t)j + c] = v;
        }
    }
}

// Right-hand-side correction of Eqs. (BEMpotpart), (BEMfldpart) from S:
// electrode cells -Vbar_j = -S_phi / A_j; dielectric cells
// -(eps+ - eps-) eps0 Ebar_j . n_j with Ebar_j = -S_F / A_j.
__global__ void infl_rhs_kernel(const double *S, const double *geo, const int *kind, const double *epsd, int np,
                                float *drhs)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double *g = geo + (size_t)OBEM_GEO64 * j;
    const double area = 0.5 * g[3];
    const double *s = S + 4 * (size_t)j;
    double v;
    if (kind[j] == OBEM_CELL_ELECTRODE) v = -s[0] / area;
    else v = epsd[j] * OBEM_EPS0 * (s[1] * g[0] + s[2] * g[1] + s[3] * g[2]) / area;
    drhs[j] = (float)v;
}

int obem_launch_influence(obem_ctx *ctx, const float4 *src, int ns, const PanelsDev &P, double *S, const double *geo,
                          const int *kind, const double *epsd, float *drhs, cudaStream_t s)
{
    if (P.np <= 0) return OBEM_OK;
    if (ns > 0) {
        infl_kernel<<<(P.np + BS_PANELS - 1) / BS_PANELS, BS_WARPS * 32, 0, s>>>(src, ns, P, S);
        OBEM_LAUNCH(ctx);
    } else {
        OBEM_CUDA(ctx, cudaMemsetAsync(S, 0, sizeof(double) * 4 * (size_t)P.np, s));
    }
    infl_rhs_kernel<<<(P.np + 255) / 256, 256, 0, s>>>(S, geo, kind, epsd, P.np, drhs);
    OBEM_LAUNCH(ctx);
    return OBEM_OK;
}

int obem_launch_backward(obem_ctx *ctx, const BwArgs &A, cudaStream_t s)
{
    BwLaunch B;
    memset(&B, 0, sizeof B);
    B.targets = (const float4 *)A.targets;
    B.nt = A.nt;
    B.sources = (const float4 *)A.sources;
    B.ns = A.sources ? A.ns : 0;
    B.self_exclude = A.self_exclude;
    B.sigma = A.sigma;
    B.panels = A.panels;
    B.g = (const float4 *)A.dL_dE;
    B.dsigma = A.dL_dsigma;
    B.dtargets = (float4 *)A.dL_dtargets;
    B.dsources = (float4 *)A.dL_dsources;
    if (B.dtargets && B.nt > 0) {
        bw_targets_kernel<<<(unsigned)(((long long)B.nt * 32 + BW_THREADS - 1) / BW_THREADS), BW_THREADS, 0, s>>>(B);
        OBEM_LAUNCH(ctx);
    }
    if (B.dsources && B.ns > 0) {
        bw_sources_kernel<<<(B.ns + BW_THREADS - 1) / BW_THREADS, BW_THREADS, 0, s>>>(B);
        OBEM_LAUNCH(ctx);
    }
    if (B.dsigma && B.panels.np > 0) {
        bw_sigma_kernel<<<(B.panels.np + BS_PANELS - 1) / BS_PANELS, BS_WARPS * 32, 0, s>>>(B);
        OBEM_LAUNCH(ctx);
    }
    return OBEM_OK;
}
