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
// operator of dL/dsigma with the forward's tiers, four sums per cell.
//
// The charges are put in spatial order (Morton bins of the cell box, blocks
// of at most 512 inside a super-bin); every block gets its bounding box and
// a copy of its charges relative to the box centre, stored by pairs in the
// f32x2 layout and padded with empty slots to a multiple of IF_FLUSH.  The
// cells are put in the same Morton order, so that a warp's 32 cells are
// neighbours.
//   infl_far_kernel   a thread block takes IF_CT cells, one per thread, and
//                     runs over the charge blocks, each copied into shared
//                     memory by TMA two blocks ahead.  For a block at least
//                     3 h from a cell's centroid the cell gets the forward's
//                     far tier (1, 3, 4, 6 or 7 points by that distance); the
//                     points of all the cells form one list, taken one or two
//                     points per thread per round against all the block's
//                     charges (broadcast reads, two charges per f32x2
//                     instruction), and a cell then adds up its points.  The
//                     blocks are cut into IF_NCH chunks (grid y), each with
//                     its own sums.
//   infl_near_kernel  one warp per cell over its blocks closer than 3 h, one
//                     charge per lane with the per-pair tier (points of every
//                     tier precomputed in shared memory); pairs within h go to
//                     a per-warp queue of the FP64 closed form, evaluated 32
//                     at a time.
// The far pass sums IF_FLUSH charges of a point in FP32 and adds these to a
// compensated (two-sum) FP32 accumulator, and a cell adds its points' sums to
// another; the near pass sums one block per lane in FP32, reduces the lanes
// by a fixed butterfly and adds the block sums in FP64.  The chunk sums and
// the near sum are added in a fixed order: the result does not depend on the
// schedule.
#define IF_NCH 8                // block chunks of the far pass
#define IF_FLUSH 64             // charges per FP32 partial sum of the far pass
#define IF_FAR_H2 TIER_7PT_H2   // far pass: blocks at least 3 h away
#define IF_Q 64                 // closed-form queue per warp (< 32 left after a flush, + 32 appended)
#define IF_NPT 151              // points of the tiers 1, 3, 7, 28, 112
#define IN_WARPS 4

// first pair of block b in the pair layout: never overlaps block b - 1's
// padded pairs (ceil(n / IF_FLUSH) * IF_FLUSH / 2 <= n / 2 + 31.5)
__device__ __forceinline__ int if_pair0(int2 bl, int b) { return (bl.x + 1) / 2 + 33 * b; }
int obem_influence_pairs(int ns, int maxblocks) { return (ns + 1) / 2 + 33 * maxblocks + 32; }

// the sorted copy of the charges (absolute: xs) and, relative to the block's
// box centre o, in pairs: xr[2 m] = (x0, x1, y0, y1), xr[2 m + 1] = (z0, z1,
// q0, q1), padding slots at o with no charge; every block's box: box[3 b] =
// lo, box[3 b + 1] = hi, box[3 b + 2] = o
__global__ void __launch_bounds__(256) infl_blocks_kernel(const float4 *src, const int32_t *perm, const int2 *blocks,
                                                          const int32_t *nblocks, float4 *xs, float4 *xr, float4 *box)
{
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= *nblocks) return;
    const int2 bl = blocks[b];
    float mn[3] = {3e38f, 3e38f, 3e38f}, mx[3] = {-3e38f, -3e38f, -3e38f};
    for (int l = lane; l < bl.y; l += 32) {
        const float4 p = src[perm[bl.x + l]];
        xs[bl.x + l] = p;
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    const float ox = 0.5f * (mn[0] + mx[0]), oy = 0.5f * (mn[1] + mx[1]), oz = 0.5f * (mn[2] + mx[2]);
    __syncwarp();
    const int npair = (bl.y + IF_FLUSH - 1) / IF_FLUSH * (IF_FLUSH / 2);
    const int p0 = if_pair0(bl, b);
    for (int m = lane; m < npair; m += 32) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * m < bl.y) a = xs[bl.x + 2 * m];
        if (2 * m + 1 < bl.y) c = xs[bl.x + 2 * m + 1];
        const bool ha = 2 * m < bl.y, hc = 2 * m + 1 < bl.y;
        xr[2 * (size_t)(p0 + m)] = make_float4(ha ? a.x - ox : 0.f, hc ? c.x - ox : 0.f, ha ? a.y - oy : 0.f,
                                               hc ? c.y - oy : 0.f);
        xr[2 * (size_t)(p0 + m) + 1] = make_float4(ha ? a.z - oz : 0.f, hc ? c.z - oz : 0.f, a.w, c.w);
    }
    if (lane == 0) {
        box[3 * b] = make_float4(mn[0], mn[1], mn[2], 0.f);
        box[3 * b + 1] = make_float4(mx[0], mx[1], mx[2], 0.f);
        box[3 * b + 2] = make_float4(ox, oy, oz, 0.f);
    }
}

__device__ __forceinline__ float if_box_d2(float4 c, float4 lo, float4 hi)
{
    const float dx = fmaxf(fmaxf(lo.x - c.x, c.x - hi.x), 0.f);
    const float dy = fmaxf(fmaxf(lo.y - c.y, c.y - hi.y), 0.f);
    const float dz = fmaxf(fmaxf(lo.z - c.z, c.z - hi.z), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

// ---- bulk copies of a block's charges into shared memory (TMA, 1D), with
// bounded waits: a wait that runs out (IF_WAIT_NS) records OBEM_ERR_TIMEOUT
#define IF_WAIT_NS 2000000000ull
__device__ __forceinline__ uint32_t if_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long if_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// (expect: bytes + extra; extra > 0 only in the self-test, where the phase
// then never completes)
__device__ __forceinline__ void if_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                             uint32_t extra)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(if_smem(bar)), "r"(bytes + extra)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(if_smem(dst)), "l"((unsigned long long)src), "r"(bytes), "r"(if_smem(bar))
                 : "memory");
}
// true once the phase of the given parity has completed, false after IF_WAIT_NS
__device__ __forceinline__ bool if_bar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = if_smem(bar);
    const unsigned long long t0 = if_now();
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((i & 255u) == 255u && if_now() - t0 > IF_WAIT_NS) return false;
    }
}

// One round of the far pass: KP points per thread (slots e0 + IF_CT k + tid
// of the point list) against every charge of the block (pairs in shared
// memory); the charges are read once for the KP points.
#define IF_CT 128               // threads (cells) per block of the far pass
#define IF_BPAIRS 256           // padded pairs of a block of 512
template <int KP>
__device__ __forceinline__ void if_round(const ulonglong2 *xs2, int ng, float4 *sp, int e0)
{
    const int tid = threadIdx.x;
    u64 cx[KP], cy[KP], cz[KP];
    float pw[KP], ps[KP][4], pc[KP][4];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const float4 pt = sp[e0 + IF_CT * k + tid];
        cx[k] = pk(pt.x, pt.x); cy[k] = pk(pt.y, pt.y); cz[k] = pk(pt.z, pt.z);
        pw[k] = pt.w;
#pragma unroll
        for (int i = 0; i < 4; ++i) ps[k][i] = pc[k][i] = 0.f;
    }
    for (int g = 0; g < ng; ++g) {
        const ulonglong2 *xg = xs2 + g * IF_FLUSH;
        u64 tp[KP], tx[KP], ty[KP], tz[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) tp[k] = tx[k] = ty[k] = tz[k] = 0ull;
#pragma unroll 4
        for (int m = 0; m < IF_FLUSH / 2; ++m) {
            const ulonglong2 A = xg[2 * m], B = xg[2 * m + 1];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const u64 dx = sub2(A.x, cx[k]), dy = sub2(A.y, cy[k]), dz = sub2(B.x, cz[k]);
                const u64 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                float r0, r1;
                upk(r2, r0, r1);
                const u64 inv = pk(rsq(r0), rsq(r1));
                const u64 w = mul2(B.y, inv);
                const u64 w3 = mul2(w, mul2(inv, inv));
                tp[k] = add2(tp[k], w);
                tx[k] = fma2(w3, dx, tx[k]); ty[k] = fma2(w3, dy, ty[k]); tz[k] = fma2(w3, dz, tz[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            float a0, a1;
            upk(tp[k], a0, a1); two_sum_acc(ps[k][0], pc[k][0], a0 + a1);
            upk(tx[k], a0, a1); two_sum_acc(ps[k][1], pc[k][1], a0 + a1);
            upk(ty[k], a0, a1); two_sum_acc(ps[k][2], pc[k][2], a0 + a1);
            upk(tz[k], a0, a1); two_sum_acc(ps[k][3], pc[k][3], a0 + a1);
        }
    }
    // each thread overwrites the slots it read: the point's weighted sums
#pragma unroll
    for (int k = 0; k < KP; ++k)
        sp[e0 + IF_CT * k + tid] = make_float4((ps[k][0] + pc[k][0]) * pw[k], (ps[k][1] + pc[k][1]) * pw[k],
                                               (ps[k][2] + pc[k][2]) * pw[k], (ps[k][3] + pc[k][3]) * pw[k]);
}

// padded pairs and bytes of block b in the pair layout
__device__ __forceinline__ uint32_t if_block_bytes(int2 bl)
{
    return (uint32_t)((bl.y + IF_FLUSH - 1) / IF_FLUSH * (IF_FLUSH / 2)) * 2u * (uint32_t)sizeof(float4);
}

// Block of IF_CT threads: cells t = IF_CT x + tid of the cell order (one per
// thread); charge blocks [b0, b1) of chunk blockIdx.y, each copied into one
// of two shared buffers (TMA) two blocks ahead.  For every charge block the
// cells' far points form one list (a block-wide scan of the point counts),
// processed in rounds of IF_CT or 2 IF_CT slots.  A far block is at least
// 3 h from the centroid and every point within 2 h / 3 of it, so no pair
// has zero distance (nor a padding slot: the box centre, no charge); padding
// points sit at 1e18 m with weight 0.
__global__ void __launch_bounds__(IF_CT) infl_far_kernel(const float4 *xr, const int2 *blocks, const int32_t *nblocks,
                                                        const float4 *box, const int32_t *corder, PanelsDev P,
                                                        double *Spart, int *err, uint32_t tx_extra)
{
    __shared__ __align__(128) float4 s_x[2][2 * IF_BPAIRS];
    __shared__ float4 s_p[IF_CT * 7];
    __shared__ int s_w[IF_CT / 32];
    __shared__ __align__(8) uint64_t s_bar[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = blockIdx.x * IF_CT + tid;
    const bool live = t < P.np;
    const int j = live ? corder[t] : 0;
    const float4 ca = P.c_a[j], cl = P.c_lo[j];
    const float h2 = P.g0_h[j].w;
    const int nb = *nblocks;
    const int b0 = (int)((long long)nb * blockIdx.y / gridDim.y);
    const int b1 = (int)((long long)nb * (blockIdx.y + 1) / gridDim.y);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(if_smem(&s_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(if_smem(&s_bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < 2 && b0 + q < b1; ++q) {
            const int2 bl = blocks[b0 + q];
            if_bulk_load(s_x[q], xr + 2 * (size_t)if_pair0(bl, b0 + q), if_block_bytes(bl), &s_bar[q], tx_extra);
        }
    }
    __syncthreads();
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b = b0; b < b1; ++b) {
        const int it = b - b0, buf = it & 1;
        const float d2 = if_box_d2(ca, box[3 * b], box[3 * b + 1]);
        int n = d2 >= TIER_1PT_H2 * h2 ? 1 : d2 >= TIER_3PT_H2 * h2 ? 3 : d2 >= TIER_4PT_H2 * h2 ? 4
              : d2 >= TIER_6PT_H2 * h2 ? 6 : d2 >= IF_FAR_H2 * h2 ? 7 : 0;
        if (!live) n = 0;
        int inc = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        int before = 0, npts = 0;
#pragma unroll
        for (int w = 0; w < IF_CT / 32; ++w) {
            const int v = s_w[w];
            before += w < warp ? v : 0;
            npts += v;
        }
        const int off = before + inc - n;
        if (n) {
            const float4 bo = box[3 * b + 2];
            const float4 g0 = P.g0_h[j], g1 = P.g1[j], g2 = P.g2[j];
            const float3 G0 = make_float3(g0.x, g0.y, g0.z), G1 = make_float3(g1.x, g1.y, g1.z),
                         G2 = make_float3(g2.x, g2.y, g2.z);
            const float bx = ca.x - bo.x, by = ca.y - bo.y, bz = ca.z - bo.z;
            for (int k = 0; k < n; ++k) {
                float3 o;
                float wf;
                far_point(n, k, G0, G1, G2, o, wf);
                s_p[off + k] = make_float4(bx + (cl.x + o.x), by + (cl.y + o.y), bz + (cl.z + o.z), ca.w * wf);
            }
        }
        const int pend = (npts + IF_CT - 1) / IF_CT * IF_CT;
        if (npts + tid < pend) s_p[npts + tid] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
        const bool ok = if_bar_wait(&s_bar[buf], (uint32_t)(it >> 1) & 1u);
        if (!__syncthreads_and(ok)) {
            // the copy of this block never completed: report, wait (bounded)
            // for the copy of the next one, and leave
            if (tid == 0) {
                atomicExch(err, OBEM_ERR_TIMEOUT);
                if (b + 1 < b1) if_bar_wait(&s_bar[buf ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
            }
            return;
        }
        if (npts > 0) {
            const int2 bl = blocks[b];
            const ulonglong2 *xs2 = (const ulonglong2 *)s_x[buf];
            const int ng = (bl.y + IF_FLUSH - 1) / IF_FLUSH;
            // a warp skips the parts of a round that hold padding only
            for (int e0 = 0; e0 < npts;) {
                const int wb = e0 + 32 * warp;
                if (npts - e0 > IF_CT) {
                    if (wb + IF_CT < npts) if_round<2>(xs2, ng, s_p, e0);
                    else if_round<1>(xs2, ng, s_p, e0);
                    e0 += 2 * IF_CT;
                } else {
                    if (wb < npts) if_round<1>(xs2, ng, s_p, e0);
                    e0 += IF_CT;
                }
            }
        }
        __syncthreads();
        if (n) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < n; ++k) {
                const float4 e = s_p[off + k];
                v[0] += e.x; v[1] += e.y; v[2] += e.z; v[3] += e.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) two_sum_acc(s[i], c[i], v[i]);
        }
        __syncthreads();
        if (tid == 0 && b + 2 < b1) {
            // every thread is done with this buffer: refill it two blocks ahead
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int2 bl = blocks[b + 2];
            if_bulk_load(s_x[buf], xr + 2 * (size_t)if_pair0(bl, b + 2), if_block_bytes(bl), &s_bar[buf], tx_extra);
        }
    }
    if (live) {
        double *o = Spart + ((size_t)blockIdx.y * P.np + j) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = (double)s[i] + (double)c[i];
    }
}

// butterfly over the warp: lanes 8 g .. 8 g + 7 end with the warp's sum of v[g]
__device__ __forceinline__ float if_reduce4(const float (&v)[4])
{
    const int lane = threadIdx.x & 31;
    const bool up = lane & 16;
    const float k0 = up ? v[2] : v[0], k1 = up ? v[3] : v[1];
    const float b0 = k0 + __shfl_xor_sync(0xffffffffu, up ? v[0] : v[2], 16);
    const float b1 = k1 + __shfl_xor_sync(0xffffffffu, up ? v[1] : v[3], 16);
    const bool u8 = lane & 8;
    float c = (u8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, u8 ? b0 : b1, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// the queued charges [0, n) of the closed-form queue, one per lane (FP64,
// result rounded to FP32 into the lane's sums)
__device__ __forceinline__ void if_closed(const PanelsDev &P, int j, const float4 *cq, int n, float (&v)[4])
{
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const float4 x = cq[lane];
        double phi, fx, fy, fz;
        tri_closed_form(P.v64 + 9 * (size_t)j, (double)x.x, (double)x.y, (double)x.z, phi, fx, fy, fz);
        const double qk = (double)x.w * OBEM_KC;
        v[0] += (float)(qk * phi); v[1] += (float)(qk * fx);
        v[2] += (float)(qk * fy); v[3] += (float)(qk * fz);
    }
    __syncwarp();
}

// first point of a tier in the near pass's point table
__device__ __forceinline__ int if_tier_base(int nq)
{
    return nq == 1 ? 0 : nq == 3 ? 1 : nq == 7 ? 4 : nq == 28 ? 11 : 39;
}

// the queued charges [0, n) of a quadrature queue (every one with the
// nq-point tier, points k0 .. k0 + nq - 1 of the table), one per lane
__device__ __forceinline__ void if_quad_flush(const float4 *cq, int n, float4 ca, const float4 *pt, int k0, int nq,
                                              float (&v)[4])
{
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const float4 x = cq[lane];
        const float ex = x.x - ca.x, ey = x.y - ca.y, ez = x.z - ca.z;
        float sp = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
        for (int k = 0; k < nq; ++k) {
            const float4 o = pt[k0 + k];
            const float dx = ex - o.x, dy = ey - o.y, dz = ez - o.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (!(r2 > 0.f)) continue;
            const float inv = rsq(r2);
            const float w = o.w * inv;
            const float w3 = w * inv * inv;
            sp += w;
            sx = fmaf(w3, dx, sx); sy = fmaf(w3, dy, sy); sz = fmaf(w3, dz, sz);
        }
        v[0] = fmaf(x.w, sp, v[0]); v[1] = fmaf(x.w, sx, v[1]);
        v[2] = fmaf(x.w, sy, v[2]); v[3] = fmaf(x.w, sz, v[3]);
    }
    __syncwarp();
}

// Warp per cell.  Per 32 charges of a near block, the pairs of the 1- to
// 7-point tiers are done in place; the 28-point, 112-point and closed-form
// pairs are appended to three per-warp queues, each evaluated 32 pairs at a
// time, so that the lanes of a warp run the same point loop.  Queue order
// is (charge slot, lane) and every lane adds its results in that order: the
// sums are deterministic.
__global__ void __launch_bounds__(IN_WARPS * 32) infl_near_kernel(const float4 *xs, const int2 *blocks,
                                                                  const int32_t *nblocks, const float4 *box,
                                                                  PanelsDev P, double *Snear)
{
    __shared__ float4 s_cq[IN_WARPS][3][IF_Q];
    __shared__ float4 s_pt[IN_WARPS][IF_NPT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * IN_WARPS + warp;
    if (j >= P.np) return;
    const float4 ca = P.c_a[j], cl = P.c_lo[j], g0 = P.g0_h[j], g1 = P.g1[j], g2 = P.g2[j];
    {
        const float3 G0 = make_float3(g0.x, g0.y, g0.z), G1 = make_float3(g1.x, g1.y, g1.z),
                     G2 = make_float3(g2.x, g2.y, g2.z);
        for (int e = lane; e < IF_NPT; e += 32) {
            const int nq = e < 1 ? 1 : e < 4 ? 3 : e < 11 ? 7 : e < 39 ? 28 : 112;
            float3 off;
            float wf;
            tier_point(nq, e - if_tier_base(nq), G0, G1, G2, off, wf);
            s_pt[warp][e] = make_float4(cl.x + off.x, cl.y + off.y, cl.z + off.z, ca.w * wf);
        }
        __syncwarp();
    }
    const float4 *pt = s_pt[warp];
    const int nb = *nblocks;
    double acc = 0.0;
    for (int bb0 = 0; bb0 < nb; bb0 += 32) {
        const int bb = bb0 + lane;
        const bool near = bb < nb && if_box_d2(ca, box[3 * bb], box[3 * bb + 1]) < IF_FAR_H2 * g0.w;
        unsigned bal = __ballot_sync(0xffffffffu, near);
        while (bal) {
            const int b = bb0 + __ffs(bal) - 1;
            bal &= bal - 1;
            const int2 bl = blocks[b];
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            int qn[3] = {0, 0, 0};
            for (int l0 = 0; l0 < bl.y; l0 += 32) {
                const int l = l0 + lane;
                const float4 x = l < bl.y ? xs[bl.x + l] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float ex = x.x - ca.x, ey = x.y - ca.y, ez = x.z - ca.z;
                const float fx = ex - cl.x, fy = ey - cl.y, fz = ez - cl.z;
                const int nq = l < bl.y ? fld_tier(fmaf(fz, fz, fmaf(fy, fy, fx * fx)), g0.w) : -1;
                if (nq > 0 && nq <= 7) {
                    float sp = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
                    const int k0 = if_tier_base(nq);
                    for (int k = 0; k < nq; ++k) {
                        const float4 o = pt[k0 + k];
                        const float dx = ex - o.x, dy = ey - o.y, dz = ez - o.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        const float inv = rsq(r2);
                        const float w = o.w * inv;
                        const float w3 = w * inv * inv;
                        sp += w;
                        sx = fmaf(w3, dx, sx); sy = fmaf(w3, dy, sy); sz = fmaf(w3, dz, sz);
                    }
                    v[0] = fmaf(x.w, sp, v[0]); v[1] = fmaf(x.w, sx, v[1]);
                    v[2] = fmaf(x.w, sy, v[2]); v[3] = fmaf(x.w, sz, v[3]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const unsigned cb = __ballot_sync(0xffffffffu, nq == (c == 0 ? 28 : c == 1 ? 112 : 0));
                    if (!cb) continue;
                    float4 *cq = s_cq[warp][c];
                    if ((cb >> lane) & 1u) cq[qn[c] + __popc(cb & ((1u << lane) - 1u))] = x;
                    qn[c] += __popc(cb);
                    __syncwarp();
                    if (qn[c] >= 32) {
                        if (c == 2) if_closed(P, j, cq, 32, v);
                        else if_quad_flush(cq, 32, ca, pt, c == 0 ? 11 : 39, c == 0 ? 28 : 112, v);
                        const float4 tq = lane < qn[c] - 32 ? cq[32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
                        __syncwarp();
                        if (lane < qn[c] - 32) cq[lane] = tq;
                        qn[c] -= 32;
                        __syncwarp();
                    }
                }
            }
            if (qn[0] > 0) if_quad_flush(s_cq[warp][0], qn[0], ca, pt, 11, 28, v);
            if (qn[1] > 0) if_quad_flush(s_cq[warp][1], qn[1], ca, pt, 39, 112, v);
            if (qn[2] > 0) if_closed(P, j, s_cq[warp][2], qn[2], v);
            acc += (double)if_reduce4(v);
        }
    }
    if ((lane & 7) == 0) Snear[4 * (size_t)j + (lane >> 3)] = acc;
}

// Right-hand-side correction of Eqs. (BEMpotpart), (BEMfldpart) from S
// (the far chunks' sums, then the near sum; S itself is kept): electrode
// cells -Vbar_j = -S_phi / A_j; dielectric cells -(eps+ - eps-) eps0
// Ebar_j . n_j with Ebar_j = -S_F / A_j.
__global__ void infl_rhs_kernel(const double *Spart, int nparts, const double *Snear, double *S, const double *geo,
                                const int *kind, const double *epsd, int np, float *drhs)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    double t[4];
    for (int i = 0; i < 4; ++i) {
        double v = 0.0;
        for (int c = 0; c < nparts; ++c) v += Spart[((size_t)c * np + j) * 4 + i];
        if (Snear) v += Snear[4 * (size_t)j + i];
        t[i] = v;
        S[4 * (size_t)j + i] = v;
    }
    const double *g = geo + (size_t)OBEM_GEO64 * j;
    const double area = 0.5 * g[3];
    double v;
    if (kind[j] == OBEM_CELL_ELECTRODE) v = -t[0] / area;
    else v = epsd[j] * OBEM_EPS0 * (t[1] * g[0] + t[2] * g[1] + t[3] * g[2]) / area;
    drhs[j] = (float)v;
}

static size_t if_align(size_t b) { return (b + 255) & ~(size_t)255; }
// scratch: point bins (charges, then the cells), the cell order, the sorted
// charges (absolute and relative), the block boxes, the chunk sums and the
// near sums
size_t obem_influence_scratch_bytes(int ns, int np)
{
    if (ns <= 0 || np <= 0) return 0;
    const size_t bins = obem_point_bins_bytes(ns > np ? ns : np);
    const int mb = obem_point_bins_maxblocks(ns);
    return bins + if_align(sizeof(int32_t) * (size_t)np) + if_align(sizeof(float4) * (size_t)ns) +
           if_align(sizeof(float4) * 2 * (size_t)obem_influence_pairs(ns, mb)) + if_align(sizeof(float4) * 3 * (size_t)mb) +
           if_align(sizeof(double) * 4 * (size_t)np * (IF_NCH + 1) + sizeof(int));
}

int obem_launch_influence(obem_ctx *ctx, const float4 *src, int ns, const PanelsDev &P, double *S, const double *geo,
                          const int *kind, const double *epsd, float *drhs, void *scratch, int selftest,
                          cudaStream_t s)
{
    if (P.np <= 0) return OBEM_OK;
    if (ns > 0) {
        char *p = (char *)scratch;
        char *bins = p;
        p += obem_point_bins_bytes(ns > P.np ? ns : P.np);
        int32_t *corder = (int32_t *)p;
        p += if_align(sizeof(int32_t) * (size_t)P.np);
        float4 *xs = (float4 *)p;
        p += if_align(sizeof(float4) * (size_t)ns);
        float4 *xr = (float4 *)p;
        p += if_align(sizeof(float4) * 2 * (size_t)obem_influence_pairs(ns, obem_point_bins_maxblocks(ns)));
        float4 *box = (float4 *)p;
        p += if_align(sizeof(float4) * 3 * (size_t)obem_point_bins_maxblocks(ns));
        double *Spart = (double *)p;
        double *Snear = Spart + 4 * (size_t)P.np * IF_NCH;
        int *err = (int *)(Snear + 4 * (size_t)P.np);
        int32_t *perm, *nblocks;
        int2 *blocks;
        // the cells in Morton order of their centroids
        int rc = obem_point_bins(ctx, P.c_a, P.np, bins, &perm, &blocks, &nblocks, s);
        if (rc != OBEM_OK) return rc;
        OBEM_CUDA(ctx, cudaMemcpyAsync(corder, perm, sizeof(int32_t) * (size_t)P.np, cudaMemcpyDeviceToDevice, s));
        // the charges in blocks
        rc = obem_point_bins(ctx, src, ns, bins, &perm, &blocks, &nblocks, s);
        if (rc != OBEM_OK) return rc;
        const int mb = obem_point_bins_maxblocks(ns);
        infl_blocks_kernel<<<(mb + 7) / 8, 256, 0, s>>>(src, perm, blocks, nblocks, xs, xr, box);
        OBEM_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
        infl_far_kernel<<<dim3((P.np + IF_CT - 1) / IF_CT, IF_NCH), IF_CT, 0, s>>>(xr, blocks, nblocks, box, corder,
                                                                                 P, Spart, err, selftest ? 16u : 0u);
        infl_near_kernel<<<(P.np + IN_WARPS - 1) / IN_WARPS, IN_WARPS * 32, 0, s>>>(xs, blocks, nblocks, box, P,
                                                                                   Snear);
        OBEM_LAUNCH(ctx);
        infl_rhs_kernel<<<(P.np + 255) / 256, 256, 0, s>>>(Spart, IF_NCH, Snear, S, geo, kind, epsd, P.np, drhs);
        OBEM_LAUNCH(ctx);
        int h = 0;
        OBEM_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        OBEM_CUDA(ctx, cudaStreamSynchronize(s));
        if (h != 0) return obem_fail(ctx, OBEM_ERR_TIMEOUT, "influence: a wait for a bulk copy timed out");
        return OBEM_OK;
    } else {
        OBEM_CUDA(ctx, cudaMemsetAsync(S, 0, sizeof(double) * 4 * (size_t)P.np, s));
        infl_rhs_kernel<<<(P.np + 255) / 256, 256, 0, s>>>(S, 1, NULL, S, geo, kind, epsd, P.np, drhs);
    }
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
