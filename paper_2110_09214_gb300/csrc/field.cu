// Field at points: BEM cell field (Eq. (BEM3), (BEM2)) + all-pairs Coulomb
// field of point charges (Eq. (nbody)), and -- in the tracking step -- the
// nearest-cation search that feeds electron-ion recombination (Sec. 3.3.3).
//
// Layout: each thread owns FT_TPT targets (two packs of two, processed with
// the packed f32x2 instructions of sm_100+), a block owns FT_THREADS*FT_TPT
// consecutive targets.  Sources are staged through shared memory in tiles of
// FT_SRC_TILE charges stored as duplicated pairs (x,x)(y,y)(z,z)(kq,kq), so a
// packed instruction serves two targets against one source.  Every tile's
// FP32 partial sum is folded into a compensated (TwoSum) accumulator.
//
// Cell field tiers, chosen per (target, cell) from the distance d to the
// centroid and the longest edge h:
//   d >= 200 h   centroid rule            (<= 3.4e-6 relative per cell)
//   d >=  16 h   3-point degree-2 rule    (<= 2.7e-6)
//   d >=   3 h   7-point degree-5 rule    (<= 1.4e-6)
//   d <    3 h   closed form in FP64 (edge logarithms + solid angle)
#include "obem_internal.cuh"

#define FT_THREADS 128
#define FT_TPT 4
#define FT_BLOCK_TARGETS (FT_THREADS * FT_TPT)
#define FT_SRC_TILE 256
#define FT_PAN_TILE 64

#define TIER_1PT_H2 40000.0f
#define TIER_3PT_H2 256.0f
#define TIER_7PT_H2 9.0f

typedef unsigned long long u64;

// ------------------------------------------------------------------ packed f32x2
__device__ __forceinline__ u64 pk(float a, float b)
{
    u64 r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float &a, float &b)
{
    asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float rsq(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// error-free sum s + e = a + b (Knuth TwoSum), e accumulated into c
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float b)
{
    float t = __fadd_rn(s, b);
    float z = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(b, z));
    s = t;
    c = __fadd_rn(c, e);
}

// ------------------------------------------------------------------ FP64 closed form
// Potential and field of a unit uniform density on a flat triangle at r:
// phi = sum_i p0_i L_i - h Omega,  F = Omega n + sum_i u_i L_i, with the edge
// integrals L_i = ln((R+ + l+)/(R- + l-)) evaluated without cancellation and
// Omega the signed solid angle (Van Oosterom & Strackee); principal value in
// the cell's plane.
__device__ __noinline__ void tri_closed_form(const double *v, double rx, double ry, double rz, double &phi,
                                double &Fx, double &Fy, double &Fz)
{
    double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    double a2 = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= a2; ny /= a2; nz /= a2;
    double ax[3], ay[3], az[3], R[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ax[i] = v[3 * i] - rx;
        ay[i] = v[3 * i + 1] - ry;
        az[i] = v[3 * i + 2] - rz;
        R[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
    double h = -(ax[0] * nx + ay[0] * ny + az[0] * nz);
    double ps = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double dx = v[3 * j] - v[3 * i], dy = v[3 * j + 1] - v[3 * i + 1], dz = v[3 * j + 2] - v[3 * i + 2];
        double len = sqrt(dx * dx + dy * dy + dz * dz);
        dx /= len; dy /= len; dz /= len;
        double ux = dy * nz - dz * ny, uy = dz * nx - dx * nz, uz = dx * ny - dy * nx;
        double lm = ax[i] * dx + ay[i] * dy + az[i] * dz;
        double lp = ax[j] * dx + ay[j] * dy + az[j] * dz;
        double p0 = ax[i] * ux + ay[i] * uy + az[i] * uz;
        double L;
        if (lm >= 0.0) L = log((R[j] + lp) / (R[i] + lm));
        else if (lp <= 0.0) L = log((R[i] - lm) / (R[j] - lp));
        else L = log((R[j] + lp) * (R[i] - lm) / (p0 * p0 + h * h));
        if (p0 != 0.0) ps += p0 * L;
        fx += ux * L; fy += uy * L; fz += uz * L;
    }
    double D = R[0] * R[1] * R[2] + (ax[0] * ax[1] + ay[0] * ay[1] + az[0] * az[1]) * R[2]
             + (ax[0] * ax[2] + ay[0] * ay[2] + az[0] * az[2]) * R[1]
             + (ax[1] * ax[2] + ay[1] * ay[2] + az[1] * az[2]) * R[0];
    double Om = (h == 0.0) ? 0.0 : 2.0 * atan2(a2 * h, D);
    phi = ps - h * Om;
    Fx = fx + Om * nx;
    Fy = fy + Om * ny;
    Fz = fz + Om * nz;
}

// one FP32 quadrature point of weight w (already k_C sigma A w_i)
__device__ __forceinline__ void qpoint(float tx, float ty, float tz, float px, float py, float pz,
                                       float w, float &ax, float &ay, float &az, float &av)
{
    float dx = tx - px, dy = ty - py, dz = tz - pz;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float inv = rsq(r2);
    float s = w * inv;
    float s3 = s * (inv * inv);
    ax = fmaf(dx, s3, ax);
    ay = fmaf(dy, s3, ay);
    az = fmaf(dz, s3, az);
    av += s;
}

// Dunavant degree-5 rule, points c + t (v_k - c)
#define D7_W0 0.225f
#define D7_W1 0.132394152788506f
#define D7_W2 0.125939180544827f
#define D7_T1 (-0.410426192315345f)
#define D7_T2 0.696140478029631f

struct __align__(16) PanTile {
    float4 cq;   // cx, cy, cz, q = k_C sigma A
    float4 g0;   // v0 - c, h^2
    float4 g1;   // v1 - c, index (bits)
    float4 g2;   // v2 - c, sigma
};

struct __align__(16) SrcPk {
    u64 xx, yy, zz, qq;
};

// ---------------------------------------------------------------- target binning
// Targets are visited by the cell kernel in the Morton order of a 64^3 grid
// over the cell bounding box (points outside are clamped to the border
// bins), so the 32 targets of a warp are neighbours and mostly take the same
// distance tier for a given cell.  Counting sort: histogram, scan, scatter;
// the order inside a bin is arbitrary, which does not change any result (each
// target's sum runs over the cells in the same order whatever its slot).
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3Fu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void bin_count_kernel(FieldLaunch L, float3 lo, float3 scale, uint32_t *code, int32_t *hist)
{
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    float4 p = L.targets[i];
    int ix = (int)fminf(fmaxf((p.x - lo.x) * scale.x, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    int iy = (int)fminf(fmaxf((p.y - lo.y) * scale.y, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    int iz = (int)fminf(fmaxf((p.z - lo.z) * scale.z, 0.f), (float)(OBEM_BINS_PER_AXIS - 1));
    uint32_t c = spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
    code[i] = c;
    atomicAdd(&hist[c], 1);
}

// exclusive scan of OBEM_NBINS counts in place, one block of 1024 threads
__global__ void bin_scan_kernel(int32_t *hist)
{
    __shared__ int32_t part[1024];
    const int per = OBEM_NBINS / 1024;
    int32_t *h = hist + threadIdx.x * per;
    int32_t s = 0;
    for (int k = 0; k < per; ++k) s += h[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int k = 0; k < per; ++k) {
        int32_t c = h[k];
        h[k] = run;
        run += c;
    }
}

__global__ void bin_scatter_kernel(FieldLaunch L, const uint32_t *code, int32_t *hist, int32_t *perm)
{
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int pos = atomicAdd(&hist[code[i]], 1);
    perm[pos] = i;
}

// ---------------------------------------------------------------- cell field kernel
#define CT_THREADS 128
#define CT_TPT 2
#define CT_BLOCK (CT_THREADS * CT_TPT)

#define TIER_28PT_H2 4.0f     // 2h <= d < 3h: 7-point rule on the 4 midpoint sub-triangles

// 7-point rule over the triangle with centroid (cx,cy,cz) and vertex offsets g*
__device__ __forceinline__ void rule7(float tx, float ty, float tz, float cx, float cy, float cz,
                                      float g0x, float g0y, float g0z, float g1x, float g1y, float g1z,
                                      float g2x, float g2y, float g2z, float q, float *P)
{
    const float w1 = q * D7_W1, w2 = q * D7_W2;
    qpoint(tx, ty, tz, cx, cy, cz, q * D7_W0, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T1, g0x, cx), fmaf(D7_T1, g0y, cy), fmaf(D7_T1, g0z, cz), w1, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T1, g1x, cx), fmaf(D7_T1, g1y, cy), fmaf(D7_T1, g1z, cz), w1, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T1, g2x, cx), fmaf(D7_T1, g2y, cy), fmaf(D7_T1, g2z, cz), w1, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T2, g0x, cx), fmaf(D7_T2, g0y, cy), fmaf(D7_T2, g0z, cz), w2, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T2, g1x, cx), fmaf(D7_T2, g1y, cy), fmaf(D7_T2, g1z, cz), w2, P[0], P[1], P[2], P[3]);
    qpoint(tx, ty, tz, fmaf(D7_T2, g2x, cx), fmaf(D7_T2, g2y, cy), fmaf(D7_T2, g2z, cz), w2, P[0], P[1], P[2], P[3]);
}

// 7-point rule on each of the 4 midpoint sub-triangles (offsets from c)
__device__ __noinline__ void rule28(float tx, float ty, float tz, float4 cq, float4 g0, float4 g1, float4 g2,
                                    float *P)
{
    const float q = 0.25f * cq.w;
    const float m01x = 0.5f * (g0.x + g1.x), m01y = 0.5f * (g0.y + g1.y), m01z = 0.5f * (g0.z + g1.z);
    const float m12x = 0.5f * (g1.x + g2.x), m12y = 0.5f * (g1.y + g2.y), m12z = 0.5f * (g1.z + g2.z);
    const float m20x = 0.5f * (g2.x + g0.x), m20y = 0.5f * (g2.y + g0.y), m20z = 0.5f * (g2.z + g0.z);
    // middle sub-triangle: centroid c, offsets m01, m12, m20
    rule7(tx, ty, tz, cq.x, cq.y, cq.z, m01x, m01y, m01z, m12x, m12y, m12z, m20x, m20y, m20z, q, P);
    // corner sub-triangles (v_k, m_k,k+1, m_k,k-1)
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        float ax = k == 0 ? g0.x : (k == 1 ? g1.x : g2.x), ay = k == 0 ? g0.y : (k == 1 ? g1.y : g2.y),
              az = k == 0 ? g0.z : (k == 1 ? g1.z : g2.z);
        float bx = k == 0 ? m01x : (k == 1 ? m12x : m20x), by = k == 0 ? m01y : (k == 1 ? m12y : m20y),
              bz = k == 0 ? m01z : (k == 1 ? m12z : m20z);
        float ex = k == 0 ? m20x : (k == 1 ? m01x : m12x), ey = k == 0 ? m20y : (k == 1 ? m01y : m12y),
              ez = k == 0 ? m20z : (k == 1 ? m01z : m12z);
        float sx = (ax + bx + ex) * (1.0f / 3.0f), sy = (ay + by + ey) * (1.0f / 3.0f), sz = (az + bz + ez) * (1.0f / 3.0f);
        rule7(tx, ty, tz, cq.x + sx, cq.y + sy, cq.z + sz, ax - sx, ay - sy, az - sz, bx - sx, by - sy, bz - sz,
              ex - sx, ey - sy, ez - sz, q, P);
    }
}

// FP64 closed form of one cell, added to the FP32 partial
__device__ __noinline__ void closed_into(const double *v, float tx, float ty, float tz, float sg, float *P)
{
    double phi, Fx, Fy, Fz;
    tri_closed_form(v, (double)tx, (double)ty, (double)tz, phi, Fx, Fy, Fz);
    const double kq = OBEM_KC * (double)sg;
    P[0] += (float)(kq * Fx);
    P[1] += (float)(kq * Fy);
    P[2] += (float)(kq * Fz);
    P[3] += (float)(kq * phi);
}

// E_out[i] = e_ext + k_C sum_j sigma_j F_j(r_i)  (w: potential if WANT_V)
template <bool WANT_V, bool COUNT>
__global__ void __launch_bounds__(CT_THREADS)
cell_kernel(FieldLaunch L)
{
    __shared__ PanTile s_pan[FT_PAN_TILE];
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    const int base = blockIdx.x * CT_BLOCK;
    if (base >= nt) return;
    const int tid = threadIdx.x;
    float tx[CT_TPT], ty[CT_TPT], tz[CT_TPT];
    float S[CT_TPT][4], C[CT_TPT][4];
    int ti[CT_TPT];
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        int i = base + k * CT_THREADS + tid;
        int ic = i < nt ? i : (nt - 1);
        ti[k] = L.perm ? L.perm[ic] : ic;
        float4 p = L.targets[ti[k]];
        tx[k] = p.x; ty[k] = p.y; tz[k] = p.z;
        if (i >= nt) ti[k] = -1;
#pragma unroll
        for (int c = 0; c < 4; ++c) { S[k][c] = 0.f; C[k][c] = 0.f; }
    }
    unsigned long long cnt1 = 0, cnt3 = 0, cnt7 = 0, cntA = 0;
    const int np = L.panels.np;
    for (int pb = 0; pb < np; pb += FT_PAN_TILE) {
        __syncthreads();
        if (tid < FT_PAN_TILE) {
            int j = pb + tid;
            PanTile t;
            if (j < np) {
                float4 ca = L.panels.c_a[j];
                float sg = L.sigma[j];
                t.cq = make_float4(ca.x, ca.y, ca.z, ca.w * sg);
                t.g0 = L.panels.g0_h[j];
                float4 g1 = L.panels.g1[j];
                float4 g2 = L.panels.g2[j];
                t.g1 = make_float4(g1.x, g1.y, g1.z, __int_as_float(j));
                t.g2 = make_float4(g2.x, g2.y, g2.z, sg);
            } else {
                t.cq = make_float4(1e18f, 1e18f, 1e18f, 0.f);
                t.g0 = make_float4(0.f, 0.f, 0.f, 0.f);
                t.g1 = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                t.g2 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            s_pan[tid] = t;
        }
        __syncthreads();
        const int cntp = min(FT_PAN_TILE, np - pb);
        float P[CT_TPT][4];
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k) { P[k][0] = P[k][1] = P[k][2] = P[k][3] = 0.f; }
        for (int jj = 0; jj < cntp; ++jj) {
            const float4 cq = s_pan[jj].cq;
            const float4 g0 = s_pan[jj].g0;
            const float h2 = g0.w;
#pragma unroll
            for (int k = 0; k < CT_TPT; ++k) {
                float dx = tx[k] - cq.x, dy = ty[k] - cq.y, dz = tz[k] - cq.z;
                float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (d2 >= TIER_1PT_H2 * h2) {
                    float inv = rsq(d2);
                    float s = cq.w * inv;
                    float s3 = s * (inv * inv);
                    P[k][0] = fmaf(dx, s3, P[k][0]);
                    P[k][1] = fmaf(dy, s3, P[k][1]);
                    P[k][2] = fmaf(dz, s3, P[k][2]);
                    if (WANT_V) P[k][3] += s;
                    if (COUNT) ++cnt1;
                } else if (d2 >= TIER_3PT_H2 * h2) {
                    const float4 g1 = s_pan[jj].g1, g2 = s_pan[jj].g2;
                    float w = cq.w * (1.0f / 3.0f);
                    qpoint(tx[k], ty[k], tz[k], fmaf(0.5f, g0.x, cq.x), fmaf(0.5f, g0.y, cq.y), fmaf(0.5f, g0.z, cq.z), w, P[k][0], P[k][1], P[k][2], P[k][3]);
                    qpoint(tx[k], ty[k], tz[k], fmaf(0.5f, g1.x, cq.x), fmaf(0.5f, g1.y, cq.y), fmaf(0.5f, g1.z, cq.z), w, P[k][0], P[k][1], P[k][2], P[k][3]);
                    qpoint(tx[k], ty[k], tz[k], fmaf(0.5f, g2.x, cq.x), fmaf(0.5f, g2.y, cq.y), fmaf(0.5f, g2.z, cq.z), w, P[k][0], P[k][1], P[k][2], P[k][3]);
                    if (COUNT) ++cnt3;
                } else if (d2 >= TIER_7PT_H2 * h2) {
                    const float4 g1 = s_pan[jj].g1, g2 = s_pan[jj].g2;
                    rule7(tx[k], ty[k], tz[k], cq.x, cq.y, cq.z, g0.x, g0.y, g0.z, g1.x, g1.y, g1.z, g2.x, g2.y,
                          g2.z, cq.w, P[k]);
                    if (COUNT) ++cnt7;
                } else if (d2 >= TIER_28PT_H2 * h2) {
                    rule28(tx[k], ty[k], tz[k], cq, g0, s_pan[jj].g1, s_pan[jj].g2, P[k]);
                    if (COUNT) ++cnt7;
                } else {
                    const int j = __float_as_int(s_pan[jj].g1.w);
                    closed_into(L.panels.v64 + 9 * (size_t)j, tx[k], ty[k], tz[k], s_pan[jj].g2.w, P[k]);
                    if (COUNT) ++cntA;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CT_TPT; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) two_sum_acc(S[k][c], C[k][c], P[k][c]);
            if (WANT_V) two_sum_acc(S[k][3], C[k][3], P[k][3]);
        }
    }
#pragma unroll
    for (int k = 0; k < CT_TPT; ++k) {
        if (ti[k] < 0) continue;
        float4 e;
        e.x = (float)((double)S[k][0] + (double)C[k][0] + (double)L.e_ext.x);
        e.y = (float)((double)S[k][1] + (double)C[k][1] + (double)L.e_ext.y);
        e.z = (float)((double)S[k][2] + (double)C[k][2] + (double)L.e_ext.z);
        e.w = WANT_V ? (float)((double)S[k][3] + (double)C[k][3]) : 0.f;
        L.E_out[ti[k]] = e;
    }
    if (COUNT && L.counters) {
        atomicAdd(&L.counters[1], cnt1);
        atomicAdd(&L.counters[2], cnt3);
        atomicAdd(&L.counters[3], cnt7);
        atomicAdd(&L.counters[4], cntA);
    }
}

// ---------------------------------------------------------------- all-pairs kernel
// E_out[i] = init + k_C sum_{p != i} q_p (r_i - r_p) / (|r_i - r_p|^2 + eps^2)^(3/2)
// init = E_out[i] when the cell kernel ran first (ADD), else e_ext.
template <bool WANT_V, bool RECOMB, bool ADD>
__global__ void __launch_bounds__(FT_THREADS)
nbody_kernel(FieldLaunch L)
{
    __shared__ SrcPk s_src[FT_SRC_TILE];

    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    const int ns = L.ns_dev ? *L.ns_dev : L.ns;
    const int base = blockIdx.x * FT_BLOCK_TARGETS;
    if (base >= nt) return;
    const int tid = threadIdx.x;

    float tx[FT_TPT], ty[FT_TPT], tz[FT_TPT];
    float S[FT_TPT][4], C[FT_TPT][4];
    float rc2f[FT_TPT];
    u64 best[FT_TPT];
#pragma unroll
    for (int k = 0; k < FT_TPT; ++k) {
        int i = base + k * FT_THREADS + tid;
        int ic = i < nt ? i : (nt - 1);
        float4 p = L.targets[ic];
        tx[k] = p.x; ty[k] = p.y; tz[k] = p.z;
        if (ADD) {
            float4 e = L.E_out[ic];
            S[k][0] = e.x; S[k][1] = e.y; S[k][2] = e.z; S[k][3] = e.w;
        } else {
            S[k][0] = L.e_ext.x; S[k][1] = L.e_ext.y; S[k][2] = L.e_ext.z; S[k][3] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) C[k][c] = 0.f;
        best[k] = ~0ull;
        rc2f[k] = -1.0f;
        if (RECOMB && i < nt && L.species[i] == OBEM_ELECTRON)
            rc2f[k] = (L.rc2 + L.eps2) * (1.0f + 3.814697265625e-06f) + 1e-30f;
    }

    const float kC = (float)OBEM_KC;
    const u64 EPS2 = pk(L.eps2, L.eps2);
    u64 TX[2], TY[2], TZ[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        TX[p] = pk(tx[2 * p], tx[2 * p + 1]);
        TY[p] = pk(ty[2 * p], ty[2 * p + 1]);
        TZ[p] = pk(tz[2 * p], tz[2 * p + 1]);
    }
    for (int sb = 0; sb < ns; sb += FT_SRC_TILE) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < FT_SRC_TILE / FT_THREADS; ++r) {
            int l = r * FT_THREADS + tid;
            int j = sb + l;
            SrcPk sp;
            if (j < ns) {
                float4 s = L.sources[j];
                float kq = kC * s.w;
                sp.xx = pk(s.x, s.x); sp.yy = pk(s.y, s.y); sp.zz = pk(s.z, s.z); sp.qq = pk(kq, kq);
            } else {
                sp.xx = sp.yy = sp.zz = pk(1e18f, 1e18f);
                sp.qq = pk(0.f, 0.f);
            }
            s_src[l] = sp;
        }
        __syncthreads();
        const bool diag = L.self_exclude && sb < base + FT_BLOCK_TARGETS && base < sb + FT_SRC_TILE;
        if (!diag) {
            u64 AX[2], AY[2], AZ[2], AV[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) AX[p] = AY[p] = AZ[p] = AV[p] = 0ull;
#pragma unroll 4
            for (int jj = 0; jj < FT_SRC_TILE; ++jj) {
                const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&s_src[jj].xx);
                const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&s_src[jj].zz);
                bool hit = false;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    u64 dx = sub2(TX[p], a.x);
                    u64 dy = sub2(TY[p], a.y);
                    u64 dz = sub2(TZ[p], b.x);
                    u64 r2 = fma2(dx, dx, EPS2);
                    r2 = fma2(dy, dy, r2);
                    r2 = fma2(dz, dz, r2);
                    float ra, rb;
                    upk(r2, ra, rb);
                    if (RECOMB) hit |= (ra < rc2f[2 * p]) | (rb < rc2f[2 * p + 1]);
                    u64 inv = pk(rsq(ra), rsq(rb));
                    u64 s = mul2(b.y, inv);
                    u64 s3 = mul2(s, mul2(inv, inv));
                    AX[p] = fma2(dx, s3, AX[p]);
                    AY[p] = fma2(dy, s3, AY[p]);
                    AZ[p] = fma2(dz, s3, AZ[p]);
                    if (WANT_V) AV[p] = add2(AV[p], s);
                }
                if (RECOMB && hit) {
                    // rare: binary32 distance without contraction, and the partner rules
                    const int j = sb + jj;
                    float sx, sy, sz, dum;
                    upk(a.x, sx, dum); upk(a.y, sy, dum); upk(b.x, sz, dum);
                    if (j < ns && L.species[j] == OBEM_CATION && !(L.birth[j] != 0u && L.birth[j] == L.step)) {
#pragma unroll
                        for (int k = 0; k < FT_TPT; ++k) {
                            if (rc2f[k] < 0.f) continue;
                            float ddx = __fsub_rn(tx[k], sx), ddy = __fsub_rn(ty[k], sy), ddz = __fsub_rn(tz[k], sz);
                            float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)), __fmul_rn(ddz, ddz));
                            if (d2 <= L.rc2) {
                                u64 key = ((u64)__float_as_uint(d2) << 32) | (u64)(uint32_t)j;
                                if (key < best[k]) best[k] = key;
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float a0, a1;
                upk(AX[p], a0, a1); two_sum_acc(S[2 * p][0], C[2 * p][0], a0); two_sum_acc(S[2 * p + 1][0], C[2 * p + 1][0], a1);
                upk(AY[p], a0, a1); two_sum_acc(S[2 * p][1], C[2 * p][1], a0); two_sum_acc(S[2 * p + 1][1], C[2 * p + 1][1], a1);
                upk(AZ[p], a0, a1); two_sum_acc(S[2 * p][2], C[2 * p][2], a0); two_sum_acc(S[2 * p + 1][2], C[2 * p + 1][2], a1);
                if (WANT_V) { upk(AV[p], a0, a1); two_sum_acc(S[2 * p][3], C[2 * p][3], a0); two_sum_acc(S[2 * p + 1][3], C[2 * p + 1][3], a1); }
            }
        } else {
            // tile holding some of this block's own targets: skip the self pair
            float P[FT_TPT][4];
#pragma unroll
            for (int k = 0; k < FT_TPT; ++k) { P[k][0] = P[k][1] = P[k][2] = P[k][3] = 0.f; }
            for (int jj = 0; jj < FT_SRC_TILE; ++jj) {
                const int j = sb + jj;
                float sx, sy, sz, sq, dum;
                upk(s_src[jj].xx, sx, dum); upk(s_src[jj].yy, sy, dum);
                upk(s_src[jj].zz, sz, dum); upk(s_src[jj].qq, sq, dum);
#pragma unroll
                for (int k = 0; k < FT_TPT; ++k) {
                    if (j == base + k * FT_THREADS + tid) continue;
                    float dx = __fsub_rn(tx[k], sx), dy = __fsub_rn(ty[k], sy), dz = __fsub_rn(tz[k], sz);
                    float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, L.eps2)));
                    float inv = rsq(r2);
                    float s = sq * inv;
                    float s3 = s * (inv * inv);
                    P[k][0] = fmaf(dx, s3, P[k][0]);
                    P[k][1] = fmaf(dy, s3, P[k][1]);
                    P[k][2] = fmaf(dz, s3, P[k][2]);
                    P[k][3] += s;
                    if (RECOMB && r2 < rc2f[k] && j < ns && L.species[j] == OBEM_CATION &&
                        !(L.birth[j] != 0u && L.birth[j] == L.step)) {
                        float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                        if (d2 <= L.rc2) {
                            u64 key = ((u64)__float_as_uint(d2) << 32) | (u64)(uint32_t)j;
                            if (key < best[k]) best[k] = key;
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < FT_TPT; ++k)
#pragma unroll
                for (int c = 0; c < 4; ++c) two_sum_acc(S[k][c], C[k][c], P[k][c]);
        }
    }

#pragma unroll
    for (int k = 0; k < FT_TPT; ++k) {
        int i = base + k * FT_THREADS + tid;
        if (i >= nt) continue;
        float4 e;
        e.x = (float)((double)S[k][0] + (double)C[k][0]);
        e.y = (float)((double)S[k][1] + (double)C[k][1]);
        e.z = (float)((double)S[k][2] + (double)C[k][2]);
        e.w = WANT_V ? (float)((double)S[k][3] + (double)C[k][3]) : 0.f;
        L.E_out[i] = e;
        if (RECOMB) L.prop[i] = best[k];
    }
}

// counters[0] += nt * (ns - self pairs): the pairs of the all-pairs kernel
__global__ void pair_count_kernel(FieldLaunch L)
{
    if (threadIdx.x != 0) return;
    const long long nt = L.nt_dev ? *L.nt_dev : L.nt;
    const long long ns = L.ns_dev ? *L.ns_dev : L.ns;
    atomicAdd(&L.counters[0], (unsigned long long)(nt * ns - (L.self_exclude ? nt : 0)));
}

// E_out = e_ext when neither cells nor charges contribute
__global__ void const_field_kernel(FieldLaunch L)
{
    const int nt = L.nt_dev ? *L.nt_dev : L.nt;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) L.E_out[i] = make_float4(L.e_ext.x, L.e_ext.y, L.e_ext.z, 0.f);
}

int obem_launch_field(obem_ctx *ctx, const FieldLaunch &L, int capacity_targets, cudaStream_t s)
{
    if (capacity_targets <= 0) return OBEM_OK;
    dim3 grid((capacity_targets + FT_BLOCK_TARGETS - 1) / FT_BLOCK_TARGETS);
    const bool cells = L.sigma != NULL && L.panels.np > 0;
    const bool charges = L.sources != NULL;
    if (cells) {
        if (L.perm) {
            // spatial order of the targets for the cell kernel
            float3 lo = make_float3(ctx->bbox_lo[0], ctx->bbox_lo[1], ctx->bbox_lo[2]);
            float3 sc;
            sc.x = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[0] - ctx->bbox_lo[0], 1e-30f);
            sc.y = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[1] - ctx->bbox_lo[1], 1e-30f);
            sc.z = (float)OBEM_BINS_PER_AXIS / fmaxf(ctx->bbox_hi[2] - ctx->bbox_lo[2], 1e-30f);
            OBEM_CUDA(ctx, cudaMemsetAsync(ctx->s_hist, 0, sizeof(int32_t) * OBEM_NBINS, s));
            const int nb = (capacity_targets + 255) / 256;
            bin_count_kernel<<<nb, 256, 0, s>>>(L, lo, sc, ctx->s_code, ctx->s_hist);
            bin_scan_kernel<<<1, 1024, 0, s>>>(ctx->s_hist);
            bin_scatter_kernel<<<nb, 256, 0, s>>>(L, ctx->s_code, ctx->s_hist, (int32_t *)L.perm);
            OBEM_LAUNCH(ctx);
            if (L.events) ctx->launches += 3;
        }
        dim3 cgrid((capacity_targets + CT_BLOCK - 1) / CT_BLOCK);
        if (L.want_v) {
            if (L.counters) cell_kernel<true, true><<<cgrid, CT_THREADS, 0, s>>>(L);
            else cell_kernel<true, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        } else {
            if (L.counters) cell_kernel<false, true><<<cgrid, CT_THREADS, 0, s>>>(L);
            else cell_kernel<false, false><<<cgrid, CT_THREADS, 0, s>>>(L);
        }
        OBEM_LAUNCH(ctx);
        if (L.events) ctx->launches++;
    }
    if (L.events) cudaEventRecord(L.events[1], s);
    if (charges) {
        if (L.counters) {
            pair_count_kernel<<<1, 32, 0, s>>>(L);
            OBEM_LAUNCH(ctx);
            if (L.events) ctx->launches++;
        }
        const bool rec = L.prop != NULL;
        if (L.want_v) {
            if (cells) nbody_kernel<true, false, true><<<grid, FT_THREADS, 0, s>>>(L);
            else nbody_kernel<true, false, false><<<grid, FT_THREADS, 0, s>>>(L);
        } else if (rec) {
            if (cells) nbody_kernel<false, true, true><<<grid, FT_THREADS, 0, s>>>(L);
            else nbody_kernel<false, true, false><<<grid, FT_THREADS, 0, s>>>(L);
        } else {
            if (cells) nbody_kernel<false, false, true><<<grid, FT_THREADS, 0, s>>>(L);
            else nbody_kernel<false, false, false><<<grid, FT_THREADS, 0, s>>>(L);
        }
        OBEM_LAUNCH(ctx);
        if (L.events) ctx->launches++;
    }
    if (!cells && !charges) {
        const_field_kernel<<<(capacity_targets + 255) / 256, 256, 0, s>>>(L);
        OBEM_LAUNCH(ctx);
        if (L.events) ctx->launches++;
    }
    if (L.events) cudaEventRecord(L.events[2], s);
    return OBEM_OK;
}
