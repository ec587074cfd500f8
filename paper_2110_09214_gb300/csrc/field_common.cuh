// Device helpers shared by the forward field kernels and the backward
// (adjoint) kernels: packed f32x2 arithmetic, compensated summation, the FP64
// closed form of a uniformly charged flat triangle, and the quadrature rules
// of the far-cell tiers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

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
static __device__ __noinline__ void tri_closed_form(const double *v, double rx, double ry, double rz, double &phi,
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

// The same closed form with the cell's geometry precomputed in FP64 (g: unit
// normal, twice the area, unit edge vectors and in-plane edge normals, the
// layout of OBEM_GEO64): per evaluation only the vertex offsets, their
// lengths, the edge logarithms and the solid angle remain.
static __device__ __noinline__ void tri_closed_form_g(const double *v, const double *g, double rx, double ry,
                                                      double rz, double &phi, double &Fx, double &Fy, double &Fz)
{
    const double nx = g[0], ny = g[1], nz = g[2], a2 = g[3];
    double ax[3], ay[3], az[3], R[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ax[i] = v[3 * i] - rx;
        ay[i] = v[3 * i + 1] - ry;
        az[i] = v[3 * i + 2] - rz;
        R[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
    const double h = -(ax[0] * nx + ay[0] * ny + az[0] * nz);
    double ps = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3;
        const double *e = g + 4 + 6 * i;
        const double dx = e[0], dy = e[1], dz = e[2], ux = e[3], uy = e[4], uz = e[5];
        const double lm = ax[i] * dx + ay[i] * dy + az[i] * dz;
        const double lp = ax[j] * dx + ay[j] * dy + az[j] * dz;
        const double p0 = ax[i] * ux + ay[i] * uy + az[i] * uz;
        double L;
        if (lm >= 0.0) L = log((R[j] + lp) / (R[i] + lm));
        else if (lp <= 0.0) L = log((R[i] - lm) / (R[j] - lp));
        else L = log((R[j] + lp) * (R[i] - lm) / (p0 * p0 + h * h));
        if (p0 != 0.0) ps += p0 * L;
        fx += ux * L; fy += uy * L; fz += uz * L;
    }
    const double D = R[0] * R[1] * R[2] + (ax[0] * ax[1] + ay[0] * ay[1] + az[0] * az[1]) * R[2]
                   + (ax[0] * ax[2] + ay[0] * ay[2] + az[0] * az[2]) * R[1]
                   + (ax[1] * ax[2] + ay[1] * ay[2] + az[1] * az[2]) * R[0];
    const double Om = (h == 0.0) ? 0.0 : 2.0 * atan2(a2 * h, D);
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

// sub-triangle s of the midpoint subdivision of (A, B, C): 0 the middle one,
// 1..3 the corner ones at A, B, C
__device__ __forceinline__ void subtri(int s, float3 &A, float3 &B, float3 &C)
{
    const float3 ab = make_float3(0.5f * (A.x + B.x), 0.5f * (A.y + B.y), 0.5f * (A.z + B.z));
    const float3 bc = make_float3(0.5f * (B.x + C.x), 0.5f * (B.y + C.y), 0.5f * (B.z + C.z));
    const float3 ca = make_float3(0.5f * (C.x + A.x), 0.5f * (C.y + A.y), 0.5f * (C.z + A.z));
    if (s == 0) { A = ab; B = bc; C = ca; }
    else if (s == 1) { B = ab; C = ca; }
    else if (s == 2) { A = B; B = bc; C = ab; }
    else { A = C; B = ca; C = bc; }
}

// Point k of the 7-point rule applied to the 4^level sub-triangles of the
// cell with vertex offsets g0, g1, g2 (from its centroid): offset and weight
// fraction of the point.
__device__ __forceinline__ void rule_point(int level, int k, float3 g0, float3 g1, float3 g2, float3 &off,
                                           float &wf)
{
    int sub = k / 7;
    const int m = k % 7;
    float3 A = g0, B = g1, C = g2;
    float scale = 1.0f;
    for (int l = level - 1; l >= 0; --l) {
        int s = (sub >> (2 * l)) & 3;
        subtri(s, A, B, C);
        scale *= 0.25f;
    }
    const float3 sc = make_float3((A.x + B.x + C.x) * (1.0f / 3.0f), (A.y + B.y + C.y) * (1.0f / 3.0f),
                                  (A.z + B.z + C.z) * (1.0f / 3.0f));
    if (m == 0) { off = sc; wf = scale * D7_W0; return; }
    const int v = (m - 1) % 3;
    const float t = m <= 3 ? D7_T1 : D7_T2;
    const float3 V = v == 0 ? A : (v == 1 ? B : C);
    off = make_float3(fmaf(t, V.x - sc.x, sc.x), fmaf(t, V.y - sc.y, sc.y), fmaf(t, V.z - sc.z, sc.z));
    wf = scale * (m <= 3 ? D7_W1 : D7_W2);
}

// Far-cell tiers by the squared distance of the cell's centroid to a box of
// points in units of h^2 (h: longest edge).  Worst-case relative error of one
// cell's field (points in every direction, in-plane toward the vertices
// included): centroid 3.6e-6 at 200 h; 3-point (degree 2) 3.0e-6 at 16 h;
// 4-point (degree 3) 2.0e-6 at 10 h; 6-point (degree 4) 1.4e-6 at 4 h;
// 7-point (degree 5) 1.7e-6 at 3 h; 28-point 2.6e-6 at 1.5 h.
#define TIER_1PT_H2 40000.0f
#define TIER_3PT_H2 256.0f
#define TIER_4PT_H2 100.0f
#define TIER_6PT_H2 16.0f
#define TIER_7PT_H2 9.0f

// point k of the n-point far tier (n = 1, 3, 4, 6, 7, 28): offset from the
// centroid (the rules' points (a, b, b) are c + (a - b) g_k, as g_0 + g_1 +
// g_2 = 0) and weight fraction
__device__ __forceinline__ void far_point(int n, int k, float3 G0, float3 G1, float3 G2, float3 &off, float &wf)
{
    if (n == 1) { off = make_float3(0.f, 0.f, 0.f); wf = 1.0f; }
    else if (n == 3) {
        // degree 2: barycentric (2/3, 1/6, 1/6), weights 1/3
        const float3 g = k == 0 ? G0 : (k == 1 ? G1 : G2);
        off = make_float3(0.5f * g.x, 0.5f * g.y, 0.5f * g.z);
        wf = 1.0f / 3.0f;
    } else if (n == 4) {
        // degree 3: centroid (weight -27/48), (0.6, 0.2, 0.2) (weights 25/48)
        if (k == 0) { off = make_float3(0.f, 0.f, 0.f); wf = -27.0f / 48.0f; }
        else {
            const float3 g = k == 1 ? G0 : (k == 2 ? G1 : G2);
            off = make_float3(0.4f * g.x, 0.4f * g.y, 0.4f * g.z);
            wf = 25.0f / 48.0f;
        }
    } else if (n == 6) {
        // degree 4 (Dunavant): (a, b, b) with a - b = -0.3378454727478950, weight
        // 0.223381589678011, and a - b = 0.7252713594706880, weight 0.109951743655322
        const float3 g = (k % 3) == 0 ? G0 : ((k % 3) == 1 ? G1 : G2);
        const float sgk = k < 3 ? -0.33784547274789500f : 0.72527135947068800f;
        off = make_float3(sgk * g.x, sgk * g.y, sgk * g.z);
        wf = k < 3 ? 0.223381589678011f : 0.109951743655322f;
    } else {
        rule_point(n == 7 ? 0 : 1, k, G0, G1, G2, off, wf);
    }
}
