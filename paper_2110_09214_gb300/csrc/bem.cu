// BEM set-up: assembly of the dense system of Eq. (matrixBEM), its LU
// factorisation, and solves with iterative refinement.  Sec. 2.2 fills the
// matrix on the GPU and keeps an inverse so that new voltages or free charges
// only need a new right-hand side; here the factors are kept instead of the
// inverse (same reuse, half the flops, better conditioned).
//
//   assemble_kernel   one thread per matrix element (row-major, coalesced over
//                     j): Q_ij = k_C phi_j(r_i) for electrode rows, W_ij for
//                     dielectric rows; FP64 closed form for near cells,
//                     FP32 quadrature (7/3/1 points by distance) for far ones
//   equilibrate       scale every row by the power of two nearest below
//                     1 / max |A_ij| (exact; solution unchanged)
//   LU                partial pivoting; panels of LU_NB columns factored by
//                       panel_kernel   cooperative: one row chunk per CTA held
//                                      in shared memory, one bounded exchange
//                                      of pivot candidates per column
//                       laswp_*        the panel's row swaps on whole rows
//                                      (plan, gather to scratch, scatter)
//                     BF16 (OBEM_LU_BF16): recursive (rec_lu / rec_trsm), every
//                       trailing update and off-diagonal TRSM block a
//                       hand-written tcgen05 GEMM (lu_tc.cu: BF16 operands,
//                       FP32 accumulation into the FP32 factors)
//                     FP32 / TF32 / BF16x9: right-looking blocked, trsm_kernel
//                       for U12 = L11^-1 A12 and cuBLAS for A22 -= L21 U12
//   solve             y = L^-1 P b, x = U^-1 y (blocked, FP32 factors) inside
//                     iterative refinement with FP64 residuals r = b - A x
#include <math.h>
#include <vector>

#include "obem_internal.cuh"

#define LU_NB 64
#define TS_R 128               // rows of a block row of the one-launch triangular solves

// ------------------------------------------------------------------ closed form (FP64)
// Same expansion as the field kernels: unit-density potential phi and field F
// of a flat triangle at r; principal value in the cell's plane.
__device__ __noinline__ void bem_closed_form(const double *v, double rx, double ry, double rz,
                                             double &phi, double &Fx, double &Fy, double &Fz)
{
    double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    double a2 = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= a2; ny /= a2; nz /= a2;
    double ax[3], ay[3], az[3], R[3];
    for (int i = 0; i < 3; ++i) {
        ax[i] = v[3 * i] - rx; ay[i] = v[3 * i + 1] - ry; az[i] = v[3 * i + 2] - rz;
        R[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
    double h = -(ax[0] * nx + ay[0] * ny + az[0] * nz);
    double ps = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
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
    Fx = fx + Om * nx; Fy = fy + Om * ny; Fz = fz + Om * nz;
}

// unit-density quadrature point (weight w = A w_k)
__device__ __forceinline__ void bq(float tx, float ty, float tz, float px, float py, float pz, float w,
                                   float &phi, float &fx, float &fy, float &fz)
{
    float dx = tx - px, dy = ty - py, dz = tz - pz;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float inv = rsqrtf(r2);
    float s = w * inv;
    float s3 = s * inv * inv;
    phi += s;
    fx = fmaf(dx, s3, fx); fy = fmaf(dy, s3, fy); fz = fmaf(dz, s3, fz);
}

#define AS_CLOSED_H2 16.0f     // d < 4 h: FP64 closed form
#define AS_7PT_H2 1024.0f      // d < 32 h: 7 points
#define AS_3PT_H2 360000.0f    // d < 600 h: 3 points, else centroid

__global__ void assemble_kernel(PanelsDev P, const int *kind, const double *em, const double *ep,
                                float *A, int n)
{
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float4 ci = P.c_a[i];
    const float4 cj = P.c_a[j];
    const float4 g0 = P.g0_h[j];
    float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float Aj = cj.w * (float)(1.0 / OBEM_KC);   // area
    double phi, Fx, Fy, Fz;
    if (i == j || d2 < AS_CLOSED_H2 * g0.w) {
        const double *vi = P.v64 + 9 * (size_t)i;
        double rx = (vi[0] + vi[3] + vi[6]) / 3.0, ry = (vi[1] + vi[4] + vi[7]) / 3.0,
               rz = (vi[2] + vi[5] + vi[8]) / 3.0;
        bem_closed_form(P.v64 + 9 * (size_t)j, rx, ry, rz, phi, Fx, Fy, Fz);
        if (i == j) { Fx = Fy = Fz = 0.0; }
    } else {
        float ph = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        const float4 g1 = P.g1[j], g2 = P.g2[j];
        if (d2 < AS_7PT_H2 * g0.w) {
            const float T1 = -0.410426192315345f, T2 = 0.696140478029631f;
            const float w0 = Aj * 0.225f, w1 = Aj * 0.132394152788506f, w2 = Aj * 0.125939180544827f;
            bq(ci.x, ci.y, ci.z, cj.x, cj.y, cj.z, w0, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T1, g0.x, cj.x), fmaf(T1, g0.y, cj.y), fmaf(T1, g0.z, cj.z), w1, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T1, g1.x, cj.x), fmaf(T1, g1.y, cj.y), fmaf(T1, g1.z, cj.z), w1, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T1, g2.x, cj.x), fmaf(T1, g2.y, cj.y), fmaf(T1, g2.z, cj.z), w1, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T2, g0.x, cj.x), fmaf(T2, g0.y, cj.y), fmaf(T2, g0.z, cj.z), w2, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T2, g1.x, cj.x), fmaf(T2, g1.y, cj.y), fmaf(T2, g1.z, cj.z), w2, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(T2, g2.x, cj.x), fmaf(T2, g2.y, cj.y), fmaf(T2, g2.z, cj.z), w2, ph, fx, fy, fz);
        } else if (d2 < AS_3PT_H2 * g0.w) {
            const float w = Aj * (1.0f / 3.0f);
            bq(ci.x, ci.y, ci.z, fmaf(0.5f, g0.x, cj.x), fmaf(0.5f, g0.y, cj.y), fmaf(0.5f, g0.z, cj.z), w, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(0.5f, g1.x, cj.x), fmaf(0.5f, g1.y, cj.y), fmaf(0.5f, g1.z, cj.z), w, ph, fx, fy, fz);
            bq(ci.x, ci.y, ci.z, fmaf(0.5f, g2.x, cj.x), fmaf(0.5f, g2.y, cj.y), fmaf(0.5f, g2.z, cj.z), w, ph, fx, fy, fz);
        } else {
            bq(ci.x, ci.y, ci.z, cj.x, cj.y, cj.z, Aj, ph, fx, fy, fz);
        }
        phi = ph; Fx = fx; Fy = fy; Fz = fz;
    }
    double a;
    if (kind[i] == OBEM_CELL_ELECTRODE) {
        a = OBEM_KC * phi;
    } else if (i == j) {
        a = 0.5 * (ep[i] + em[i]);
    } else {
        const float4 ni = P.nrm[i];
        a = (ep[i] - em[i]) / (4.0 * OBEM_PI) * (Fx * ni.x + Fy * ni.y + Fz * ni.z);
    }
    A[(size_t)i * n + j] = (float)a;
}

// one block per row: scale by 2^-floor(log2 max |a_ij|), record the scale and |row|_1
__global__ void equilibrate_kernel(float *A, int n, double *rowscale, double *rownorm)
{
    __shared__ float smax[32];
    __shared__ double ssum[32];
    float *row = A + (size_t)blockIdx.x * n;
    float m = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(row[j]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? smax[threadIdx.x] : 0.f;
        for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) smax[0] = v;
    }
    __syncthreads();
    const float mx = smax[0];
    // a power of two: the scaled row is exact, so the equilibrated system is
    // D A itself and the refined solution keeps FP64 accuracy for A
    const float sc = mx > 0.f ? ldexpf(1.0f, -ilogbf(mx)) : 1.0f;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float v = row[j] * sc;
        row[j] = v;
        s += fabs((double)v);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ssum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ssum[w];
        rownorm[blockIdx.x] = t;
        rowscale[blockIdx.x] = (double)sc;
    }
}

// ------------------------------------------------------------------ panel exchange
// The CTAs of the pivoting panel (a cooperative launch) meet once per column:
// each CTA writes its pivot candidate (a 64-bit record and the candidate's
// row), then arrives on a monotonic counter (zero at the launch) with a
// release add; a CTA waits for column j until the counter reaches (j + 1) x
// the CTAs (acquire loads) and then reads every record.  Records and rows go
// to two buffer sets used by alternate columns: a CTA rewrites a set two
// columns later, after every CTA has arrived for the column in between, i.e.
// has finished reading it.  The wait is bounded: after BARRIER_WAIT_NS on
// the global timer the CTA records OBEM_ERR_TIMEOUT in flag[0] and gives up.
#define BARRIER_WAIT_NS 2000000000ull
#define PAN_MAXG 1024           // largest panel grid
// records [2][PAN_MAXG] (64-bit), gdiag [2][LU_NB], candidate rows [2][PAN_MAXG][LU_NB]
#define PAN_REC_FLOATS (4 * PAN_MAXG)
#define PAN_SCRATCH_FLOATS (PAN_REC_FLOATS + 2 * LU_NB + 2 * PAN_MAXG * LU_NB)
#define PAN_PLAN_FLOATS 260     // the row swaps' plan (1 + 4 LU_NB ints, padded to 16 bytes)

__device__ __forceinline__ unsigned long long gb_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Called by warp 0 only: waits until *count >= target and returns the
// largest of the G records (in every lane), 0 when the wait ran out (then
// flag[0] = OBEM_ERR_TIMEOUT).  Lane 0 polls with acquire loads; the warp
// barrier after it orders the other lanes' reads of the records.
__device__ unsigned long long pan_wait_records(const unsigned long long *recs, int G, const unsigned *count,
                                               unsigned target, int *flag)
{
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane == 0) {
        const unsigned long long t0 = gb_now();
        for (unsigned it = 1;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if ((it & 63u) == 0u && gb_now() - t0 > BARRIER_WAIT_NS) {
                ok = 0;
                atomicExch(flag, OBEM_ERR_TIMEOUT);
                break;
            }
        }
    }
    __syncwarp();
    ok = __shfl_sync(0xffffffffu, ok, 0);
    unsigned long long best = 0ull;
    if (ok)
        for (int t = lane; t < G; t += 32) {
            const unsigned long long v = __ldcg(recs + t);
            best = v > best ? v : best;
        }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long v2 = __shfl_xor_sync(0xffffffffu, best, o);
        best = v2 > best ? v2 : best;
    }
    return ok ? (best ? best : 1ull) : 0ull;
}

// Failure-detection self-test: the blocks arrive and wait for one block more
// than was launched, so every wait runs out after BARRIER_WAIT_NS and records
// OBEM_ERR_TIMEOUT in flag[0] (flag[1]: the counter, flag[2..]: records).
__global__ void barrier_timeout_kernel(int *flag)
{
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"((unsigned *)&flag[1]) : "memory");
    pan_wait_records((const unsigned long long *)(flag + 2), 1, (const unsigned *)&flag[1], gridDim.x + 1, flag);
}

extern "C" int obem_selftest_wait_timeout(obem_ctx *c, obem_stream stream)
{
    if (!c) return OBEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *flag = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&flag, sizeof(int) * 8));
    int h = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int) * 8, s);
    if (e == cudaSuccess) {
        barrier_timeout_kernel<<<2, 32, 0, s>>>(flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return obem_fail(c, OBEM_ERR_CUDA, "wait self-test: %s", cudaGetErrorString(e));
    if (h != OBEM_ERR_TIMEOUT) return obem_fail(c, OBEM_ERR_STATE, "wait self-test: status %d, expected a timeout", h);
    return OBEM_OK;
}

struct PanelArgs {
    float *A;
    int n, k, kb, rows_per_cta;
    int *piv;
    int *flag;          // [0] status, [1] arrival counter (zero at the launch)
    unsigned long long *rec;    // [2][PAN_MAXG] CTA b's candidate: |pivot| bits << 32 | ~row, 1: none
    float *crows;       // [2][PAN_MAXG][LU_NB] the candidate row's panel values
    float *gdiag;       // [2][LU_NB] the row receiving the pivot, before the swap
};

// best candidate over the CTA, in every thread: v = |a| (-1: none), r = its
// row, larger |a| first, ties to the lower row.  One CTA barrier; the warps'
// results go to the buffer set `par` (calls alternate the sets, so a set is
// rewritten only after the barriers of the call in between).
__device__ __forceinline__ void pan_reduce(float &v, int &r, unsigned (*sv)[8], unsigned (*sr)[8], int par)
{
    // non-negative floats order as their bits; +1 leaves 0 for "none"
    const unsigned kv = v < 0.f ? 0u : __float_as_uint(v) + 1u;
    const unsigned m = __reduce_max_sync(0xffffffffu, kv);
    const unsigned rm = __reduce_min_sync(0xffffffffu, kv == m ? (unsigned)r : 0xffffffffu);
    if ((threadIdx.x & 31) == 0) {
        sv[par][threadIdx.x >> 5] = m;
        sr[par][threadIdx.x >> 5] = rm;
    }
    __syncthreads();
    unsigned bm = sv[par][0], br = sr[par][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        const unsigned m2 = sv[par][w], r2 = sr[par][w];
        if (m2 > bm || (m2 == bm && r2 < br)) { bm = m2; br = r2; }
    }
    v = bm == 0u ? -1.f : __uint_as_float(bm - 1u);
    r = bm == 0u ? 0x7fffffff : (int)br;
}

// Warp 0 publishes the CTA's candidate for column col: the candidate row bi
// and, from its owner, the row that receives the pivot (both up to date),
// then the record, then the arrival.  With j >= 0 the two rows' columns
// j + 2 .. kb - 1 are first brought up to date with the multipliers of
// column j (the rest of the CTA's rows are updated after the publication);
// j = -1: no update.
__device__ __forceinline__ void pan_publish(const PanelArgs &a, int col, int j, float bv, int bi, int r0, int rows,
                                            float *sp, int ld, const float *urow)
{
    const int lane = threadIdx.x & 31, kb = a.kb, b = blockIdx.x;
    const int par = col & 1;
    const int pr = a.k + col;
    float *crow = a.crows + ((size_t)par * PAN_MAXG + b) * LU_NB;
    float *gd = a.gdiag + par * LU_NB;
    const bool has = bi != 0x7fffffff;
    const bool own = pr >= r0 && pr < r0 + rows;
    for (int c = lane; c < kb; c += 32) {
        if (has) {
            float *row = sp + (size_t)(bi - r0) * ld;
            float x = row[c];
            if (j >= 0 && c >= j + 2) {
                x = fmaf(-row[j], urow[c], x);
                row[c] = x;
            }
            crow[c] = x;
            if (bi == pr) gd[c] = x;
        }
        if (own && bi != pr) {
            float *row = sp + (size_t)(pr - r0) * ld;
            float x = row[c];
            if (j >= 0 && c >= j + 2) {
                x = fmaf(-row[j], urow[c], x);
                row[c] = x;
            }
            gd[c] = x;
        }
    }
    if (lane == 0)
        a.rec[(size_t)par * PAN_MAXG + b] =
            has ? ((unsigned long long)__float_as_uint(bv) << 32) | (unsigned)(~(unsigned)bi) : 1ull;
    __syncwarp();
    // release: the warp's writes above are visible to any CTA that acquires
    // the counter after this arrival
    if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"((unsigned *)&a.flag[1]) : "memory");
}

// Panel factorisation of A[k:n, k:k+kb] with partial pivoting.  CTA b owns
// rows k + b*R .. k + (b+1)*R - 1 of the panel in shared memory.  Per column
// j: wait for every CTA's candidate of column j and take the largest (the
// same pivot in every CTA), fetch the pivot row, swap, form the multipliers
// and update column j + 1 of the own rows, find the CTA's candidate for
// column j + 1 and publish it (warp 0, which then waits for the next
// column); the other warps update the other columns of the own rows
// meanwhile.
__global__ void __launch_bounds__(256)
panel_kernel(PanelArgs a)
{
    extern __shared__ float sp[];            // [R][kb + 1] (padded against bank conflicts)
    __shared__ unsigned sv[2][8], sr[2][8];
    __shared__ unsigned long long skey;
    __shared__ float urow[LU_NB];
    const int R = a.rows_per_cta, kb = a.kb, n = a.n, k = a.k;
    const int ld = kb + 1;
    const int b = blockIdx.x, G = gridDim.x;
    const int r0 = k + b * R;
    const int rows = max(0, min(R, n - r0));
    const int tid = threadIdx.x, warp = tid >> 5;
    // a factorisation that already failed (zero pivot, a wait that ran out)
    // stops here instead of waiting again in every later panel
    if (*(volatile const int *)a.flag != 0) return;
    {
        // 8 loads in flight per thread before the shared-memory stores
        const int tot = rows * kb;
        for (int t0 = 0; t0 < tot; t0 += 8 * 256) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u * 256 + tid;
                v[u] = t < tot ? a.A[(size_t)(r0 + t / kb) * n + k + t % kb] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u * 256 + tid;
                if (t < tot) sp[(t / kb) * ld + t % kb] = v[u];
            }
        }
    }
    __syncthreads();
    {
        // candidate of column 0
        float bv = -1.f;
        int bi = 0x7fffffff;
        for (int r = tid; r < rows; r += blockDim.x) {
            const float v = fabsf(sp[r * ld]);
            if (v > bv) { bv = v; bi = r0 + r; }
        }
        pan_reduce(bv, bi, sv, sr, 0);
        if (warp == 0) pan_publish(a, 0, -1, bv, bi, r0, rows, sp, ld, urow);
    }
    for (int j = 0; j < kb; ++j) {
        const int par = j & 1;
        const int pr = k + j;                     // row receiving the pivot
        if (warp == 0) {
            const unsigned long long kw =
                pan_wait_records(a.rec + (size_t)par * PAN_MAXG, G, (const unsigned *)&a.flag[1],
                                 (unsigned)(j + 1) * (unsigned)G, a.flag);
            if (tid == 0) skey = kw;
        }
        __syncthreads();
        const unsigned long long key = skey;
        if (key == 0ull) return;                  // the wait ran out
        const float v = __uint_as_float((unsigned)(key >> 32));
        const int p = (int)(~(unsigned)(key & 0xffffffffu));
        if (key == 1ull || !(v > 0.f)) {
            // singular: every CTA stops here; the panel's remaining pivots
            // are set to no swap
            if (tid == 0) atomicCAS(a.flag, 0, OBEM_ERR_SINGULAR);
            if (b == 0)
                for (int jj = j + tid; jj < kb; jj += blockDim.x) a.piv[k + jj] = k + jj;
            return;
        }
        const int q = (p - k) / R;                // the CTA holding the pivot row
        if (tid < kb) {
            const float u = __ldcg(a.crows + ((size_t)par * PAN_MAXG + q) * LU_NB + tid);
            const float g = __ldcg(a.gdiag + par * LU_NB + tid);
            urow[tid] = u;
            if (pr >= r0 && pr < r0 + rows) sp[(pr - r0) * ld + tid] = u;
            if (p != pr && p >= r0 && p < r0 + rows) sp[(p - r0) * ld + tid] = g;
        }
        if (b == 0 && tid == 0) a.piv[pr] = p;
        __syncthreads();
        const float inv = 1.0f / urow[j];
        if (j + 1 == kb) {
            for (int r = tid; r < rows; r += blockDim.x)
                if (r0 + r > pr) sp[r * ld + j] *= inv;
            break;
        }
        // multipliers of column j, column j + 1 of the own rows, candidate
        const float u1 = urow[j + 1];
        float bv = -1.f;
        int bi = 0x7fffffff;
        for (int r = tid; r < rows; r += blockDim.x) {
            const int gr = r0 + r;
            if (gr <= pr) continue;
            const float l = sp[r * ld + j] * inv;
            sp[r * ld + j] = l;
            const float x = fmaf(-l, u1, sp[r * ld + j + 1]);
            sp[r * ld + j + 1] = x;
            const float ax = fabsf(x);
            if (ax > bv) { bv = ax; bi = gr; }
        }
        pan_reduce(bv, bi, sv, sr, (j + 1) & 1);
        if (warp == 0) {
            pan_publish(a, j + 1, j, bv, bi, r0, rows, sp, ld, urow);
        } else {
            // the other rows' columns j + 2 .. kb - 1, while warp 0 waits
            // for the next column (the barrier after that wait comes before
            // any of them is read)
            const int nx = pr + 1;
            for (int r = tid - 32; r < rows; r += (int)blockDim.x - 32) {
                const int gr = r0 + r;
                if (gr <= pr || gr == bi || gr == nx) continue;
                float *row = sp + (size_t)r * ld;
                const float l = row[j];
#pragma unroll 8
                for (int c = j + 2; c < kb; ++c) row[c] = fmaf(-l, urow[c], row[c]);
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < rows * kb; t += blockDim.x) {
        int r = t / kb, c = t % kb;
        a.A[(size_t)(r0 + r) * n + k + c] = sp[r * ld + c];
    }
}

// The panel's kb row swaps (piv[k .. k + kb)) applied to the columns outside
// the panel, unless the factorisation's status (flag[0]) records a failure,
// in three launches: laswp_plan_kernel lists the rows the swaps touch (the kb
// panel rows and the distinct pivot rows below the panel, at most 2 kb) and,
// for each, the touched row whose content it receives (the swaps undone in
// reverse order, independently per row); laswp_gather_kernel copies the
// touched rows whole into a scratch block, laswp_scatter_kernel writes each
// receiving row from it.  Whole-row copies stream at the HBM rate; a
// single-pass permutation in shared memory (every block holding a column
// slice of all touched rows) ran at a fifth of it.
#define LS_PLAN_INTS (1 + 4 * LU_NB)        // m, rows[2 LU_NB], src[2 LU_NB]
__global__ void __launch_bounds__(LU_NB) laswp_plan_kernel(int k, int kb, const int *piv, int *flag, int *plan)
{
    // the panel's arrival counter, zeroed for the next panel
    if (threadIdx.x == 0) flag[1] = 0;
    // a panel that stopped (zero pivot, a wait that ran out) may have left
    // pivots unwritten: no swaps then
    if (*(volatile const int *)flag != 0) {
        if (threadIdx.x == 0) plan[0] = 0;
        return;
    }
    __shared__ int s_piv[LU_NB], s_pos[LU_NB], s_row[2 * LU_NB];
    __shared__ unsigned s_first[LU_NB / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    // the position of every swap's pivot row among the touched rows: panel
    // rows first, then the pivot rows below the panel by first appearance
    const int p = tid < kb ? piv[k + tid] : -1;
    s_piv[tid] = p;
    __syncthreads();
    // the first swap with the same pivot row (all 64 reads in flight)
    int f = tid;
#pragma unroll
    for (int q = LU_NB - 1; q >= 0; --q)
        if (q < tid && s_piv[q] == p) f = q;
    const bool first = tid < kb && p >= k + kb && f == tid;
    const unsigned bal = __ballot_sync(0xffffffffu, first);
    if (lane == 0) s_first[tid >> 5] = bal;
    __syncthreads();
    const unsigned long long mask = (unsigned long long)s_first[0] | ((unsigned long long)s_first[1] << 32);
    if (tid < kb) {
        s_pos[tid] = p < k + kb ? p - k : kb + __popcll(mask & ((1ull << f) - 1ull));
        s_row[tid] = k + tid;
    }
    if (first) s_row[kb + __popcll(mask & ((1ull << tid) - 1ull))] = p;
    const int m = kb + __popcll(mask);
    __syncthreads();
    // the touched row whose content ends in touched row t: the swaps
    // (position q <-> s_pos[q], q = 0 .. kb-1, in order) undone in reverse
    for (int t = tid; t < m; t += blockDim.x) {
        int j = t;
#pragma unroll
        for (int q = LU_NB - 1; q >= 0; --q) {
            const int pq = q < kb ? s_pos[q] : q;
            j = j == q ? pq : (j == pq ? q : j);
        }
        plan[1 + t] = s_row[t];
        plan[1 + 2 * LU_NB + t] = j;
    }
    if (tid == 0) plan[0] = m;
}

// S[q][:] = A[rows[q]][:] for the touched rows q < m (grid y: q)
__global__ void laswp_gather_kernel(const float *__restrict__ A, int n, const int *plan, float *__restrict__ S)
{
    const int q = blockIdx.y;
    if (q >= plan[0]) return;
    const float *a = A + (size_t)plan[1 + q] * n;
    float *d = S + (size_t)q * n;
    const int stride = gridDim.x * blockDim.x;
    if ((n & 3) == 0) {
        for (int c4 = blockIdx.x * blockDim.x + threadIdx.x; c4 < n / 4; c4 += stride)
            ((float4 *)d)[c4] = __ldcs((const float4 *)a + c4);
    } else {
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) d[c] = __ldcs(a + c);
    }
}

// A[rows[t]][c] = S[src[t]][c] for the touched rows t < m that receive
// another row, outside the panel's own columns [k, k + kb) (the panel kernel
// already swapped those)
__global__ void laswp_scatter_kernel(float *__restrict__ A, int n, int k, int kb, const int *plan,
                                     const float *__restrict__ S)
{
    const int t = blockIdx.y;
    if (t >= plan[0]) return;
    const int sq = plan[1 + 2 * LU_NB + t];
    if (sq == t) return;
    float *d = A + (size_t)plan[1 + t] * n;
    const float *a = S + (size_t)sq * n;
    const int stride = gridDim.x * blockDim.x;
    if ((n & 3) == 0 && (k & 3) == 0 && ((k + kb) & 3) == 0) {
        for (int c4 = blockIdx.x * blockDim.x + threadIdx.x; c4 < n / 4; c4 += stride)
            if (4 * c4 < k || 4 * c4 >= k + kb) ((float4 *)d)[c4] = __ldcs((const float4 *)a + c4);
    } else {
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride)
            if (c < k || c >= k + kb) d[c] = __ldcs(a + c);
    }
}

// U12 = L11^-1 A12 with L11 unit lower triangular (kb x kb); a CTA of
// TRSM_COLS threads owns TRSM_COLS columns, held in shared memory
#define TRSM_COLS 64
__global__ void trsm_kernel(float *A, int n, int k, int kb)
{
    __shared__ float L[LU_NB][LU_NB + 1];
    __shared__ float X[LU_NB][TRSM_COLS];
    for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) {
        int r = t / kb, c = t % kb;
        L[r][c] = A[(size_t)(k + r) * n + k + c];
    }
    const int c = k + kb + blockIdx.x * TRSM_COLS + threadIdx.x;
    const bool act = c < n;
    for (int r = 0; r < kb; ++r) X[r][threadIdx.x] = act ? A[(size_t)(k + r) * n + c] : 0.f;
    __syncthreads();
    for (int q = 0; q < kb; ++q) {
        const float xq = X[q][threadIdx.x];
        for (int r = q + 1; r < kb; ++r) X[r][threadIdx.x] = fmaf(-L[r][q], xq, X[r][threadIdx.x]);
    }
    if (act)
        for (int r = 0; r < kb; ++r) A[(size_t)(k + r) * n + c] = X[r][threadIdx.x];
}

// T[r][c] = M[(r0 + r) * n + c0 + c] for r, c < kb (kb <= LU_NB), loaded by
// blockDim.x (a multiple of 64) threads with 16 loads in flight per thread
// before the shared-memory stores (the loads of a few-CTA kernel are
// latency-bound otherwise)
__device__ __forceinline__ void load_block(float (*T)[LU_NB + 1], const float *M, int n, int r0, int c0, int kb,
                                           bool transpose)
{
    const int c = threadIdx.x & 63, rstep = blockDim.x >> 6;
    for (int rb = threadIdx.x >> 6; rb < kb; rb += 16 * rstep) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = rb + i * rstep;
            v[i] = (r < kb && c < kb) ? M[(size_t)(r0 + r) * n + c0 + c] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = rb + i * rstep;
            if (r < kb && c < kb) {
                if (transpose) T[c][r] = v[i];
                else T[r][c] = v[i];
            }
        }
    }
}

// X = L^-1 X for the unit lower triangular block L = A[r0:r0+m, r0:r0+m]
// (m <= M) and X = A[r0:r0+m, c0:c0+nc]: one thread per column of X, the
// block's columns staged through shared memory (coalesced loads and stores)
// and each column's M values held in registers; L transposed in shared
// memory (zero outside its strict lower triangle; a column of L read as
// broadcast float4).  For q = 0 .. M-2, x[r] -= L[r][q] x[q] for every
// r > q, in FP32 (64 rows at a time in registers, each row's updates still
// in the order of q).  M = 64 or 128: the leaves of the recursive TRSM (a 128-row
// leaf replaces two 64-row leaves and the BF16 tensor-core update between
// them).
#define TRSM_LEAF 128
#define TRSM_LEAF_THREADS 128
__device__ __forceinline__ unsigned tl_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int M>
constexpr size_t trsm_leaf_smem() { return sizeof(float) * (size_t)M * (M + TRSM_LEAF_THREADS); }
template <int M>
__global__ void __launch_bounds__(TRSM_LEAF_THREADS)
trsm_leaf_kernel(float *A, int n, int r0, int m, int c0, int nc)
{
    extern __shared__ float4 tl_L4[];            // [M][M / 4]: row q = column q of L
    float *Lt = (float *)tl_L4;
    float *Xs = Lt + M * M;                      // [M][TRSM_LEAF_THREADS]
    const int tid = threadIdx.x;
    const int col = blockIdx.x * TRSM_LEAF_THREADS + tid;
    const bool live = col < nc;
    float *x = A + (size_t)r0 * n + c0 + col;
    // every load of the block in flight at once: 4-byte asynchronous copies
    // into shared memory (a zero-size source writes a zero).  L: lanes take
    // consecutive rows (conflict-free transposed stores); X: lanes take
    // consecutive columns (coalesced).
    for (int t = tid; t < M * M; t += blockDim.x) {
        const int r = t % M, q = t / M;
        const bool in = r < m && q < r;
        const float *src = in ? A + (size_t)(r0 + r) * n + r0 + q : A;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tl_smem(&Lt[q * M + r])), "l"(src),
                     "r"(in ? 4 : 0)
                     : "memory");
    }
    for (int r = 0; r < M; ++r) {
        const bool in = live && r < m;
        const float *src = in ? x + (size_t)r * n : A;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tl_smem(&Xs[r * TRSM_LEAF_THREADS + tid])),
                     "l"(src), "r"(in ? 4 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // 64 rows at a time in registers: the rows of the earlier blocks (already
    // solved, back in shared memory) first, then the block's own triangle
#pragma unroll
    for (int h = 0; h < M / 64; ++h) {
        float v[64];
#pragma unroll
        for (int r = 0; r < 64; ++r) v[r] = Xs[(64 * h + r) * TRSM_LEAF_THREADS + tid];
#pragma unroll 4
        for (int q = 0; q < 64 * h; ++q) {
            const float xq = Xs[q * TRSM_LEAF_THREADS + tid];
#pragma unroll
            for (int r4 = 0; r4 < 64; r4 += 4) {
                const float4 l = tl_L4[q * (M / 4) + (64 * h + r4) / 4];
                v[r4] = fmaf(-l.x, xq, v[r4]);
                v[r4 + 1] = fmaf(-l.y, xq, v[r4 + 1]);
                v[r4 + 2] = fmaf(-l.z, xq, v[r4 + 2]);
                v[r4 + 3] = fmaf(-l.w, xq, v[r4 + 3]);
            }
        }
#pragma unroll
        for (int q = 0; q < 63; ++q) {
            const float xq = v[q];
#pragma unroll
            for (int r4 = (q + 1) & ~3; r4 < 64; r4 += 4) {
                const float4 l = tl_L4[(64 * h + q) * (M / 4) + (64 * h + r4) / 4];
                if (r4 > q) v[r4] = fmaf(-l.x, xq, v[r4]);
                if (r4 + 1 > q) v[r4 + 1] = fmaf(-l.y, xq, v[r4 + 1]);
                if (r4 + 2 > q) v[r4 + 2] = fmaf(-l.z, xq, v[r4 + 2]);
                if (r4 + 3 > q) v[r4 + 3] = fmaf(-l.w, xq, v[r4 + 3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 64; ++r) Xs[(64 * h + r) * TRSM_LEAF_THREADS + tid] = v[r];
    }
    if (!live) return;
#pragma unroll 8
    for (int r = 0; r < m; ++r) x[(size_t)r * n] = Xs[r * TRSM_LEAF_THREADS + tid];
}

// The same leaf solve for narrow X (few blocks: the latency of one block
// decides): one warp per 4 columns, lane l holding rows l, l + 32, ... of
// them in registers, L row-major in shared memory (padded: the column reads
// are conflict-free), x[q] broadcast by a shuffle at step q.  Same updates
// in the same order as trsm_leaf_kernel (the results are identical).
#define TL2_C 4
#define TL2_W 8
#define TL2_BC (TL2_C * TL2_W)
template <int M>
constexpr size_t trsm_leaf2_smem() { return sizeof(float) * ((size_t)M * (M + 1) + (size_t)M * (TL2_BC + 1)); }
template <int M>
__global__ void __launch_bounds__(TL2_W * 32)
trsm_leaf2_kernel(float *A, int n, int r0, int m, int c0, int nc)
{
    constexpr int RL = M / 32;
    extern __shared__ float tl2_s[];
    float *Ls = tl2_s;                    // [M][M + 1]: L row-major, padded (column reads conflict-free)
    float *Xs = tl2_s + M * (M + 1);      // [M][TL2_BC + 1]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cb = blockIdx.x * TL2_BC;
    for (int t = tid; t < M * M; t += blockDim.x) {
        const int r = t / M, q = t % M;           // coalesced over q
        const bool in = r < m && q < r;
        const float *src = in ? A + (size_t)(r0 + r) * n + r0 + q : A;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tl_smem(&Ls[r * (M + 1) + q])), "l"(src),
                     "r"(in ? 4 : 0)
                     : "memory");
    }
    for (int e = tid; e < M * TL2_BC; e += blockDim.x) {
        const int r = e / TL2_BC, c = e % TL2_BC;
        const bool in = r < m && cb + c < nc;
        const float *src = in ? A + (size_t)(r0 + r) * n + c0 + cb + c : A;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tl_smem(&Xs[r * (TL2_BC + 1) + c])),
                     "l"(src), "r"(in ? 4 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    float v[TL2_C][RL];
#pragma unroll
    for (int j = 0; j < TL2_C; ++j)
#pragma unroll
        for (int i = 0; i < RL; ++i) v[j][i] = Xs[(32 * i + lane) * (TL2_BC + 1) + warp * TL2_C + j];
#pragma unroll
    for (int q = 0; q < M - 1; ++q) {
        float lq[RL];
#pragma unroll
        for (int i = 0; i < RL; ++i) lq[i] = Ls[(32 * i + lane) * (M + 1) + q];
#pragma unroll
        for (int j = 0; j < TL2_C; ++j) {
            const float xq = __shfl_sync(0xffffffffu, v[j][q / 32], q % 32);
#pragma unroll
            for (int i = 0; i < RL; ++i)
                if (32 * i + 31 > q && 32 * i + lane > q) v[j][i] = fmaf(-lq[i], xq, v[j][i]);
        }
    }
#pragma unroll
    for (int j = 0; j < TL2_C; ++j)
#pragma unroll
        for (int i = 0; i < RL; ++i) Xs[(32 * i + lane) * (TL2_BC + 1) + warp * TL2_C + j] = v[j][i];
    __syncthreads();
    for (int e = tid; e < M * TL2_BC; e += blockDim.x) {
        const int r = e / TL2_BC, c = e % TL2_BC;
        if (r < m && cb + c < nc) A[(size_t)(r0 + r) * n + c0 + cb + c] = Xs[r * (TL2_BC + 1) + c];
    }
}

// ------------------------------------------------------------------ solve kernels
// b_i = rowscale_i * (V_group or free density) + drhs_i  (drhs unscaled input)
__global__ void rhs_kernel(const int *kind, const int *group, const double *gv, const float *sigma_free,
                           const float *drhs, const double *rowscale, double *b, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    if (kind[i] == OBEM_CELL_ELECTRODE) v = gv[group[i]];
    else if (sigma_free) v = (double)sigma_free[i];
    if (drhs) v += (double)drhs[i];
    b[i] = v * rowscale[i];
}

// r = b - A x (FP64 accumulation over the FP32 matrix), one warp per row
// x = xh + xl in two floats (xl: the rounding remainder of xh, so that
// |x - xh - xl| <= 2^-48 |x|)
__global__ void split_kernel(const double *x, float *xh, float *xl, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)x[i];
    xh[i] = h;
    xl[i] = (float)(x[i] - (double)h);
}

// r = b - A x in FP64 without FP64 products: a warp per row; each product
// a xh is split exactly (FMA) into its float value p and error e, p goes to
// a per-lane two-sum (s, c) and e + a xl to c; the lanes' s + c are added
// in FP64.  The result differs from the FP64 dot product by a few units of
// 2^-48 of sum |a x|.
__device__ __forceinline__ void df_acc(float &s, float &c, float a, float h, float l)
{
    const float p = __fmul_rn(a, h);
    const float e = __fmaf_rn(a, h, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(a, l, e)));
    s = t;
}
__global__ void __launch_bounds__(256) residual_kernel(const float *A, const float *xh, const float *xl,
                                                       const double *b, double *r, int n)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *a = A + (size_t)row * n;
    float s = 0.f, c = 0.f;
    int j = lane;
    for (; j + 32 * 7 < n; j += 32 * 8) {
        float av[8], hv[8], lv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            av[u] = __ldcs(a + j + 32 * u);
            hv[u] = xh[j + 32 * u];
            lv[u] = xl[j + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) df_acc(s, c, av[u], hv[u], lv[u]);
    }
    for (; j < n; j += 32) df_acc(s, c, a[j], xh[j], xl[j]);
    double v = (double)s + (double)c;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) r[row] = b[row] - v;
}
__global__ void norms_kernel(const double *r, const double *x, const double *b, int n, double *out)
{
    __shared__ double s[3][256];
    double a0 = 0, a1 = 0, a2 = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a0 = fmax(a0, fabs(r[i])); a1 = fmax(a1, fabs(x[i])); a2 = fmax(a2, fabs(b[i]));
    }
    s[0][threadIdx.x] = a0; s[1][threadIdx.x] = a1; s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] = fmax(s[q][threadIdx.x], s[q][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s[0][0]; out[1] = s[1][0]; out[2] = s[2][0]; }
}

// y = P r / sc in FP32 (sc = max |r|): the factorisation's row swaps as one
// gather, y[i] = r[perm[i]] / sc
__global__ void permute_kernel(const double *r, float *y, const int *perm, int n, const double *norms)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = norms[0] > 0 ? norms[0] : 1.0;
    y[i] = (float)(r[perm[i]] / sc);
}



__global__ void axpy_kernel(double *x, const float *d, const double *norms, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sc = norms[0] > 0 ? norms[0] : 1.0;
    x[i] += (double)d[i] * sc;
}

__global__ void to_float_kernel(const double *x, float *a, float *b, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = (float)x[i];
    a[i] = v;
    if (b) b[i] = v;
}

// ------------------------------------------------------------------ one-launch triangular solves
// Forward (unit lower L) or backward (upper U) substitution with the factors
// in one launch.  Block row i of TS_R rows is taken by the thread block that
// draws ticket i (in dependency order: i = 0 is the first block row of L,
// the last of U), so every block row it depends on belongs to a thread block
// that started before it, whatever the scheduling.  Each warp owns TS_R / 8
// rows and runs over the solved blocks of y in dependency order; the loads
// of y wait for that block's flag to show the launch's epoch.  The block row
// then multiplies its right-hand side, less the solved part, by the inverse
// of its diagonal block (computed once after the factorisation) and
// publishes its y values and flag.  A wait on a flag is bounded
// (TS_WAIT_NS): one that runs out records OBEM_ERR_TIMEOUT and goes on, so
// that the launch always ends.
#define TS_WAIT_NS 2000000000ull
#define TS_SMEM (sizeof(float) * (TS_R * (TS_R + 1) + TS_R))
#define TS_INV_SMEM (sizeof(float) * 2 * TS_R * (TS_R + 1))

__device__ __forceinline__ unsigned long long ts_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ts_ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ts_st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct TsArgs {
    const float *LU;
    const float *dinv;  // inverses of the diagonal blocks (inv_diag_kernel)
    float *y;           // right-hand side in, solution out
    int n, lower, epoch;
    int *flags;         // [nbk] epoch of the last launch that solved the block row
    int *ticket;        // zero before the launch
    int *err;
};

// Inverses of the diagonal blocks (TS_R x TS_R) of the unit lower factor L
// (blockIdx.y = 0) and of the upper factor U (blockIdx.y = 1): thread c
// solves for column c of the inverse by substitution; rows and columns past
// the matrix are zero.
#define TS_LD (TS_R + 1)
__global__ void __launch_bounds__(TS_R) inv_diag_kernel(const float *LU, int n, float *dinv)
{
    extern __shared__ float ts_sm[];
    float *T = ts_sm, *X = ts_sm + TS_R * TS_LD;
    const int blk = blockIdx.x, upper = blockIdx.y, c = threadIdx.x;
    const int r0 = blk * TS_R, rows = min(TS_R, n - r0);
    for (int e = c; e < TS_R * TS_R; e += TS_R) {
        const int i = e / TS_R, k = e % TS_R;
        T[i * TS_LD + k] = (i < rows && k < rows) ? LU[(size_t)(r0 + i) * n + r0 + k] : 0.f;
    }
    __syncthreads();
    if (!upper) {
        for (int i = 0; i < TS_R; ++i) {
            float v = (i == c && i < rows) ? 1.f : 0.f;
            for (int k = c; k < i; ++k) v = fmaf(-T[i * TS_LD + k], X[k * TS_LD + c], v);
            X[i * TS_LD + c] = (i < rows && c < rows) ? v : 0.f;
        }
    } else {
        for (int i = TS_R - 1; i >= 0; --i) {
            float v = (i == c && i < rows) ? 1.f : 0.f;
            for (int k = i + 1; k <= c; ++k) v = fmaf(-T[i * TS_LD + k], X[k * TS_LD + c], v);
            X[i * TS_LD + c] = (i < rows && c < rows) ? v / T[i * TS_LD + i] : 0.f;
        }
    }
    __syncthreads();
    float *D = dinv + (size_t)(2 * blk + upper) * TS_R * TS_R;
    for (int e = c; e < TS_R * TS_R; e += TS_R) D[e] = X[(e / TS_R) * TS_LD + e % TS_R];
}

__global__ void __launch_bounds__(256) trsv_chain_kernel(TsArgs a)
{
    extern __shared__ float ts_sm[];
    float *D = ts_sm;                        // [TS_R][TS_LD] inverse of the diagonal block
    float *s_b = ts_sm + TS_R * TS_LD;       // [TS_R] right-hand side minus the solved part
    __shared__ int s_t;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    constexpr int RW = TS_R / 8;             // rows per warp
    const int n = a.n, nbk = (n + TS_R - 1) / TS_R;
    if (tid == 0) s_t = atomicAdd(a.ticket, 1);
    __syncthreads();
    const int t = s_t;
    const int blk = a.lower ? t : nbk - 1 - t;
    const int r0 = blk * TS_R, rows = min(TS_R, n - r0);
    {
        const float *g = a.dinv + (size_t)(2 * blk + (a.lower ? 0 : 1)) * TS_R * TS_R;
        for (int e = tid; e < TS_R * TS_R; e += 256) D[(e / TS_R) * TS_LD + e % TS_R] = g[e];
    }
    float acc[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) acc[r] = 0.f;
    int ready = 0;          // dependency steps this warp knows to be solved
    for (int st = 0; st < t; ++st) {
        const int j = a.lower ? st : nbk - 1 - st;
        const int c0 = j * TS_R, cols = min(TS_R, n - c0);
        if (st >= ready) {
            // flags of steps st .. st + 31, until step st is solved
            const unsigned long long t0 = ts_now();
            for (unsigned it = 0;; ++it) {
                const int q = st + lane;
                const int f = q < t ? ts_ld_acquire(a.flags + (a.lower ? q : nbk - 1 - q)) : 0;
                const unsigned ok = __ballot_sync(0xffffffffu, q < t && f == a.epoch);
                if (ok & 1u) {
                    ready = st + (~ok ? __ffs(~ok) - 1 : 32);
                    break;
                }
                if ((it & 63u) == 63u && ts_now() - t0 > TS_WAIT_NS) {
                    if (lane == 0) atomicExch(a.err, OBEM_ERR_TIMEOUT);
                    ready = st + 1;
                    break;
                }
                __nanosleep(32);
            }
            __syncwarp();
        }
#pragma unroll
        for (int h = 0; h < TS_R; h += 64) {
            float l0[RW], l1[RW];
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int row = RW * w + r;
                const float *arow = a.LU + (size_t)(r0 + row) * n + c0 + h;
                l0[r] = (row < rows && h + lane < cols) ? arow[lane] : 0.f;
                l1[r] = (row < rows && h + lane + 32 < cols) ? arow[lane + 32] : 0.f;
            }
            const float y0 = h + lane < cols ? __ldcg(a.y + c0 + h + lane) : 0.f;
            const float y1 = h + lane + 32 < cols ? __ldcg(a.y + c0 + h + lane + 32) : 0.f;
#pragma unroll
            for (int r = 0; r < RW; ++r) acc[r] = fmaf(l0[r], y0, fmaf(l1[r], y1, acc[r]));
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        float v = acc[r];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int row = RW * w + r;
        if (lane == 0) s_b[row] = row < rows ? a.y[r0 + row] - v : 0.f;
    }
    __syncthreads();
    if (tid < rows) {
        const float *d = D + tid * TS_LD;
        float v = 0.f;
        for (int k = 0; k < rows; ++k) v = fmaf(d[k], s_b[k], v);
        a.y[r0 + tid] = v;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) ts_st_release(a.flags + blk, a.epoch);
}

// The transposed substitutions of the adjoint solve, A^T x = b with
// P A = L U: U^T (lower, forward; lower = 1) and L^T (unit upper, backward;
// lower = 0) in one launch each, with the same tickets and flags.  Block row
// i of U^T (L^T) is block column i of U (L): thread (c, half) sums column c
// over every other row of each solved block j, whose y values warp 0 puts in
// shared memory (double-buffered, one barrier per block); the diagonal block
// uses the transposed inverse.
#define TS_T_SMEM (sizeof(float) * (TS_R * (TS_R + 1) + 4 * TS_R))
__global__ void __launch_bounds__(256) trsv_chain_t_kernel(TsArgs a)
{
    extern __shared__ float ts_sm[];
    float *D = ts_sm;                        // [TS_R][TS_LD]
    float *s_b = D + TS_R * TS_LD;           // [TS_R]
    float *s_z = s_b + TS_R;                 // [2][TS_R]
    float *s_h = s_z + 2 * TS_R;             // [TS_R]
    __shared__ int s_t;
    const int tid = threadIdx.x, lane = tid & 31, c = tid & (TS_R - 1), half = tid / TS_R;
    const int n = a.n, nbk = (n + TS_R - 1) / TS_R;
    if (tid == 0) s_t = atomicAdd(a.ticket, 1);
    __syncthreads();
    const int t = s_t;
    const int blk = a.lower ? t : nbk - 1 - t;
    const int i0 = blk * TS_R, ni = min(TS_R, n - i0);
    {
        const float *g = a.dinv + (size_t)(2 * blk + (a.lower ? 1 : 0)) * TS_R * TS_R;
        for (int e = tid; e < TS_R * TS_R; e += 256) D[(e / TS_R) * TS_LD + e % TS_R] = g[e];
    }
    float acc = 0.f;
    int ready = 0;
    for (int st = 0; st < t; ++st) {
        const int j = a.lower ? st : nbk - 1 - st;
        const int j0 = j * TS_R, nj = min(TS_R, n - j0);
        float *z = s_z + (st & 1) * TS_R;
        if (tid < 32) {
            if (st >= ready) {
                const unsigned long long t0 = ts_now();
                for (unsigned it = 0;; ++it) {
                    const int q = st + lane;
                    const int f = q < t ? ts_ld_acquire(a.flags + (a.lower ? q : nbk - 1 - q)) : 0;
                    const unsigned ok = __ballot_sync(0xffffffffu, q < t && f == a.epoch);
                    if (ok & 1u) {
                        ready = st + (~ok ? __ffs(~ok) - 1 : 32);
                        break;
                    }
                    if ((it & 63u) == 63u && ts_now() - t0 > TS_WAIT_NS) {
                        if (lane == 0) atomicExch(a.err, OBEM_ERR_TIMEOUT);
                        ready = st + 1;
                        break;
                    }
                    __nanosleep(32);
                }
                __syncwarp();
            }
#pragma unroll
            for (int q = 0; q < TS_R / 32; ++q) {
                const int r = lane + 32 * q;
                z[r] = r < nj ? __ldcg(a.y + j0 + r) : 0.f;
            }
        }
        __syncthreads();
        if (c < ni) {
            const float *col = a.LU + (size_t)j0 * n + i0 + c;
            int r = half;
            for (; r + 14 < nj; r += 16) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = col[(size_t)(r + 2 * u) * n];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc = fmaf(v[u], z[r + 2 * u], acc);
            }
            for (; r < nj; r += 2) acc = fmaf(col[(size_t)r * n], z[r], acc);
        }
    }
    if (half == 1) s_h[c] = acc;
    __syncthreads();
    if (half == 0) s_b[c] = c < ni ? a.y[i0 + c] - (acc + s_h[c]) : 0.f;
    __syncthreads();
    if (tid < ni) {
        float v = 0.f;
        for (int k = 0; k < ni; ++k) v = fmaf(D[k * TS_LD + tid], s_b[k], v);
        a.y[i0 + tid] = v;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) ts_st_release(a.flags + blk, a.epoch);
}

// ------------------------------------------------------------------ host drivers
// A22 -= L21 U12 for the panel at column k (width kb) in cuBLAS (FP32, TF32
// or BF16x9 arithmetic).  A is row-major; cuBLAS sees it column-major, i.e.
// transposed, so the call computes A22^T -= U12^T L21^T with U12 as its first
// operand.
static int gemm_update(obem_ctx *c, int precision, float *A, int n, int k, int kb, cudaStream_t s)
{
    const int M = n - k - kb;
    if (M <= 0) return OBEM_OK;
    const float alpha = -1.0f, beta = 1.0f;
    float *A22 = A + (size_t)(k + kb) * n + (k + kb);
    float *L21 = A + (size_t)(k + kb) * n + k;
    float *U12 = A + (size_t)k * n + (k + kb);
    cublasComputeType_t ct = CUBLAS_COMPUTE_32F;
    if (precision == OBEM_LU_TF32) ct = CUBLAS_COMPUTE_32F_FAST_TF32;
    else if (precision == OBEM_LU_BF16X9) ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    cublasStatus_t st = cublasGemmEx(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, M, M, kb, &alpha, U12,
                                     CUDA_R_32F, n, L21, CUDA_R_32F, n, &beta, A22, CUDA_R_32F, n, ct,
                                     CUBLAS_GEMM_DEFAULT);
    if (st != CUBLAS_STATUS_SUCCESS)
        return obem_fail(c, OBEM_ERR_CUDA, "cublasGemmEx failed (status %d)", (int)st);
    return OBEM_OK;
}

// Pivoting panel factorisation of A[k:n, k:k+kb] (cooperative panel_kernel)
// followed by its row swaps on every other column.
struct PanelScratch {
    float *cval, *crows, *gdiag;    // cval: the 2 x PAN_MAXG 64-bit candidate records
    int *plan;                      // the row swaps' plan (LS_PLAN_INTS)
    float *rows;                    // [2 LU_NB][n] the touched rows during the swaps
    int nsm;
};

static int factor_panel(obem_ctx *c, const PanelScratch &P, int k, int kb, cudaStream_t s)
{
    const int n = c->nsys;
    const int rows = n - k;
    int G = (rows + 31) / 32;
    if (G > P.nsm) G = P.nsm;
    // above ~nsm x 787 rows (about 120k cells) one chunk per SM no longer
    // fits a CTA's shared memory: m = 2, 3, 4 co-resident CTAs per SM,
    // each chunk within 1/m of the SM's 224 KB (the occupancy check
    // below rejects a size that still does not fit)
    const size_t row_b = sizeof(float) * (size_t)(kb + 1);
    if ((size_t)((rows + G - 1) / G) * row_b > 200 * 1024)
        for (int m = 2; m <= 4; ++m) {
            G = m * P.nsm;
            if ((size_t)((rows + G - 1) / G) * row_b <= (size_t)224 * 1024 / m) break;
        }
    if (G > PAN_MAXG) G = PAN_MAXG;
    int R = (rows + G - 1) / G;
    G = (rows + R - 1) / R;
    size_t smem = sizeof(float) * (size_t)R * (kb + 1);
    if (smem > 200 * 1024)
        return obem_fail(c, OBEM_ERR_ARG, "LU panel of %d rows does not fit shared memory", rows);
    // host-side queries once, not per panel (they cost tens of microseconds
    // each, and the factorisation issues a panel every few hundred): the
    // attribute at the largest panel size; one CTA per SM always fits (at
    // most 200 KB of shared memory, 48 registers x 256 threads), so the
    // occupancy is checked only when there are more CTAs than SMs
    static unsigned long long attr = 0;   // devices done (a bit each)
    if (!(attr >> (c->device & 63) & 1ull)) {
        OBEM_CUDA(c, cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr |= 1ull << (c->device & 63);
    }
    if (G > P.nsm) {
        int per_sm = 0;
        OBEM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel, 256, smem));
        if (per_sm * P.nsm < G)
            return obem_fail(c, OBEM_ERR_CUDA, "LU panel: %d CTAs cannot be co-resident", G);
    }
    PanelArgs pa;
    pa.A = c->d_LU; pa.n = n; pa.k = k; pa.kb = kb; pa.rows_per_cta = R; pa.piv = c->d_piv;
    pa.flag = c->d_flag; pa.rec = (unsigned long long *)P.cval; pa.crows = P.crows; pa.gdiag = P.gdiag;
    void *args[] = {&pa};
    OBEM_CUDA(c, cudaLaunchCooperativeKernel((void *)panel_kernel, dim3(G), dim3(256), args, smem, s));
    laswp_plan_kernel<<<1, LU_NB, 0, s>>>(k, kb, c->d_piv, c->d_flag, P.plan);
    const dim3 lg(n / 1024 + 1 < 64 ? n / 1024 + 1 : 64, 2 * LU_NB);
    laswp_gather_kernel<<<lg, 256, 0, s>>>(c->d_LU, n, P.plan, P.rows);
    laswp_scatter_kernel<<<lg, 256, 0, s>>>(c->d_LU, n, k, kb, P.plan, P.rows);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

// Split of a recursive block of w columns: a multiple of LU_NB near w / 2.
static int rec_split(int w)
{
    const int h = (w / (2 * LU_NB)) * LU_NB;
    return h > LU_NB ? h : LU_NB;
}

// X = L^-1 X with L = LU[r0:r0+m, r0:r0+m] (unit lower) and X = LU[r0:r0+m,
// c0:c0+nc], recursively: X1 = L11^-1 X1, X2 -= L21 X1 (tensor-core GEMM),
// X2 = L22^-1 X2.
static int rec_trsm(obem_ctx *c, int r0, int m, int c0, int nc, cudaStream_t s)
{
    const int n = c->nsys;
    float *A = c->d_LU;
    if (nc <= 0 || m <= 0) return OBEM_OK;
    if (m <= TRSM_LEAF) {
        const int nb = (nc + TRSM_LEAF_THREADS - 1) / TRSM_LEAF_THREADS;
        static unsigned long long attr = 0;   // devices done (a bit each)
        if (!(attr >> (c->device & 63) & 1ull)) {
            OBEM_CUDA(c, cudaFuncSetAttribute(trsm_leaf_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)trsm_leaf_smem<64>()));
            OBEM_CUDA(c, cudaFuncSetAttribute(trsm_leaf_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)trsm_leaf_smem<128>()));
            OBEM_CUDA(c, cudaFuncSetAttribute(trsm_leaf2_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)trsm_leaf2_smem<64>()));
            OBEM_CUDA(c, cudaFuncSetAttribute(trsm_leaf2_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)trsm_leaf2_smem<128>()));
            attr |= 1ull << (c->device & 63);
        }
        const int nb2 = (nc + TL2_BC - 1) / TL2_BC;
        if (nc <= 8192) {
            // narrow: the warp-per-columns form has the shorter block latency
            if (m <= 64)
                trsm_leaf2_kernel<64><<<nb2, TL2_W * 32, trsm_leaf2_smem<64>(), s>>>(A, n, r0, m, c0, nc);
            else
                trsm_leaf2_kernel<128><<<nb2, TL2_W * 32, trsm_leaf2_smem<128>(), s>>>(A, n, r0, m, c0, nc);
        } else if (m <= 64) {
            trsm_leaf_kernel<64><<<nb, TRSM_LEAF_THREADS, trsm_leaf_smem<64>(), s>>>(A, n, r0, m, c0, nc);
        } else {
            trsm_leaf_kernel<128><<<nb, TRSM_LEAF_THREADS, trsm_leaf_smem<128>(), s>>>(A, n, r0, m, c0, nc);
        }
        OBEM_LAUNCH(c);
        return OBEM_OK;
    }
    const int m1 = rec_split(m);
    int rc = rec_trsm(c, r0, m1, c0, nc, s);
    if (rc == OBEM_OK)
        rc = obem_tc_gemm_sub(c, A + (size_t)(r0 + m1) * n + c0, n, A + (size_t)(r0 + m1) * n + r0, n,
                              A + (size_t)r0 * n + c0, n, m - m1, nc, m1, c->d_flag + 4, s);
    if (rc == OBEM_OK) rc = rec_trsm(c, r0 + m1, m - m1, c0, nc, s);
    return rc;
}

// Largest BF16 operands (elements, rows x 8-padded K) of the GEMMs that
// rec_lu / rec_trsm issue, so that the scratch is reserved once.
static void rec_trsm_sizes(int m, int nc, size_t &a, size_t &b)
{
    if (nc <= 0 || m <= TRSM_LEAF) return;
    const int m1 = rec_split(m);
    const size_t k8 = ((size_t)m1 + 7) / 8 * 8;
    a = a > (size_t)(m - m1) * k8 ? a : (size_t)(m - m1) * k8;
    b = b > (size_t)nc * k8 ? b : (size_t)nc * k8;
    rec_trsm_sizes(m1, nc, a, b);
    rec_trsm_sizes(m - m1, nc, a, b);
}

static void rec_lu_sizes(int n, int k0, int w, size_t &a, size_t &b)
{
    if (w <= LU_NB) return;
    const int w1 = rec_split(w);
    const size_t k8 = ((size_t)w1 + 7) / 8 * 8;
    rec_lu_sizes(n, k0, w1, a, b);
    rec_trsm_sizes(w1, w - w1, a, b);
    a = a > (size_t)(n - k0 - w1) * k8 ? a : (size_t)(n - k0 - w1) * k8;
    b = b > (size_t)(w - w1) * k8 ? b : (size_t)(w - w1) * k8;
    rec_lu_sizes(n, k0 + w1, w - w1, a, b);
}

// Recursive LU with partial pivoting of the columns [k0, k0 + w) of rows
// [k0, n) (Toledo's recursion): factor the left half, U12 = L11^-1 A12,
// A22 -= L21 U12 on the tensor cores (BF16 operands, FP32 accumulation into
// the FP32 matrix), factor the right half.  Panels of LU_NB columns are the
// leaves; their row swaps are applied to whole rows at once.
static int rec_lu(obem_ctx *c, const PanelScratch &P, int k0, int w, cudaStream_t s)
{
    const int n = c->nsys;
    float *A = c->d_LU;
    if (w <= LU_NB) return factor_panel(c, P, k0, w, s);
    const int w1 = rec_split(w);
    int rc = rec_lu(c, P, k0, w1, s);
    if (rc == OBEM_OK) rc = rec_trsm(c, k0, w1, k0 + w1, w - w1, s);
    if (rc == OBEM_OK)
        rc = obem_tc_gemm_sub(c, A + (size_t)(k0 + w1) * n + (k0 + w1), n, A + (size_t)(k0 + w1) * n + k0, n,
                              A + (size_t)k0 * n + (k0 + w1), n, n - k0 - w1, w - w1, w1, c->d_flag + 4, s);
    if (rc == OBEM_OK) rc = rec_lu(c, P, k0 + w1, w - w1, s);
    return rc;
}

// Buffers of an n x n system (matrix, factors, pivots, scaling, refinement
// and panel scratch), reallocated when n changes.
static int alloc_system(obem_ctx *c, int n)
{
    if (c->d_A && c->nsys_alloc == n) return OBEM_OK;
    void *bufs[] = {c->d_A, c->d_LU, c->d_piv, c->d_rowscale, c->d_work64, c->d_work32, c->d_flag, c->d_panel,
                    c->d_perm, c->d_trsv, c->d_dinv};
    for (void *q : bufs)
        if (q) cudaFree(q);
    c->d_A = c->d_LU = NULL;
    c->d_piv = c->d_flag = c->d_perm = c->d_trsv = NULL;
    c->d_dinv = NULL;
    c->d_rowscale = c->d_work64 = NULL;
    c->d_work32 = c->d_panel = NULL;
    c->nsys_alloc = 0;
    const size_t nn = (size_t)n * n;
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_A, sizeof(float) * nn));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_LU, sizeof(float) * nn));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_piv, sizeof(int) * n));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_rowscale, sizeof(double) * n));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_work64, sizeof(double) * (4 * (size_t)n + 8)));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_work32, sizeof(float) * (2 * (size_t)n + 4096)));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_flag, sizeof(int) * 8));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_panel,
                            sizeof(float) * (PAN_SCRATCH_FLOATS + PAN_PLAN_FLOATS + 2 * (size_t)LU_NB * n)));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_perm, sizeof(int) * n));
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_trsv, sizeof(int) * ((size_t)n / TS_R + 16)));
    OBEM_CUDA(c, cudaMemset(c->d_trsv, 0, sizeof(int) * ((size_t)n / TS_R + 16)));
    c->trsv_epoch = 0;
    OBEM_CUDA(c, cudaMalloc((void **)&c->d_dinv, sizeof(float) * 2 * TS_R * TS_R * (size_t)((n + TS_R - 1) / TS_R)));
    c->nsys_alloc = n;
    return OBEM_OK;
}

static int factor_system(obem_ctx *c, int precision, cudaStream_t s);

int obem_assemble_and_factor(obem_ctx *c, int precision, cudaStream_t s)
{
    c->factored = 0;
    c->nsys = c->np;
    const int n = c->nsys;
    int rc0 = alloc_system(c, n);
    if (rc0 != OBEM_OK) return rc0;
    // --- assembly
    PanelsDev P;
    P.c_a = c->d_c_a; P.g0_h = c->d_g0_h; P.g1 = c->d_g1; P.g2 = c->d_g2; P.nrm = c->d_nrm;
    P.c_lo = c->d_c_lo;
    P.v64 = c->d_v64; P.geo = c->d_geo64; P.np = n;
    double *d_em = NULL, *d_ep = NULL;
    struct FreeOnExit { void *p; ~FreeOnExit() { if (p) cudaFree(p); } };
    OBEM_CUDA(c, cudaMalloc((void **)&d_em, sizeof(double) * n));
    FreeOnExit em_guard{d_em};
    OBEM_CUDA(c, cudaMalloc((void **)&d_ep, sizeof(double) * n));
    FreeOnExit ep_guard{d_ep};
    OBEM_CUDA(c, cudaMemcpyAsync(d_em, c->h_em, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    OBEM_CUDA(c, cudaMemcpyAsync(d_ep, c->h_ep, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    dim3 ag(n, (n + 127) / 128);
    assemble_kernel<<<ag, 128, 0, s>>>(P, c->d_kind, d_em, d_ep, c->d_A, n);
    OBEM_LAUNCH(c);
    return factor_system(c, precision, s);
}

// A caller-given dense system in place of an assembled one (see obem.h).
int obem_factor_dense(obem_ctx *c, const float *A, int n, int precision, cudaStream_t s)
{
    c->factored = 0;
    c->nsys = n;
    int rc = alloc_system(c, n);
    if (rc != OBEM_OK) return rc;
    OBEM_CUDA(c, cudaMemcpyAsync(c->d_A, A, sizeof(float) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    return factor_system(c, precision, s);
}

// Row equilibration of d_A (rows scaled by 1 / max |a_ij|, ||A||_inf kept for
// the backward error), LU factorisation into d_LU in the requested
// arithmetic, and the row permutation of the pivots.
static int factor_system(obem_ctx *c, int precision, cudaStream_t s)
{
    const int n = c->nsys;
    const size_t nn = (size_t)n * n;
    if (!c->cublas) {
        if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS)
            return obem_fail(c, OBEM_ERR_CUDA, "cublasCreate failed");
    }
    cublasSetStream(c->cublas, s);
    double *d_rownorm = c->d_work64;     // reused as scratch here
    equilibrate_kernel<<<n, 256, 0, s>>>(c->d_A, n, c->d_rowscale, d_rownorm);
    OBEM_LAUNCH(c);
    std::vector<double> rn(n);
    OBEM_CUDA(c, cudaMemcpyAsync(rn.data(), d_rownorm, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    c->a_norm_inf = 0.0;
    for (int i = 0; i < n; ++i) c->a_norm_inf = rn[i] > c->a_norm_inf ? rn[i] : c->a_norm_inf;
    // --- factorisation
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    OBEM_CUDA(c, cudaMemcpyAsync(c->d_LU, c->d_A, sizeof(float) * nn, cudaMemcpyDeviceToDevice, s));
    OBEM_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int) * 8, s));
    cudaEventRecord(e0, s);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    PanelScratch PS;
    PS.cval = c->d_panel;
    PS.gdiag = c->d_panel + PAN_REC_FLOATS;
    PS.crows = c->d_panel + PAN_REC_FLOATS + 2 * LU_NB;
    PS.plan = (int *)(c->d_panel + PAN_SCRATCH_FLOATS);
    PS.rows = c->d_panel + PAN_SCRATCH_FLOATS + PAN_PLAN_FLOATS;
    PS.nsm = nsm;
    if (precision == OBEM_LU_BF16) {
        // recursive factorisation, trailing updates on the tensor cores
        size_t ea = 0, eb = 0;
        rec_lu_sizes(n, 0, n, ea, eb);
        int rc = obem_tc_reserve(c, ea, eb);
        if (rc == OBEM_OK) rc = rec_lu(c, PS, 0, n, s);
        if (rc != OBEM_OK) return rc;
    } else {
        // right-looking blocked factorisation, trailing updates in cuBLAS
        for (int k = 0; k < n; k += LU_NB) {
            const int kb = n - k < LU_NB ? n - k : LU_NB;
            int rc = factor_panel(c, PS, k, kb, s);
            if (rc != OBEM_OK) return rc;
            if (k + kb < n) {
                trsm_kernel<<<(n - k - kb + TRSM_COLS - 1) / TRSM_COLS, TRSM_COLS, 0, s>>>(c->d_LU, n, k, kb);
                OBEM_LAUNCH(c);
                rc = gemm_update(c, precision, c->d_LU, n, k, kb, s);
                if (rc != OBEM_OK) return rc;
            }
        }
    }
    cudaEventRecord(e1, s);
    int flag[8] = {0};
    OBEM_CUDA(c, cudaMemcpyAsync(flag, c->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->factor_ms = ms;
    if (flag[0] == OBEM_ERR_SINGULAR) return obem_fail(c, OBEM_ERR_SINGULAR, "LU: zero pivot");
    if (flag[0] == OBEM_ERR_TIMEOUT) return obem_fail(c, OBEM_ERR_TIMEOUT, "LU: a panel's wait for the pivot candidates timed out");
    if (flag[4] != 0) return obem_fail(c, OBEM_ERR_TIMEOUT, "LU: a tensor-core GEMM wait timed out");
    // the row swaps as one permutation: (P b)[i] = b[perm[i]]
    {
        std::vector<int> piv(n), perm(n);
        OBEM_CUDA(c, cudaMemcpy(piv.data(), c->d_piv, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = 0; i < n; ++i)
            if (piv[i] != i) { const int t = perm[i]; perm[i] = perm[piv[i]]; perm[piv[i]] = t; }
        OBEM_CUDA(c, cudaMemcpy(c->d_perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    }
    // inverses of the diagonal blocks for the one-launch substitutions
    {
        static unsigned long long attr = 0;   // devices done (a bit each)
        if (!(attr >> (c->device & 63) & 1ull)) {
            OBEM_CUDA(c, cudaFuncSetAttribute(inv_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)TS_INV_SMEM));
            OBEM_CUDA(c, cudaFuncSetAttribute(trsv_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)TS_SMEM));
            attr |= 1ull << (c->device & 63);
        }
        inv_diag_kernel<<<dim3((n + TS_R - 1) / TS_R, 2), TS_R, TS_INV_SMEM, s>>>(c->d_LU, n, c->d_dinv);
        OBEM_LAUNCH(c);
    }
    c->factored = 1;
    return OBEM_OK;
}

// y <- U^-1 L^-1 y with the stored factors: two one-launch substitutions.
// A flag wait that ran out is reported as OBEM_ERR_TIMEOUT after the launch.
static int lu_solve(obem_ctx *c, float *y, cudaStream_t s)
{
    const int n = c->nsys, nbk = (n + TS_R - 1) / TS_R;
    int *ticket = c->d_trsv + nbk, *err = ticket + 2;
    OBEM_CUDA(c, cudaMemsetAsync(ticket, 0, sizeof(int) * 3, s));
    for (int lower = 1; lower >= 0; --lower) {
        TsArgs a;
        a.LU = c->d_LU;
        a.dinv = c->d_dinv;
        a.y = y;
        a.n = n;
        a.lower = lower;
        a.epoch = ++c->trsv_epoch;
        a.flags = c->d_trsv;
        a.ticket = ticket + (lower ? 0 : 1);
        a.err = err;
        trsv_chain_kernel<<<nbk, 256, TS_SMEM, s>>>(a);
        OBEM_LAUNCH(c);
    }
    int h = 0;
    OBEM_CUDA(c, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    if (h != 0) return obem_fail(c, OBEM_ERR_TIMEOUT, "LU solve: a wait for a solved block timed out");
    return OBEM_OK;
}

// Failure-detection self-test of the substitutions' flag wait: one thread
// block draws ticket 1 (the counter starts at 1) and waits for block row 0,
// which no block solves; the wait runs out after TS_WAIT_NS and records
// OBEM_ERR_TIMEOUT.  Needs the factors of a system of at least 2 TS_R rows.
int obem_selftest_solve_wait(obem_ctx *c, cudaStream_t s)
{
    if (!c->factored || c->nsys < 2 * TS_R)
        return obem_fail(c, OBEM_ERR_STATE, "wait self-test: needs the factors of a system of >= %d rows", 2 * TS_R);
    const int n = c->nsys, nbk = (n + TS_R - 1) / TS_R;
    int *ticket = c->d_trsv + nbk, *err = ticket + 2;
    const int one = 1;
    OBEM_CUDA(c, cudaMemsetAsync(ticket, 0, sizeof(int) * 3, s));
    OBEM_CUDA(c, cudaMemcpyAsync(ticket, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    TsArgs a;
    a.LU = c->d_LU;
    a.dinv = c->d_dinv;
    a.y = c->d_work32;
    a.n = n;
    a.lower = 1;
    a.epoch = ++c->trsv_epoch;
    a.flags = c->d_trsv;
    a.ticket = ticket;
    a.err = err;
    trsv_chain_kernel<<<1, 256, TS_SMEM, s>>>(a);
    OBEM_LAUNCH(c);
    int h = 0;
    OBEM_CUDA(c, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    if (h != OBEM_ERR_TIMEOUT) return obem_fail(c, OBEM_ERR_STATE, "wait self-test: status %d, expected a timeout", h);
    return OBEM_OK;
}

// Iterative refinement of A x = b with the stored factors: b (device, FP64,
// rows already equilibrated) in c->d_work64[0, n), x in [n, 2n); FP64
// residuals r = b - A x from the FP32 equilibrated matrix, corrections from
// the factors.  Returns the iterations, status and backward error.
static int refine(obem_ctx *c, int &it, int &status, double &be, cudaStream_t s)
{
    const int n = c->nsys;
    double *b = c->d_work64, *x = b + n, *r = x + n, *nrm = r + n;
    float *y = c->d_work32;
    OBEM_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    double be_prev = 2.0;
    be = 1.0;
    it = 0;
    status = OBEM_ERR_NOT_CONVERGED;
    const int max_it = 30;
    for (; it <= max_it; ++it) {
        split_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, y, y + n, n);
        residual_kernel<<<(n + 7) / 8, 256, 0, s>>>(c->d_A, y, y + n, b, r, n);
        norms_kernel<<<1, 256, 0, s>>>(r, x, b, n, nrm);
        OBEM_LAUNCH(c);
        double h[3];
        OBEM_CUDA(c, cudaMemcpyAsync(h, nrm, sizeof h, cudaMemcpyDeviceToHost, s));
        OBEM_CUDA(c, cudaStreamSynchronize(s));
        be = h[0] / (c->a_norm_inf * h[1] + h[2] + 1e-300);
        // converged: at the FP64 rounding level, or no longer decreasing once
        // below 1e-9 (the residual's own rounding floor for large n)
        if (be < 1e-12 || (be < 1e-9 && be > 0.5 * be_prev)) { status = OBEM_OK; break; }
        be_prev = be;
        if (it == max_it) break;
        permute_kernel<<<(n + 255) / 256, 256, 0, s>>>(r, y, c->d_perm, n, nrm);
        OBEM_LAUNCH(c);
        int rc = lu_solve(c, y, s);
        if (rc != OBEM_OK) return rc;
        axpy_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, y, nrm, n);
        OBEM_LAUNCH(c);
    }
    return OBEM_OK;
}

static void fill_report(obem_ctx *c, obem_solve_report *rep, int it, int status, double be, float ms)
{
    if (!rep) return;
    rep->iterations = it;
    rep->status = status;
    rep->backward_error = be;
    rep->factor_ms = c->factor_ms;
    rep->solve_ms = ms;
}

int obem_solve_system(obem_ctx *c, const double *gv, const float *sigma_free, const float *drhs,
                      float *sigma_out, obem_solve_report *rep, cudaStream_t s)
{
    const int n = c->nsys;
    cublasSetStream(c->cublas, s);
    double *b = c->d_work64, *x = b + n;
    double *d_gv = NULL;
    int ng = c->n_groups > 0 ? c->n_groups : 1;
    OBEM_CUDA(c, cudaMalloc((void **)&d_gv, sizeof(double) * ng));
    struct FreeOnExit { void *p; ~FreeOnExit() { if (p) cudaFree(p); } } gv_guard{d_gv};
    if (c->n_groups > 0)
        OBEM_CUDA(c, cudaMemcpyAsync(d_gv, gv, sizeof(double) * c->n_groups, cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    rhs_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->d_kind, c->d_group, d_gv, sigma_free, drhs, c->d_rowscale, b, n);
    OBEM_LAUNCH(c);
    int it = 0, status = OBEM_ERR_NOT_CONVERGED;
    double be = 1.0;
    int rc = refine(c, it, status, be, s);
    if (rc != OBEM_OK) return rc;
    to_float_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, sigma_out, c->d_sigma, n);
    OBEM_LAUNCH(c);
    cudaEventRecord(e1, s);
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sigma_valid = 1;
    c->sigma_ver++;
    fill_report(c, rep, it, status, be, ms);
    if (status != OBEM_OK)
        return obem_fail(c, OBEM_ERR_NOT_CONVERGED, "refinement stopped at backward error %.3e after %d iterations", be, it);
    return OBEM_OK;
}

// b_i = rowscale_i * bin_i
__global__ void scale_rhs_kernel(const double *bin, const double *rowscale, double *b, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = bin[i] * rowscale[i];
}

// Solve of the dense system given to obem_dense_factor for one right-hand
// side (device FP64 b, x), with the same refinement as the BEM solve.
int obem_solve_dense_rhs(obem_ctx *c, const double *bin, double *xout, obem_solve_report *rep, cudaStream_t s)
{
    const int n = c->nsys;
    double *b = c->d_work64, *x = b + n;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    scale_rhs_kernel<<<(n + 255) / 256, 256, 0, s>>>(bin, c->d_rowscale, b, n);
    OBEM_LAUNCH(c);
    int it = 0, status = OBEM_ERR_NOT_CONVERGED;
    double be = 1.0;
    int rc = refine(c, it, status, be, s);
    if (rc != OBEM_OK) return rc;
    OBEM_CUDA(c, cudaMemcpyAsync(xout, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    cudaEventRecord(e1, s);
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fill_report(c, rep, it, status, be, ms);
    if (status != OBEM_OK)
        return obem_fail(c, OBEM_ERR_NOT_CONVERGED, "refinement stopped at backward error %.3e after %d iterations", be, it);
    return OBEM_OK;
}

// ====================================================================
// Adjoint of the solve: mu = A^-T g (g = dL/dsigma) is dL/db for the right-hand
// side of Eq. (matrixBEM).  With the row-equilibrated matrix At = D A and its
// factors P At = L U:  A^T mu = g  <=>  At^T nu = g,  mu = D nu,  and
// At^T = U^T L^T P, so each refinement step solves U^T z = r (forward),
// L^T w = z (backward, unit diagonal) and undoes the row swaps (nu = P^-1 w).
// The residual g - At^T nu is accumulated in FP64 from the stored FP32 At.
// ====================================================================
#define ADJ_SPLIT 16           // row ranges of the transposed residual

// part[s][j] = sum over rows i of range s of At[i][j] x[i]; one thread per column
__global__ void residual_t_part_kernel(const float *A, const float *xh, const float *xl, double *part, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const int i0 = (int)((long long)n * s / ADJ_SPLIT), i1 = (int)((long long)n * (s + 1) / ADJ_SPLIT);
    if (j >= n) return;
    float sm = 0.f, cm = 0.f;
    int i = i0;
    for (; i + 7 < i1; i += 8) {
        float av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) av[u] = __ldcs(A + (size_t)(i + u) * n + j);
#pragma unroll
        for (int u = 0; u < 8; ++u) df_acc(sm, cm, av[u], xh[i + u], xl[i + u]);
    }
    for (; i < i1; ++i) df_acc(sm, cm, A[(size_t)i * n + j], xh[i], xl[i]);
    part[(size_t)s * n + j] = (double)sm + (double)cm;
}
__global__ void residual_t_fold_kernel(const double *part, const double *b, double *r, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int q = 0; q < ADJ_SPLIT; ++q) s += part[(size_t)q * n + j];
    r[j] = b[j] - s;
}

// colsum[j] = sum_i |At[i][j]|  (for the transposed system's infinity norm)
__global__ void colsum_kernel(const float *A, double *colsum, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs((double)A[(size_t)i * n + j]);
    colsum[j] = s;
}

__global__ void max_kernel(const double *v, int n, double *out)
{
    __shared__ double s[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a = fmax(a, v[i]);
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void load_adjoint_kernel(const float *g, double *b, double *x, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = (double)g[i];
    x[i] = 0.0;
}

// y = r / sc in FP32 (sc = max|r|)
__global__ void scale_to_float_kernel(const double *r, float *y, int n, const double *norms)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = norms[0] > 0 ? norms[0] : 1.0;
    y[i] = (float)(r[i] / sc);
}

// x += P^T y sc: the transposed row permutation as a scatter, x[perm[i]] +=
// y[i] sc (sc = max |r|)
__global__ void axpy_unpermute_kernel(double *x, const float *y, const int *perm, const double *norms, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = norms[0] > 0 ? norms[0] : 1.0;
    x[perm[i]] += (double)y[i] * sc;
}



// y <- L^-T U^-T y with the stored factors (the adjoint's substitutions)
static int lu_solve_t(obem_ctx *c, float *y, cudaStream_t s)
{
    const int n = c->nsys, nbk = (n + TS_R - 1) / TS_R;
    int *ticket = c->d_trsv + nbk, *err = ticket + 2;
    static unsigned long long attr = 0;   // devices done (a bit each)
    if (!(attr >> (c->device & 63) & 1ull)) {
        OBEM_CUDA(c, cudaFuncSetAttribute(trsv_chain_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)TS_T_SMEM));
        attr |= 1ull << (c->device & 63);
    }
    OBEM_CUDA(c, cudaMemsetAsync(ticket, 0, sizeof(int) * 3, s));
    for (int lower = 1; lower >= 0; --lower) {
        TsArgs a;
        a.LU = c->d_LU;
        a.dinv = c->d_dinv;
        a.y = y;
        a.n = n;
        a.lower = lower;
        a.epoch = ++c->trsv_epoch;
        a.flags = c->d_trsv;
        a.ticket = ticket + (lower ? 0 : 1);
        a.err = err;
        trsv_chain_t_kernel<<<nbk, 256, TS_T_SMEM, s>>>(a);
        OBEM_LAUNCH(c);
    }
    int h = 0;
    OBEM_CUDA(c, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    if (h != 0) return obem_fail(c, OBEM_ERR_TIMEOUT, "adjoint solve: a wait for a solved block timed out");
    return OBEM_OK;
}

int obem_solve_adjoint(obem_ctx *c, const float *g, double *dL_dgv, float *dL_db, obem_solve_report *rep,
                       cudaStream_t s)
{
    const int n = c->nsys;
    double *b = c->d_work64, *x = b + n, *r = x + n, *nrm = r + n;
    float *y = c->d_work32;
    double *part = NULL, *col = NULL, *mu = NULL;
    int rc = OBEM_OK, it = 0, status = OBEM_ERR_NOT_CONVERGED;
    double be = 1.0, be_prev = 2.0, a1 = 0.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
#define ADJ_CUDA(call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            rc = obem_fail(c, OBEM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
            goto done;                                                                             \
        }                                                                                          \
    } while (0)
    ADJ_CUDA(cudaMalloc((void **)&part, sizeof(double) * (size_t)ADJ_SPLIT * n));
    ADJ_CUDA(cudaMalloc((void **)&col, sizeof(double) * ((size_t)n + 1)));
    colsum_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->d_A, col, n);
    max_kernel<<<1, 256, 0, s>>>(col, n, col + n);
    load_adjoint_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, b, x, n);
    ADJ_CUDA(cudaGetLastError());
    ADJ_CUDA(cudaMemcpyAsync(&a1, col + n, sizeof(double), cudaMemcpyDeviceToHost, s));
    for (; it <= 30; ++it) {
        split_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, y, y + n, n);
        residual_t_part_kernel<<<dim3((n + 255) / 256, ADJ_SPLIT), 256, 0, s>>>(c->d_A, y, y + n, part, n);
        residual_t_fold_kernel<<<(n + 255) / 256, 256, 0, s>>>(part, b, r, n);
        norms_kernel<<<1, 256, 0, s>>>(r, x, b, n, nrm);
        ADJ_CUDA(cudaGetLastError());
        double h[3];
        ADJ_CUDA(cudaMemcpyAsync(h, nrm, sizeof h, cudaMemcpyDeviceToHost, s));
        ADJ_CUDA(cudaStreamSynchronize(s));
        be = h[0] / (a1 * h[1] + h[2] + 1e-300);
        if (be < 1e-12 || (be < 1e-9 && be > 0.5 * be_prev)) { status = OBEM_OK; break; }
        be_prev = be;
        if (it == 30) break;
        scale_to_float_kernel<<<(n + 255) / 256, 256, 0, s>>>(r, y, n, nrm);
        ADJ_CUDA(cudaGetLastError());
        rc = lu_solve_t(c, y, s);
        if (rc != OBEM_OK) goto done;
        axpy_unpermute_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, y, c->d_perm, nrm, n);
        ADJ_CUDA(cudaGetLastError());
    }
    // mu = D nu: the row scale of the equilibrated system
    mu = (double *)malloc(sizeof(double) * (size_t)n);
    {
        double *ds = (double *)malloc(sizeof(double) * (size_t)n);
        if (!mu || !ds) { free(ds); rc = obem_fail(c, OBEM_ERR_ARG, "adjoint: host allocation failed"); goto done; }
        ADJ_CUDA(cudaMemcpyAsync(mu, x, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        ADJ_CUDA(cudaMemcpyAsync(ds, c->d_rowscale, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        ADJ_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) mu[i] *= ds[i];
        free(ds);
    }
    if (dL_dgv) {
        for (int k = 0; k < c->n_groups; ++k) dL_dgv[k] = 0.0;
        for (int i = 0; i < n; ++i)
            if (c->h_kind[i] == OBEM_CELL_ELECTRODE && c->h_group[i] >= 0 && c->h_group[i] < c->n_groups)
                dL_dgv[c->h_group[i]] += mu[i];
    }
    if (dL_db) {
        float *hf = (float *)malloc(sizeof(float) * (size_t)n);
        if (!hf) { rc = obem_fail(c, OBEM_ERR_ARG, "adjoint: host allocation failed"); goto done; }
        for (int i = 0; i < n; ++i) hf[i] = (float)mu[i];
        cudaError_t e = cudaMemcpyAsync(dL_db, hf, sizeof(float) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        free(hf);
        ADJ_CUDA(e);
    }
    cudaEventRecord(e1, s);
    ADJ_CUDA(cudaStreamSynchronize(s));
    if (rep) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        rep->iterations = it;
        rep->status = status;
        rep->backward_error = be;
        rep->factor_ms = c->factor_ms;
        rep->solve_ms = ms;
    }
    if (status != OBEM_OK)
        rc = obem_fail(c, OBEM_ERR_NOT_CONVERGED, "adjoint refinement stopped at backward error %.3e after %d iterations",
                       be, it);
done:
#undef ADJ_CUDA
    free(mu);
    if (part) cudaFree(part);
    if (col) cudaFree(col);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
