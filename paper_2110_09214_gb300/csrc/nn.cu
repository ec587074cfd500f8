// Approximate N-body field (Sec. 3.2.4, the nearest-neighbour "NN" option of
// the paper, O(N) in the number of charges for a fixed grid): the exact
// Coulomb sum of Eq. (nbody) over the charges near a particle, charge centres
// for the farther ones.  The paper gives one sentence; the reading built here:
//   - cubic cells of edge W / G (W: the largest extent of the charges'
//     bounding box, G cells per axis); the cell of a charge is
//     floor((x - lo) * (G / W)) per axis, computed in binary32 with one
//     rounding per operation and clamped to 0..G-1;
//   - near: the exact softened pair sum over the charges of the 27 cells
//     around the particle's cell, itself excluded;
//   - far: every other cell contributes its positive and its negative charge
//     separately, each as the total charge at its charge-weighted centre.
// Pipeline: bounding box (min/max reductions on order-preserving integer
// images of the floats), cell of every charge + counts, exclusive scan,
// counting-sort scatter, per-cell aggregates (FP64 sums), then one thread per
// charge in cell order (so a warp walks the same neighbour lists) for the near
// sum and the far sum over all cells' aggregates staged in shared memory.
#include "obem_internal.cuh"
#include "field_common.cuh"

#define NN_THREADS 256
#define NN_AGG_TILE 256            // cells per shared-memory tile of the far sum
#define NN_CHUNK 32                // pair terms summed in FP32 before each FP64 add

// float <-> integer with the same order (for atomic min / max)
__device__ __forceinline__ int nn_ford(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float nn_fval(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void nn_bbox_init_kernel(int *bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fffffff;              // min
    else if (threadIdx.x < 6) bb[threadIdx.x] = (int)0x80000000;    // max
}

__global__ void nn_bbox_kernel(const float4 *pos, const int32_t *n_dev, int n, int *bb)
{
    const int nn = n_dev ? *n_dev : n;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if ((threadIdx.x & 31) == 0 && mn[0] <= mx[0]) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bb[a], nn_ford(mn[a]));
            atomicMax(&bb[3 + a], nn_ford(mx[a]));
        }
    }
}

struct NnGrid {
    float lo[3], inv;
    int G;
};

__device__ __forceinline__ NnGrid nn_grid(const int *bb, int G)
{
    NnGrid g;
    float wmax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = nn_fval(bb[a]);
        const float w = __fsub_rn(nn_fval(bb[3 + a]), g.lo[a]);
        wmax = w > wmax ? w : wmax;
    }
    if (!(wmax > 0.0f)) wmax = 1.0f;
    g.inv = __fdiv_rn((float)G, wmax);
    g.G = G;
    return g;
}

__device__ __forceinline__ int nn_coord(const NnGrid &g, float x, int a)
{
    const float t = __fmul_rn(__fsub_rn(x, g.lo[a]), g.inv);
    int k = (int)floorf(t);
    return k < 0 ? 0 : (k > g.G - 1 ? g.G - 1 : k);
}

// cell of every charge (packed cx | cy << 10 | cz << 20) and counts
__global__ void nn_cell_kernel(const float4 *pos, const int32_t *n_dev, int n, const int *bb, int G, int32_t *cell,
                               int32_t *count)
{
    const int nn = n_dev ? *n_dev : n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const NnGrid g = nn_grid(bb, G);
    const float4 p = pos[i];
    const int cx = nn_coord(g, p.x, 0), cy = nn_coord(g, p.y, 1), cz = nn_coord(g, p.z, 2);
    cell[i] = cx | (cy << 10) | (cz << 20);
    atomicAdd(&count[(cz * G + cy) * G + cx], 1);
}

// start = exclusive scan of count[0..nc) (nc <= 1024 * 256), start[nc] = total; cursor = start
__global__ void __launch_bounds__(1024) nn_scan_kernel(const int32_t *count, int nc, int32_t *start, int32_t *cursor)
{
    __shared__ int32_t s_sum[1024];
    const int per = (nc + 1023) / 1024;
    const int t = threadIdx.x, b0 = t * per;
    int32_t acc = 0;
    for (int k = 0; k < per && b0 + k < nc; ++k) acc += count[b0 + k];
    s_sum[t] = acc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int32_t v = t >= o ? s_sum[t - o] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    int32_t run = s_sum[t] - acc;
    for (int k = 0; k < per && b0 + k < nc; ++k) {
        start[b0 + k] = run;
        cursor[b0 + k] = run;
        run += count[b0 + k];
    }
    if (t == 1023) start[nc] = s_sum[1023];
}

__global__ void nn_scatter_kernel(const int32_t *n_dev, int n, const int32_t *cell, int G, int32_t *cursor,
                                  int32_t *sorted)
{
    const int nn = n_dev ? *n_dev : n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const int32_t c = cell[i];
    const int idx = (((c >> 20) & 1023) * G + ((c >> 10) & 1023)) * G + (c & 1023);
    sorted[atomicAdd(&cursor[idx], 1)] = i;
}

// per cell: positive and negative charge centres (x, y, z, k_C Q)
__global__ void nn_agg_kernel(const float4 *pos, const int32_t *start, const int32_t *sorted, int nc, float4 *agg)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double sp[4] = {0.0, 0.0, 0.0, 0.0}, sn[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = start[c]; k < start[c + 1]; ++k) {
        const float4 p = pos[sorted[k]];
        double *s = p.w >= 0.0f ? sp : sn;
        const double q = (double)p.w;
        s[0] += q * p.x; s[1] += q * p.y; s[2] += q * p.z; s[3] += q;
    }
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (sp[3] != 0.0) a = make_float4((float)(sp[0] / sp[3]), (float)(sp[1] / sp[3]), (float)(sp[2] / sp[3]),
                                      (float)(OBEM_KC * sp[3]));
    if (sn[3] != 0.0) b = make_float4((float)(sn[0] / sn[3]), (float)(sn[1] / sn[3]), (float)(sn[2] / sn[3]),
                                      (float)(OBEM_KC * sn[3]));
    agg[2 * c] = a;
    agg[2 * c + 1] = b;
}

// softened point-charge field term w (x - y) / (|x - y|^2 + eps^2)^(3/2)
__device__ __forceinline__ void nn_term(float4 x, float4 y, float w, float eps2, float &ax, float &ay, float &az)
{
    const float dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
    if (!(r2 > 0.f)) return;
    const float inv = rsq(r2);
    const float s3 = w * inv * inv * inv;
    ax = fmaf(dx, s3, ax);
    ay = fmaf(dy, s3, ay);
    az = fmaf(dz, s3, az);
}

// field at every charge (one thread per charge, in cell order); E_out adds to
// its initial value when add is set, else starts from e_ext
__global__ void __launch_bounds__(NN_THREADS) nn_field_kernel(const float4 *pos, const int32_t *n_dev, int n,
                                                              const int32_t *cell, const int32_t *start,
                                                              const int32_t *sorted, const float4 *agg, int G,
                                                              float eps2, float4 *E_out, float3 e_ext, int add)
{
    __shared__ float4 s_agg[2 * NN_AGG_TILE];
    const int nn = n_dev ? *n_dev : n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < nn;
    const int i = live ? sorted[t] : 0;
    const float4 x = live ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int32_t ci = live ? cell[i] : 0;
    const int cx = ci & 1023, cy = (ci >> 10) & 1023, cz = (ci >> 20) & 1023;
    const float kC = (float)OBEM_KC;
    double e[3] = {0.0, 0.0, 0.0};
    if (live) {
        // near: charges of the 27 cells around
        for (int dz = -1; dz <= 1; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= G) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= G) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = cx + dx;
                    if (xx < 0 || xx >= G) continue;
                    const int c = (z * G + y) * G + xx;
                    const int k1 = start[c + 1];
                    for (int k0 = start[c]; k0 < k1; k0 += NN_CHUNK) {
                        float ax = 0.f, ay = 0.f, az = 0.f;
                        for (int k = k0; k < min(k1, k0 + NN_CHUNK); ++k) {
                            const int j = sorted[k];
                            if (j == i) continue;
                            const float4 y4 = pos[j];
                            nn_term(x, y4, kC * y4.w, eps2, ax, ay, az);
                        }
                        e[0] += ax; e[1] += ay; e[2] += az;
                    }
                }
            }
        }
    }
    // far: charge centres of every cell outside the 27
    const int nc = G * G * G;
    for (int cb = 0; cb < nc; cb += NN_AGG_TILE) {
        __syncthreads();
        for (int l = threadIdx.x; l < 2 * NN_AGG_TILE; l += blockDim.x) {
            const int c = cb + l / 2;
            s_agg[l] = c < nc ? agg[2 * cb + l] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (!live) continue;
        const int cn = min(NN_AGG_TILE, nc - cb);
        for (int l0 = 0; l0 < cn; l0 += NN_CHUNK / 2) {
            float ax = 0.f, ay = 0.f, az = 0.f;
            for (int l = l0; l < min(cn, l0 + NN_CHUNK / 2); ++l) {
                const int c = cb + l;
                const int ux = c % G, uy = (c / G) % G, uz = c / (G * G);
                if (abs(ux - cx) <= 1 && abs(uy - cy) <= 1 && abs(uz - cz) <= 1) continue;
                const float4 a = s_agg[2 * l], b = s_agg[2 * l + 1];
                if (a.w != 0.f) nn_term(x, a, a.w, eps2, ax, ay, az);
                if (b.w != 0.f) nn_term(x, b, b.w, eps2, ax, ay, az);
            }
            e[0] += ax; e[1] += ay; e[2] += az;
        }
    }
    if (!live) return;
    if (add) {
        const float4 q = E_out[i];
        e[0] += q.x; e[1] += q.y; e[2] += q.z;
    } else {
        e[0] += e_ext.x; e[1] += e_ext.y; e[2] += e_ext.z;
    }
    E_out[i] = make_float4((float)e[0], (float)e[1], (float)e[2], 0.f);
}

int obem_launch_nbody_nn(obem_ctx *c, const float4 *pos, const int32_t *n_dev, int n, int G, float eps2,
                         float4 *E_out, float3 e_ext, int add, cudaStream_t s)
{
    if (n <= 0) return OBEM_OK;
    if (G < 1 || G > OBEM_NN_GMAX) return obem_fail(c, OBEM_ERR_ARG, "nbody NN: grid %d outside 1..%d", G, OBEM_NN_GMAX);
    const int nc = G * G * G;
    const int nb = (n + NN_THREADS - 1) / NN_THREADS;
    nn_bbox_init_kernel<<<1, 32, 0, s>>>(c->nn_bbox);
    nn_bbox_kernel<<<nb < 1024 ? nb : 1024, NN_THREADS, 0, s>>>(pos, n_dev, n, c->nn_bbox);
    OBEM_CUDA(c, cudaMemsetAsync(c->nn_count, 0, sizeof(int32_t) * nc, s));
    nn_cell_kernel<<<nb, NN_THREADS, 0, s>>>(pos, n_dev, n, c->nn_bbox, G, c->nn_cell, c->nn_count);
    nn_scan_kernel<<<1, 1024, 0, s>>>(c->nn_count, nc, c->nn_start, c->nn_cursor);
    nn_scatter_kernel<<<nb, NN_THREADS, 0, s>>>(n_dev, n, c->nn_cell, G, c->nn_cursor, c->nn_sorted);
    nn_agg_kernel<<<(nc + 255) / 256, 256, 0, s>>>(pos, c->nn_start, c->nn_sorted, nc, c->nn_agg);
    nn_field_kernel<<<nb, NN_THREADS, 0, s>>>(pos, n_dev, n, c->nn_cell, c->nn_start, c->nn_sorted, c->nn_agg, G,
                                             eps2, E_out, e_ext, add);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}
